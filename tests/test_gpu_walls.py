"""No-slip walls (Eq. velBn) and rigid bodies of wall particles translating
with a prescribed velocity, on the GPU against the oracle."""
import numpy as np
import pytest

import oracle
from paper_2608_22269_gb300 import scenes as S
from tests.helpers import dynamic, scaled_err, scales

pytestmark = pytest.mark.gpu
TOL = 1e-12


def _sim(sc, precision=0):
    from paper_2608_22269_gb300 import wbsph
    sim = wbsph.Sim(sc.params, precision=precision, water_height=sc.water_height)
    sim.set_scene(sc)
    return sim


def _body2d(bc):
    sc = dynamic(S.moving_body(2, body_u=(0.5, 0.1)), amp=0.2)
    sc.params.update(wall_bc=bc)
    return sc


def _body3d(bc):
    sc = dynamic(S.moving_body(3, dx=0.02, tank=(0.6, 0.3, 0.4), depth=0.3, body=(0.1, 0.1, 0.1),
                               center=(0.2, 0.15, 0.15), body_u=(0.5, 0.0, 0.05)), amp=0.2)
    sc.params.update(wall_bc=bc)
    return sc


def _dam_noslip():
    sc = dynamic(S.dam_break_2d(dx=0.01, width=1.0, column=(0.3, 0.2)))
    sc.params.update(wall_bc=1)
    return sc


CASES = [("body2d_slip", lambda: _body2d(0)), ("body2d_noslip", lambda: _body2d(1)),
         ("body3d_slip", lambda: _body3d(0)), ("body3d_noslip", lambda: _body3d(1)),
         ("dam2d_noslip", _dam_noslip)]


@pytest.mark.parametrize("name,make", CASES)
def test_wall_options_rates_match_oracle(name, make):
    sc = make()
    sim = _sim(sc)
    sim.eval_rates()
    m = oracle.mass(sc.params, sc.phi)
    r = oracle.stage_rates(sc.params, sc.x, sc.u, sc.phi, m, sc.type, sc.normal)
    sk = scales(sc.params, sc.water_height)
    f = sc.type == 0
    assert scaled_err(sim.get("dudt")[:, f], r["dudt"][:, f], sk["dudt"]) <= TOL
    assert scaled_err(sim.get("dphidt")[f], r["dphidt"][f], sk["dphidt"]) <= TOL
    assert scaled_err(sim.get("dushift")[:, f], r["dushift"][:, f], sk["dushift"]) <= TOL
    assert scaled_err(sim.get("u"), r["u"], sk["u"]) <= TOL  # wall velocities after the update
    assert scaled_err(sim.get("phi"), r["phi"], sk["phi"]) <= TOL


@pytest.mark.parametrize("name,make", CASES)
def test_wall_options_steps_match_oracle(name, make):
    sc = make()
    sim = _sim(sc)
    sim.step(3)
    st = oracle.State(sc).step(3)
    sk = scales(sc.params, sc.water_height)
    assert abs(sim.stats()["t"] - st.t) <= 4e-15 * st.t
    assert scaled_err(sim.get("x"), st.x, sk["x"]) <= TOL
    assert scaled_err(sim.get("u"), st.u, sk["u"]) <= TOL
    assert scaled_err(sim.get("phi"), st.phi, sk["phi"]) <= TOL
    b = sc.type == 2
    if b.any():  # the body moved rigidly by body_u t
        want = sc.x[:, b] + np.asarray(sc.params["body_u"][:sc.x.shape[0]])[:, None] * st.t
        assert np.abs(sim.get("x")[:, b] - want).max() <= 1e-13


def test_mixed_path_with_a_moving_body():
    """The mixed path on the 2D body scene: its rates within the mixed
    tolerance of the oracle (particles near the TIC switch excluded)."""
    from paper_2608_22269_gb300 import wbsph
    sc = _body2d(1)
    sim = _sim(sc, wbsph.MIXED)
    sim.eval_rates()
    m = oracle.mass(sc.params, sc.phi)
    r = oracle.stage_rates(sc.params, sc.x, sc.u, sc.phi, m, sc.type, sc.normal)
    sk = scales(sc.params, sc.water_height)
    f = sc.type == 0
    keep = np.abs(r["lam"][f] - sc.params["tic_lambda"]) > 1e-4
    assert scaled_err(sim.get("dudt")[:, f][:, keep], r["dudt"][:, f][:, keep], sk["dudt"]) <= 2e-5
    assert scaled_err(sim.get("dphidt")[f][keep], r["dphidt"][f][keep], sk["dphidt"]) <= 2e-5
