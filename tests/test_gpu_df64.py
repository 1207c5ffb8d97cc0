"""Double-float pair pass (pairs of FP32 on offsets in cell units, the
hydrostatic split, FP64 epilogue, the exact FP64 neighbour lists) against
the FP64 oracle, held to the bar of the FP64 path: within 1e-12 of the
natural field scale (max |a - b| / max(max |b|, scale)) for the rates of a
stage and the fields after SSP-RK2 steps; the hydrostatic tanks at rest to
1e-12. The same scenes as the FP64 parity tests, plus the wall options, the
general shifting exponent, the edge cases and the grid limit of the packed
cell coordinates.
"""
import numpy as np
import pytest

import oracle
from paper_2608_22269_gb300 import scenes as S
from tests.helpers import dynamic, scaled_err, scales

pytestmark = pytest.mark.gpu
TOL = 1e-12


def _sim(scene):
    from paper_2608_22269_gb300 import wbsph
    sim = wbsph.Sim(scene.params, precision=wbsph.DF64, water_height=scene.water_height)
    sim.set_scene(scene)
    return sim


def _body(dim, bc):
    if dim == 2:
        sc = dynamic(S.moving_body(2, body_u=(0.5, 0.1)), amp=0.2)
    else:
        sc = dynamic(S.moving_body(3, dx=0.02, tank=(0.6, 0.3, 0.4), depth=0.3, body=(0.1, 0.1, 0.1),
                                   center=(0.2, 0.15, 0.15), body_u=(0.5, 0.0, 0.05)), amp=0.2)
    sc.params.update(wall_bc=bc)
    return sc


SMALL = [
    ("dam2d", lambda: dynamic(S.dam_break_2d(dx=0.01, width=1.0, column=(0.3, 0.2)))),
    ("topo_gauss", lambda: dynamic(S.topography_tank_2d("gauss", dx=0.01, width=1.0, use_delta=1,
                                                        use_pst=1, use_tic=1))),
    ("dam3d", lambda: dynamic(S.dam_break_3d(dx=0.02, box=(0.4, 0.2, 0.3), column=(0.16, 0.2, 0.14)))),
    ("slosh3d", lambda: dynamic(S.sloshing_3d(dx=0.025, tank=(0.4, 0.2, 0.3), depth=0.15))),
]
WALLS = [
    ("body2d_noslip", lambda: _body(2, 1)),
    ("body3d_slip", lambda: _body(3, 0)),
    ("body3d_noslip", lambda: _body(3, 1)),
]


def _rates_errs(sc, sim):
    sim.eval_rates()
    m = oracle.mass(sc.params, sc.phi)
    r = oracle.stage_rates(sc.params, sc.x, sc.u, sc.phi, m, sc.type, sc.normal)
    sk = scales(sc.params, sc.water_height)
    f = sc.type == 0
    return {
        "dudt": scaled_err(sim.get("dudt")[:, f], r["dudt"][:, f], sk["dudt"]),
        "dphidt": scaled_err(sim.get("dphidt")[f], r["dphidt"][f], sk["dphidt"]),
        "dushift": scaled_err(sim.get("dushift")[:, f], r["dushift"][:, f], sk["dushift"]),
        "lambda": scaled_err(sim.get("lambda")[f], r["lam"][f], 1.0),
        "u_walls": scaled_err(sim.get("u"), r["u"], sk["u"]),
        "phi_walls": scaled_err(sim.get("phi"), r["phi"], sk["phi"]),
    }


def _check(errs, tag):
    print(tag, {k: f"{v:.2e}" for k, v in errs.items()})
    for k, v in errs.items():
        assert v <= TOL, (tag, k, v)


@pytest.mark.parametrize("name,make", SMALL + WALLS)
def test_df64_stage_rates_match_oracle(name, make):
    sc = make()
    _check(_rates_errs(sc, _sim(sc)), name)


def test_df64_long_candidate_lists():
    """h = 1.48 dx in 3D: 90 to 110 neighbours per particle."""
    sc = dynamic(S.dam_break_3d(dx=0.02, box=(0.4, 0.2, 0.3), column=(0.16, 0.2, 0.14), h_over_dx=1.48))
    _check(_rates_errs(sc, _sim(sc)), "h1.48")


def test_df64_tait_eos_and_general_shifting_exponent():
    """Tait EOS, and a shifting exponent n = 3 (the FP64 power per pair
    replaces the double-float fourth power)."""
    sc = dynamic(S.dam_break_2d(dx=0.01, width=1.0, column=(0.3, 0.2), eos=1))
    _check(_rates_errs(sc, _sim(sc)), "tait")
    sc = dynamic(S.topography_tank_2d("gauss", dx=0.01, width=1.0, use_delta=1, use_pst=1, use_tic=1))
    sc.params.update(pst_n=3.0)
    _check(_rates_errs(sc, _sim(sc)), "pst_n3")


@pytest.mark.parametrize("name,make", SMALL + WALLS[1:2])
@pytest.mark.parametrize("nsteps", [1, 3])
def test_df64_fields_after_steps_match_oracle(name, make, nsteps):
    sc = make()
    sim = _sim(sc)
    sim.step(nsteps)
    st = oracle.State(sc)
    st.step(nsteps)
    assert abs(sim.stats()["t"] - st.t) <= 4e-15 * max(st.t, 1e-30)
    sk = scales(sc.params, sc.water_height)
    f = sc.type == 0
    _check({"x": scaled_err(sim.get("x"), st.x, sk["x"]),
            "u": scaled_err(sim.get("u"), st.u, sk["u"]),
            "phi": scaled_err(sim.get("phi"), st.phi, sk["phi"]),
            "dudt": scaled_err(sim.get("dudt")[:, f], st.dudt[:, f], sk["dudt"])}, f"{name} x{nsteps}")


def test_df64_forced_tank_at_nonzero_time():
    sc = dynamic(S.sloshing_3d(dx=0.025, tank=(0.4, 0.2, 0.3), depth=0.15, amp=0.05, period=0.01))
    sim = _sim(sc)
    sim.step(2)
    st = oracle.State(sc)
    st.step(2)
    sk = scales(sc.params, sc.water_height)
    _check({"u": scaled_err(sim.get("u"), st.u, sk["u"]),
            "phi": scaled_err(sim.get("phi"), st.phi, sk["phi"])}, "forced")


def test_df64_hydrostatic_closed_tank_200_steps():
    sc = S.hydrostatic_tank_2d(lid=True)
    sim = _sim(sc)
    sim.step(200)
    u = sim.get("u")[:, sc.type == 0]
    assert np.abs(u).max() <= 1e-12


@pytest.mark.parametrize("eos", [0, 1])
def test_df64_hydrostatic_open_tank_100_steps(eos):
    sc = S.hydrostatic_tank_2d(eos=eos)
    sim = _sim(sc)
    sim.step(100)
    u = sim.get("u")[:, sc.type == 0]
    assert np.sqrt((u * u).sum(0)).max() <= 1e-12


@pytest.mark.parametrize("kind", ["flat", "rect", "tri", "gauss"])
def test_df64_hydrostatic_rates_vanish_on_topographies(kind):
    sc = S.topography_tank_2d(kind, dx=0.01, width=1.0)
    sim = _sim(sc)
    sim.eval_rates()
    f = sc.type == 0
    assert np.abs(sim.get("dudt")[:, f]).max() <= 1e-12 * 9.81
    assert np.abs(sim.get("dphidt")[f]).max() <= 1e-9


def test_df64_3d_hydrostatic_box_rates_vanish():
    sc = S.box_tank(3, (0.3, 0.2, 0.25), 0.01, lambda g: g[2] < 0.2, 0.2)
    sim = _sim(sc)
    sim.eval_rates()
    f = sc.type == 0
    assert np.abs(sim.get("dudt")[:, f]).max() <= 1e-12 * 9.81


def test_df64_lone_particle_falls_exactly():
    """No neighbours: L = 0, the TIC branch takes the conservative gradient
    (zero) and the FP64 epilogue gives DU/Dt = G exactly."""
    p = S.default_params(2, 0.01, 30.0, use_tic=1, domain_min=[-5, -20, 0], domain_max=[5, 5, 1])
    sc = S.Scene(p, np.array([[0.1], [0.2]]), np.array([[0.5], [1.0]]), np.zeros(1),
                 np.zeros(1, np.uint8), np.zeros((2, 1)))
    sim = _sim(sc)
    sim.step(50)
    t = sim.stats()["t"]
    x = sim.get("x")[:, 0]
    assert abs(x[0] - (0.1 + 0.5 * t)) < 1e-14
    assert abs(x[1] - (0.2 + t - 0.5 * 9.81 * t * t)) < 1e-13


def test_df64_empty_set_steps():
    """No particles: the single-sort step (one eager, then the captured
    graphs) launches nothing that needs a particle and reports n = 0."""
    p = S.default_params(2, 0.01, 30.0, use_tic=1, domain_min=[-5, -20, 0], domain_max=[5, 5, 1])
    empty = S.Scene(p, np.zeros((2, 0)), np.zeros((2, 0)), np.zeros(0), np.zeros(0, np.uint8),
                    np.zeros((2, 0)))
    sim = _sim(empty)
    sim.step(3)
    sim.sync()
    assert sim.stats()["n"] == 0


def test_df64_wall_particles_only():
    sc = S.dam_break_2d(dx=0.02, width=1.0, column=(0.3, 0.2))
    walls = sc.type != 0
    only = S.Scene(dict(sc.params), sc.x[:, walls].copy(), sc.u[:, walls].copy(), sc.phi[walls].copy(),
                   sc.type[walls].copy(), sc.normal[:, walls].copy())
    sim = _sim(only)
    sim.step(2)
    sim.sync()
    assert sim.stats()["n_fluid"] == 0
    assert np.array_equal(sim.get("x"), only.x)
    assert np.array_equal(sim.get("phi"), only.phi)


def test_df64_rejects_grids_beyond_its_packed_cell_coordinates():
    """More than 2048 cells on an axis (cells of 2h plus the kept lists'
    skin, 3 CFL dx 0.3 / 1.3): refused with WBSPH_E_INVAL."""
    from paper_2608_22269_gb300 import wbsph
    p = S.default_params(2, 0.01, 30.0, domain_min=[-5, -60, 0], domain_max=[5, 5, 1])
    R = 2.0 * p["h_over_dx"] * p["dx"] + 3.0 * p["cfl"] * p["dx"] * 0.3 / 1.3
    assert int(np.floor(65.0 / R)) + 1 > 2048
    sc = S.Scene(p, np.array([[0.1], [0.2]]), np.zeros((2, 1)), np.zeros(1), np.zeros(1, np.uint8),
                 np.zeros((2, 1)))
    sim = _sim(sc)
    with pytest.raises(wbsph.WbsphError) as ei:
        sim.step(1)
    assert ei.value.code == -1


def test_df64_counts_the_same_pairs_as_fp64():
    """The double-float step keeps stage 1's lists (radius 2h + 3 dt U*) for
    stage 2 and applies Algorithm 1's test in the pass; the FP64 step builds
    exact lists per stage. Both count the same pairs."""
    from paper_2608_22269_gb300 import wbsph
    sc = SMALL[2][1]()
    a = _sim(sc)
    a.step(1)
    b = wbsph.Sim(sc.params, precision=wbsph.FP64, water_height=sc.water_height)
    b.set_scene(sc)
    b.step(1)
    assert a.stats()["pairs"] == b.stats()["pairs"] > 0


def test_df64_kept_lists_in_a_fast_flow():
    """Particles thrown at 2.5 m/s (Mach 0.14) move furthest between the
    stages; the kept lists and the pass's exact test still give the oracle's
    fields within the FP64 bar after four steps."""
    sc = S.jitter(S.dam_break_2d(dx=0.01, width=0.8, column=(0.4, 0.25)), 0.3, seed=3)
    f = sc.type == 0
    sc.u[0, f] = 2.5
    sc.u[1, f] = 0.5 * np.random.default_rng(1).normal(size=f.sum())
    sim = _sim(sc)
    sim.step(4)
    st = oracle.State(sc)
    st.step(4)
    sk = scales(sc.params, sc.water_height)
    _check({"x": scaled_err(sim.get("x"), st.x, sk["x"]),
            "u": scaled_err(sim.get("u"), st.u, sk["u"]),
            "phi": scaled_err(sim.get("phi"), st.phi, sk["phi"]),
            "dudt": scaled_err(sim.get("dudt")[:, f], st.dudt[:, f], sk["dudt"])}, "fast flow x4")
