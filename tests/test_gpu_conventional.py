"""The conventional WCSPH foil on the GPU (csrc/pair_conventional.cu)
against the oracle's, and the hydrostatic contrast of Sec. 4.1: on the same
tanks at rest, the well-balanced scheme keeps the spurious velocity at
rounding level and the conventional one does not."""
import numpy as np
import pytest

import oracle
from paper_2608_22269_gb300 import scenes as S
from tests.helpers import dynamic, scaled_err, scales

pytestmark = pytest.mark.gpu
TOL = 1e-12


def _conv(sc):
    sc = sc.copy()
    sc.params.update(scheme=1, use_delta=0, use_pst=0, use_tic=0)
    return sc


def _sim(sc):
    from paper_2608_22269_gb300 import wbsph
    sim = wbsph.Sim(sc.params, water_height=sc.water_height)
    sim.set_scene(sc)
    return sim


CASES = [
    ("dam2d", lambda: dynamic(S.dam_break_2d(dx=0.01, width=1.0, column=(0.3, 0.2)))),
    ("tank2d_tait", lambda: dynamic(S.hydrostatic_tank_2d(dx=0.02, eos=1), amp=0.1)),
    ("dam3d", lambda: dynamic(S.dam_break_3d(dx=0.02, box=(0.4, 0.2, 0.3), column=(0.16, 0.2, 0.14)))),
]


@pytest.mark.parametrize("name,make", CASES)
def test_conventional_rates_match_oracle(name, make):
    sc = _conv(make())
    sim = _sim(sc)
    sim.eval_rates()
    m = oracle.mass(sc.params, sc.phi)
    r = oracle.stage_rates(sc.params, sc.x, sc.u, sc.phi, m, sc.type, sc.normal)
    sk = scales(sc.params, sc.water_height)
    f = sc.type == 0
    assert scaled_err(sim.get("dudt")[:, f], r["dudt"][:, f], sk["dudt"]) <= TOL
    assert scaled_err(sim.get("dphidt")[f], r["dphidt"][f], sk["dphidt"]) <= TOL
    assert np.all(sim.get("dushift") == 0.0)


@pytest.mark.parametrize("name,make", CASES)
def test_conventional_steps_match_oracle(name, make):
    sc = _conv(make())
    sim = _sim(sc)
    sim.step(3)
    st = oracle.State(sc).step(3)
    sk = scales(sc.params, sc.water_height)
    assert scaled_err(sim.get("x"), st.x, sk["x"]) <= TOL
    assert scaled_err(sim.get("u"), st.u, sk["u"]) <= TOL
    assert scaled_err(sim.get("phi"), st.phi, sk["phi"]) <= TOL


def _l2(sim, sc):
    """L2 spurious velocity sqrt(sum |U|^2 V / sum V) over fluid (Sec. 4.1)."""
    f = sc.type == 0
    u = sim.get("u")[:, f]
    v = sim.get("vol")[f]
    return float(np.sqrt(((u ** 2).sum(0) * v).sum() / v.sum()))


@pytest.mark.parametrize("kind,steps", [("flat", 100), ("rect", 100), ("tri", 100), ("gauss", 100),
                                        ("closed", 400)])
def test_hydrostatic_contrast(kind, steps):
    """Tanks at rest, linear EOS, stabilisers off, dx = 0.01: open tanks over
    flat, rectangular, triangular and Gaussian bottoms for 100 steps (beyond
    that the printed scheme's rounding-seeded free-surface mode grows), and
    the closed tank of the paper's setting (water up to the lid) for 400.
    The well-balanced L2 spurious velocity stays at rounding level; the
    conventional scheme's reaches the 1e-3 level the paper reports for it
    (the oracle gives 2.0e-3 and 1.8e-3 on these cases)."""
    if kind == "flat":
        base = S.hydrostatic_tank_2d(dx=0.01, eos=0)
    elif kind == "closed":
        base = S.hydrostatic_tank_2d(dx=0.01, eos=0, lid=True)
    else:
        base = S.topography_tank_2d(kind, dx=0.01, width=1.0, eos=0)
    base.params.update(use_delta=0, use_pst=0, use_tic=0)
    out = {}
    for scheme in (0, 1):
        sc = base.copy()
        sc.params.update(scheme=scheme)
        sim = _sim(sc)
        sim.step(steps)
        out[scheme] = _l2(sim, sc)
    print(kind, "L2 spurious velocity after", steps, "steps: well-balanced", out[0], "conventional", out[1])
    assert out[0] <= 1e-12
    assert out[1] >= 1e-4
