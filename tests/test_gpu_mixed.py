"""Mixed-precision path (cell-relative FP32 pair sums with Kahan compensation,
FP64 epilogue and hydrostatic split) against the FP64 oracle.

The mixed path computes the same definition in different arithmetic, so its
fields are not held to 1e-12: the tests bound the scaled error at levels the
FP32 sums support and record it. Its well-balance holds by construction
(the hydrostatic part never enters the FP32 sums), checked at 1e-12.
"""
import numpy as np
import pytest

import oracle
from paper_2608_22269_gb300 import scenes as S
from tests.helpers import scaled_err, scales

pytestmark = pytest.mark.gpu

MIXED_TOL = {"dudt": 2e-5, "dphidt": 2e-5, "dushift": 2e-5, "lambda": 2e-5}


def _sim(scene):
    from paper_2608_22269_gb300 import wbsph
    sim = wbsph.Sim(scene.params, precision=wbsph.MIXED, water_height=scene.water_height)
    sim.set_scene(scene)
    return sim


def _dynamic(scene, seed=5, amp=0.3):
    s = S.jitter(scene, 0.15, seed=seed)
    rng = np.random.default_rng(seed)
    f = s.type == 0
    s.u[:, f] = amp * rng.normal(size=(s.x.shape[0], f.sum()))
    s.phi[f] += 0.05 * rng.normal(size=f.sum())
    return s


CASES = [
    ("dam2d", lambda: S.dam_break_2d(dx=0.01, width=1.0, column=(0.3, 0.2))),
    ("topo_tri", lambda: S.topography_tank_2d("tri", dx=0.01, width=1.0, use_delta=1, use_pst=1,
                                              use_tic=1)),
    ("dam3d", lambda: S.dam_break_3d(dx=0.02, box=(0.4, 0.2, 0.3), column=(0.16, 0.2, 0.14))),
    ("slosh3d", lambda: S.sloshing_3d(dx=0.025, tank=(0.4, 0.2, 0.3), depth=0.15)),
]


@pytest.mark.parametrize("name,make", CASES)
def test_mixed_rates_close_to_oracle(name, make):
    sc = _dynamic(make())
    sim = _sim(sc)
    sim.eval_rates()
    m = oracle.mass(sc.params, sc.phi)
    r = oracle.stage_rates(sc.params, sc.x, sc.u, sc.phi, m, sc.type, sc.normal)
    sk = scales(sc.params, sc.water_height)
    f = sc.type == 0
    lam_o = r["lam"][f]
    # particles whose TIC branch may flip under FP32 rounding are excluded
    keep = np.abs(lam_o - sc.params["tic_lambda"]) > 1e-4
    errs = {
        "dudt": scaled_err(sim.get("dudt")[:, f][:, keep], r["dudt"][:, f][:, keep], sk["dudt"]),
        "dphidt": scaled_err(sim.get("dphidt")[f][keep], r["dphidt"][f][keep], sk["dphidt"]),
        "dushift": scaled_err(sim.get("dushift")[:, f][:, keep], r["dushift"][:, f][:, keep], sk["dushift"]),
        "lambda": scaled_err(sim.get("lambda")[f], lam_o, 1.0),
    }
    print(name, {k: f"{v:.2e}" for k, v in errs.items()})
    for k, v in errs.items():
        assert v <= MIXED_TOL[k], (name, k, v)


@pytest.mark.parametrize("name,make", CASES)
def test_mixed_step_close_to_oracle(name, make):
    sc = _dynamic(make(), amp=0.2)
    sim = _sim(sc)
    sim.step(2)
    st = oracle.State(sc)
    st.step(2)
    sk = scales(sc.params, sc.water_height)
    ex = scaled_err(sim.get("x"), st.x, sk["x"])
    eu = scaled_err(sim.get("u"), st.u, sk["u"])
    ep = scaled_err(sim.get("phi"), st.phi, sk["phi"])
    print(name, f"x {ex:.2e} u {eu:.2e} phi {ep:.2e}")
    assert ex <= 1e-9 and eu <= 1e-6 and ep <= 1e-6


def test_mixed_closed_tank_is_well_balanced():
    sc = S.hydrostatic_tank_2d(lid=True)
    sim = _sim(sc)
    sim.step(200)
    u = sim.get("u")[:, sc.type == 0]
    assert np.abs(u).max() <= 1e-12


@pytest.mark.parametrize("kind", ["flat", "rect", "gauss"])
def test_mixed_hydrostatic_rates_vanish(kind):
    sc = S.topography_tank_2d(kind, dx=0.01, width=1.0)
    sim = _sim(sc)
    sim.eval_rates()
    f = sc.type == 0
    assert np.abs(sim.get("dudt")[:, f]).max() <= 1e-12 * 9.81


def test_mixed_3d_hydrostatic_box_rates_vanish():
    sc = S.box_tank(3, (0.3, 0.2, 0.25), 0.01, lambda g: g[2] < 0.2, 0.2)
    sim = _sim(sc)
    sim.eval_rates()
    f = sc.type == 0
    assert np.abs(sim.get("dudt")[:, f]).max() <= 1e-12 * 9.81


def test_mixed_lone_particle_falls_exactly():
    """A lone fluid particle has no neighbours: its renormalisation matrix is
    zero, the TIC branch takes the conservative gradient (zero), and the
    mixed path's FP64 epilogue gives DU/Dt = G exactly, so the SSP-RK2 step
    reproduces the free fall to rounding."""
    p = S.default_params(2, 0.01, 30.0, use_tic=1, domain_min=[-5, -20, 0], domain_max=[5, 5, 1])
    sc = S.Scene(p, np.array([[0.1], [0.2]]), np.array([[0.5], [1.0]]), np.zeros(1),
                 np.zeros(1, np.uint8), np.zeros((2, 1)))
    sim = _sim(sc)
    sim.step(50)
    t = sim.stats()["t"]
    x = sim.get("x")[:, 0]
    assert abs(x[0] - (0.1 + 0.5 * t)) < 1e-14
    assert abs(x[1] - (0.2 + t - 0.5 * 9.81 * t * t)) < 1e-13


def test_mixed_empty_set_steps():
    """No particles: the single-sort step (one eager, then the captured
    graphs) launches nothing that needs a particle and reports n = 0."""
    p = S.default_params(2, 0.01, 30.0, use_tic=1, domain_min=[-5, -20, 0], domain_max=[5, 5, 1])
    empty = S.Scene(p, np.zeros((2, 0)), np.zeros((2, 0)), np.zeros(0), np.zeros(0, np.uint8),
                    np.zeros((2, 0)))
    sim = _sim(empty)
    sim.step(3)
    sim.sync()
    assert sim.stats()["n"] == 0


def test_mixed_wall_particles_only():
    """Walls and no fluid: no kept lists and no pair pass; the walls keep
    their positions and, with no fluid particle to copy, their phi."""
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


def _mixed_cell(p):
    """Cell size of the mixed path: 2h widened by the skin of its kept lists,
    3 CFL dx 0.3 / 1.3 (the move of two particles in one stage at Mach 0.3)."""
    return 2.0 * p["h_over_dx"] * p["dx"] + 3.0 * p["cfl"] * p["dx"] * 0.3 / 1.3


def test_mixed_rejects_grids_beyond_its_packed_cell_coordinates():
    """The mixed path packs cell coordinates in 11/11/10 bits: a grid with
    more than 2048 cells on an axis is refused at the first step with
    WBSPH_E_INVAL (the FP64 path has no such limit)."""
    from paper_2608_22269_gb300 import wbsph
    p = S.default_params(2, 0.01, 30.0, domain_min=[-5, -60, 0], domain_max=[5, 5, 1])
    sc = S.Scene(p, np.array([[0.1], [0.2]]), np.zeros((2, 1)), np.zeros(1), np.zeros(1, np.uint8),
                 np.zeros((2, 1)))
    assert int(np.floor(65.0 / _mixed_cell(p))) + 1 > 2048
    sim = _sim(sc)
    with pytest.raises(wbsph.WbsphError) as ei:
        sim.step(1)
    assert ei.value.code == -1


def test_mixed_kept_lists_in_a_fast_flow():
    """The mixed step sorts once and keeps stage 1's lists (radius 2h +
    3 dt U_max) for stage 2. In a flow thrown at 2.5 m/s (Mach 0.14), where
    particles move furthest between the stages, four steps stay as close to
    the oracle as two steps of the slow case above: a pair missing from the
    kept lists would show at the 1e-3 level."""
    sc = S.jitter(S.dam_break_2d(dx=0.01, width=0.8, column=(0.4, 0.25)), 0.3, seed=3)
    f = sc.type == 0
    sc.u[0, f] = 2.5
    sc.u[1, f] = 0.5 * np.random.default_rng(1).normal(size=f.sum())
    sim = _sim(sc)
    sim.step(4)
    st = oracle.State(sc)
    st.step(4)
    sk = scales(sc.params, sc.water_height)
    ex = scaled_err(sim.get("x"), st.x, sk["x"])
    eu = scaled_err(sim.get("u"), st.u, sk["u"])
    ep = scaled_err(sim.get("phi"), st.phi, sk["phi"])
    print(f"fast flow: x {ex:.2e} u {eu:.2e} phi {ep:.2e}")
    assert ex <= 1e-9 and eu <= 1e-6 and ep <= 1e-6


def test_mixed_kept_lists_report_a_move_beyond_the_skin():
    """A fixed time step that lets a particle move further in one stage than
    the widened cells allow (3 dt U > 3 CFL dx 0.3 / 1.3) is reported as
    WBSPH_E_CAPACITY at the next synchronising call."""
    from paper_2608_22269_gb300 import wbsph
    sc = S.dam_break_2d(dx=0.01, width=0.8, column=(0.4, 0.25))
    f = sc.type == 0
    sc.u[0, f] = 2.0
    p = dict(sc.params, fixed_dt=5e-4)
    assert 3 * 5e-4 * 2.0 > _mixed_cell(p) - 2.0 * p["h_over_dx"] * p["dx"]
    sim = wbsph.Sim(p, precision=wbsph.MIXED, water_height=sc.water_height)
    sim.set_scene(sc)
    with pytest.raises(wbsph.WbsphError) as ei:
        sim.step(1)
        sim.sync()
    assert ei.value.code == -9 and "skin" in str(ei.value)
