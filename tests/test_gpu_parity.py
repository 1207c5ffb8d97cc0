"""GPU (CUDA path through the C-ABI) against the FP64 CPU oracle.

Bit-exact: cell keys, sort permutation, neighbour sets. Within 1e-12 of the
natural field scale (max |a - b| / max(max |b|, scale)): rates of a stage and
fields after SSP-RK2 steps. Sizes span several warps/tiles and ragged tails;
edge cases cover an empty set, a lone particle and the error paths.
"""
import numpy as np
import pytest

import oracle
from paper_2608_22269_gb300 import scenes as S
from tests.helpers import scaled_err, scales

pytestmark = pytest.mark.gpu
TOL = 1e-12


def _sim(scene, precision=0):
    from paper_2608_22269_gb300 import wbsph
    sim = wbsph.Sim(scene.params, precision=precision, water_height=scene.water_height)
    sim.set_scene(scene)
    return sim


def _dynamic(scene, seed=5, amp=0.3):
    """Jittered positions, random fluid velocities and potential noise."""
    s = S.jitter(scene, 0.15, seed=seed)
    rng = np.random.default_rng(seed)
    f = s.type == 0
    s.u[:, f] = amp * rng.normal(size=(s.x.shape[0], f.sum()))
    s.phi[f] += 0.05 * rng.normal(size=f.sum())
    return s


SMALL = [
    ("dam2d", lambda: S.dam_break_2d(dx=0.01, width=1.0, column=(0.3, 0.2))),
    ("topo_gauss", lambda: S.topography_tank_2d("gauss", dx=0.01, width=1.0, use_delta=1,
                                                use_pst=1, use_tic=1)),
    ("dam3d", lambda: S.dam_break_3d(dx=0.02, box=(0.4, 0.2, 0.3), column=(0.16, 0.2, 0.14))),
    ("slosh3d", lambda: S.sloshing_3d(dx=0.025, tank=(0.4, 0.2, 0.3), depth=0.15)),
]


@pytest.mark.parametrize("name,make", SMALL + [("box3d", lambda: S.random_box(3001, 3, 0.2, 0.01)),
                                              ("box2d", lambda: S.random_box(2500, 2, 0.3, 0.01))])
def test_keys_and_sort_order_bitexact(name, make):
    sc = make()
    sim = _sim(sc)
    sim.build_neighbors()
    keys, ids = sim.cell_keys()
    ok = oracle.cell_keys(sc.params, sc.x)
    perm = oracle.sort_by_key(ok)
    assert np.array_equal(keys, ok[perm])
    assert np.array_equal(ids, perm)


@pytest.mark.parametrize("name,make", SMALL + [("box3d", lambda: S.random_box(3001, 3, 0.2, 0.01)),
                                              ("box2d", lambda: S.random_box(2500, 2, 0.3, 0.01))])
def test_neighbour_sets_bitexact(name, make):
    sc = _dynamic(make()) if name not in ("box3d", "box2d") else make()
    sim = _sim(sc)
    row, col = sim.neighbors()
    orow, ocol = oracle.neighbors(sc.params, sc.x)
    assert np.array_equal(row, orow)
    assert np.array_equal(col, ocol)


def _compare_rates(sc, sim, tag):
    sim.eval_rates()
    m = oracle.mass(sc.params, sc.phi)
    r = oracle.stage_rates(sc.params, sc.x, sc.u, sc.phi, m, sc.type, sc.normal)
    sk = scales(sc.params, sc.water_height)
    f = sc.type == 0
    errs = {
        "dudt": scaled_err(sim.get("dudt")[:, f], r["dudt"][:, f], sk["dudt"]),
        "dphidt": scaled_err(sim.get("dphidt")[f], r["dphidt"][f], sk["dphidt"]),
        "dushift": scaled_err(sim.get("dushift")[:, f], r["dushift"][:, f], sk["dushift"]),
        "phi_dummy": scaled_err(sim.get("phi"), r["phi"], sk["phi"]),
        "u_dummy": scaled_err(sim.get("u"), r["u"], sk["u"]),
    }
    lam_g, lam_o = sim.get("lambda")[f], r["lam"][f]
    errs["lambda"] = scaled_err(lam_g, lam_o, 1.0)
    for k, v in errs.items():
        assert v <= TOL, (tag, k, v)
    return errs


@pytest.mark.parametrize("name,make", SMALL)
def test_stage_rates_match_oracle(name, make):
    sc = _dynamic(make())
    sim = _sim(sc)
    _compare_rates(sc, sim, name)


def test_long_candidate_lists_match_oracle():
    """h = 1.48 dx in 3D gives 90 to 110 neighbours per particle: list
    entries past the shared-memory staging depth take the direct-store path
    of the candidate-list kernel."""
    sc = _dynamic(S.dam_break_3d(dx=0.02, box=(0.4, 0.2, 0.3), column=(0.16, 0.2, 0.14),
                                 h_over_dx=1.48))
    sim = _sim(sc)
    row, _ = sim.neighbors()
    assert np.diff(row).max() > 100
    _compare_rates(sc, sim, "h1.48")


@pytest.mark.parametrize("name,make", SMALL)
@pytest.mark.parametrize("nsteps", [1, 3])
def test_fields_after_steps_match_oracle(name, make, nsteps):
    sc = _dynamic(make(), amp=0.2)
    sim = _sim(sc)
    sim.step(nsteps)
    st = oracle.State(sc)
    st.step(nsteps)
    stats = sim.stats()
    assert abs(stats["t"] - st.t) <= 1e-15 * max(st.t, 1e-30) * 4
    sk = scales(sc.params, sc.water_height)
    assert scaled_err(sim.get("x"), st.x, sk["x"]) <= TOL
    assert scaled_err(sim.get("u"), st.u, sk["u"]) <= TOL
    assert scaled_err(sim.get("phi"), st.phi, sk["phi"]) <= TOL
    f = sc.type == 0
    assert scaled_err(sim.get("dudt")[:, f], st.dudt[:, f], sk["dudt"]) <= TOL


def test_tait_and_linear_eos_rates():
    for eos in (0, 1):
        sc = _dynamic(S.dam_break_2d(dx=0.01, width=1.0, column=(0.3, 0.2), eos=eos))
        _compare_rates(sc, _sim(sc), f"eos{eos}")


def test_forced_tank_rates_at_nonzero_time():
    sc = _dynamic(S.sloshing_3d(dx=0.025, tank=(0.4, 0.2, 0.3), depth=0.15, amp=0.05, period=0.01))
    sim = _sim(sc)
    sim.step(2)
    st = oracle.State(sc)
    st.step(2)
    sk = scales(sc.params, sc.water_height)
    assert scaled_err(sim.get("u"), st.u, sk["u"]) <= TOL
    assert scaled_err(sim.get("phi"), st.phi, sk["phi"]) <= TOL


def test_hydrostatic_closed_tank_200_steps():
    sc = S.hydrostatic_tank_2d(lid=True)
    sim = _sim(sc)
    sim.step(200)
    u = sim.get("u")[:, sc.type == 0]
    assert np.abs(u).max() <= 1e-12


@pytest.mark.parametrize("eos", [0, 1])
def test_hydrostatic_open_tank_100_steps(eos):
    sc = S.hydrostatic_tank_2d(eos=eos)
    sim = _sim(sc)
    sim.step(100)
    u = sim.get("u")[:, sc.type == 0]
    assert np.sqrt((u * u).sum(0)).max() <= 1e-12


@pytest.mark.parametrize("kind", ["flat", "rect", "tri", "gauss"])
def test_hydrostatic_rates_vanish_on_topographies(kind):
    sc = S.topography_tank_2d(kind, dx=0.01, width=1.0)
    sim = _sim(sc)
    sim.eval_rates()
    f = sc.type == 0
    assert np.abs(sim.get("dudt")[:, f]).max() <= 1e-12 * 9.81
    assert np.abs(sim.get("dphidt")[f]).max() <= 1e-9


def test_lone_particle_and_empty_set():
    from paper_2608_22269_gb300 import wbsph
    p = S.default_params(2, 0.01, 30.0, use_tic=1, domain_min=[-5, -50, 0], domain_max=[5, 5, 1])
    sc = S.Scene(p, np.array([[0.1], [0.2]]), np.array([[0.5], [1.0]]), np.zeros(1),
                 np.zeros(1, np.uint8), np.zeros((2, 1)))
    sim = _sim(sc)
    sim.step(50)
    t = sim.stats()["t"]
    x = sim.get("x")[:, 0]
    assert abs(x[0] - (0.1 + 0.5 * t)) < 1e-14
    assert abs(x[1] - (0.2 + t - 0.5 * 9.81 * t * t)) < 1e-13
    empty = S.Scene(p, np.zeros((2, 0)), np.zeros((2, 0)), np.zeros(0), np.zeros(0, np.uint8),
                    np.zeros((2, 0)))
    sim0 = _sim(empty)
    sim0.step(3)
    sim0.sync()
    assert sim0.stats()["n"] == 0
    p2 = dict(p, use_tic=0)
    sim2 = _sim(S.Scene(p2, sc.x, sc.u, sc.phi, sc.type, sc.normal))
    sim2.step(1)
    with pytest.raises(wbsph.WbsphError) as ei:
        sim2.sync()
    assert ei.value.code == -5


@pytest.mark.parametrize("dim,n_dense,n_sparse,side,precision", [
    (2, 2000, 250, 0.2, 0), (2, 2000, 250, 0.2, 1), (2, 2000, 250, 0.2, 2), (3, 4000, 600, 0.1, 0)])
def test_list_overflow_is_reported_and_the_handle_recovers(dim, n_dense, n_sparse, side, precision):
    """Particles packed far below dx: about 106 neighbours per particle in 2D
    (a list holds 48) and about 290 in 3D (a list holds 128). The lists stop
    at their capacity and the rates are not the method's, so the next
    synchronising call returns WBSPH_E_CAPACITY naming the overflow, ahead
    of anything the truncated sums may have caused. Loading a sparse set
    (about 13 and 44 neighbours) clears it: the rates are then finite."""
    from paper_2608_22269_gb300 import wbsph
    dense = S.random_box(n_dense, dim, side=side, dx=0.01, seed=70 + dim, on_faces=False)
    sparse = S.random_box(n_sparse, dim, side=side, dx=0.01, seed=80 + dim, on_faces=False)
    p = dict(dense.params, use_tic=1)
    sim = wbsph.Sim(p, precision=precision)
    sim.set_particles(dense.x, dense.u, dense.phi, dense.type, dense.normal)
    with pytest.raises(wbsph.WbsphError) as ei:
        sim.eval_rates()
        sim.sync()
    assert ei.value.code == -9 and "overflow" in str(ei.value)
    sim.set_particles(sparse.x, sparse.u, sparse.phi, sparse.type, sparse.normal)
    sim.eval_rates()
    sim.sync()
    assert np.isfinite(sim.get("dudt")).all() and np.isfinite(sim.get("dphidt")).all()


def test_error_paths():
    from paper_2608_22269_gb300 import wbsph
    sc = S.dam_break_2d(dx=0.02, width=1.0, column=(0.3, 0.2))
    sim = wbsph.Sim(sc.params)
    with pytest.raises(wbsph.WbsphError) as ei:
        sim.step(1)
    assert ei.value.code == -8
    bad = sc.copy()
    bad.x[0, 3] = sc.params["domain_max"][0] + 0.5
    sim.set_scene(bad)
    sim.step(1)
    with pytest.raises(wbsph.WbsphError) as ei:
        sim.sync()
    assert ei.value.code == -4
    t = sc.type.copy()
    t[0] = 7
    with pytest.raises(wbsph.WbsphError) as ei:
        sim.set_particles(sc.x, sc.u, sc.phi, t, sc.normal)
    assert ei.value.code == -1


def test_device_resident_inputs_and_outputs():
    import torch
    sc = _dynamic(S.dam_break_2d(dx=0.01, width=1.0, column=(0.3, 0.2)))
    from paper_2608_22269_gb300 import wbsph
    sim = wbsph.Sim(sc.params, water_height=sc.water_height)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    sim.set_particles(dev(sc.x), dev(sc.u), dev(sc.phi), dev(sc.type), dev(sc.normal))
    sim.step(2)
    out = torch.empty((2, sc.n), dtype=torch.float64, device="cuda")
    sim.get("x", out)
    host = _sim(sc)
    host.step(2)
    assert np.array_equal(out.cpu().numpy(), host.get("x"))


def test_profile_and_stats_count_launches():
    sc = S.dam_break_2d(dx=0.01, width=1.0, column=(0.3, 0.2))
    sim = _sim(sc)
    sim.set_profiling(True)
    sim.step(2)
    prof = sim.profile(reset=True)
    assert prof["pair"][1] == 4 and prof["pair"][0] > 0
    assert prof["nlist"][1] == 4 and prof["nlist"][0] > 0
    st = sim.stats()
    assert st["launches"] > 20 and st["steps"] == 2


def test_non_finite_input_is_reported():
    from paper_2608_22269_gb300 import wbsph
    sc = S.dam_break_2d(dx=0.02, width=1.0, column=(0.3, 0.2))
    bad = sc.copy()
    bad.phi[5] = np.nan
    sim = _sim(bad)
    sim.step(1)
    with pytest.raises(wbsph.WbsphError) as ei:
        sim.sync()
    assert ei.value.code == -6


def test_restart_from_fields_continues_the_run():
    """get_fields + set_particles restart: x, U, phi and masses carry the whole
    state of a flow without forcing (the dummies are rebuilt every stage)."""
    sc = _dynamic(S.dam_break_2d(dx=0.01, width=1.0, column=(0.3, 0.2)))
    a = _sim(sc)
    a.step(4)
    b = _sim(sc)
    b.step(2)
    st = {k: b.get(k) for k in ("x", "u", "phi", "mass")}
    c = _sim(sc)
    c.set_particles(st["x"], st["u"], st["phi"], sc.type, sc.normal, st["mass"])
    c.step(2)
    sk = scales(sc.params, sc.water_height)
    assert scaled_err(c.get("x"), a.get("x"), sk["x"]) <= 1e-13
    assert scaled_err(c.get("u"), a.get("u"), sk["u"]) <= 1e-12


def test_bounded_device_wait_reports_timeout_and_context_survives():
    """A device wait that nothing satisfies gives up after its limit, and a
    second warp's wait (64 times the limit) leaves on the abort flag it
    raises, as the fused layer's roles do; together they report
    WBSPH_E_TIMEOUT through the status word (no trap, no fault). The same
    handle then reloads and steps normally. A limit out of range is refused
    before any launch."""
    from paper_2608_22269_gb300 import wbsph
    sc = S.dam_break_2d(dx=0.02, width=1.0, column=(0.3, 0.2))
    sim = _sim(sc)
    with pytest.raises(wbsph.WbsphError) as ei:
        sim.test_bounded_wait(4096)
    assert ei.value.code == -7
    for bad in (0, (1 << 20) + 1):
        with pytest.raises(wbsph.WbsphError) as ei:
            sim.test_bounded_wait(bad)
        assert ei.value.code == -1
    sim.set_scene(sc)
    sim.step(2)
    sim.sync()
    st = oracle.State(sc)
    st.step(2)
    sk = scales(sc.params, sc.water_height)
    assert scaled_err(sim.get("x"), st.x, sk["x"]) <= TOL


def test_allocation_failure_is_reported_and_the_handle_recovers():
    """Fault injection on the host (no GPU fault): the caller's allocator
    refuses one request during set_particles. The call returns
    WBSPH_E_NOMEM and the handle holds no particle set (a step is refused
    with WBSPH_E_STATE). The next set_particles, whose requests all
    succeed, gives a handle that steps to oracle parity, and every block the
    library took is back with the allocator once the handle is closed."""
    import torch
    from paper_2608_22269_gb300 import wbsph
    sc = S.dam_break_2d(dx=0.02, width=1.0, column=(0.3, 0.2))
    stream = torch.cuda.Stream()
    live, calls = {}, [0]

    def alloc(size):
        calls[0] += 1
        if calls[0] == 5:
            return 0
        p = torch.cuda.caching_allocator_alloc(size, 0, stream)
        live[p] = size
        return p

    def free(p):
        del live[p]
        torch.cuda.caching_allocator_delete(p)

    sim = wbsph.Sim(sc.params, water_height=sc.water_height, stream=stream, allocator=(alloc, free))
    with pytest.raises(wbsph.WbsphError) as ei:
        sim.set_scene(sc)
    assert ei.value.code == -2
    with pytest.raises(wbsph.WbsphError) as ei:
        sim.step(1)
    assert ei.value.code == -8
    sim.set_scene(sc)
    sim.step(2)
    sim.sync()
    st = oracle.State(sc)
    st.step(2)
    sk = scales(sc.params, sc.water_height)
    assert scaled_err(sim.get("x"), st.x, sk["x"]) <= TOL
    assert calls[0] > 5 and live
    sim.close()
    assert not live


@pytest.mark.parametrize("precision", [0, 1])
def test_wall_particles_only(precision):
    """No fluid at all: the dummy update finds no fluid within 2h and leaves
    every wall particle as it is, the pair passes have no rows, and time
    still advances with U_max = 0 (FP64 and mixed paths)."""
    sc = S.dam_break_2d(dx=0.02, width=1.0, column=(0.3, 0.2))
    walls = sc.type != 0
    only = S.Scene(dict(sc.params), sc.x[:, walls].copy(), sc.u[:, walls].copy(), sc.phi[walls].copy(),
                   sc.type[walls].copy(), sc.normal[:, walls].copy())
    sim = _sim(only, precision)
    sim.step(2)
    sim.sync()
    st = sim.stats()
    assert st["n_fluid"] == 0 and st["n"] == int(walls.sum())
    assert np.array_equal(sim.get("x"), only.x)
    assert np.array_equal(sim.get("u"), only.u)
    assert np.array_equal(sim.get("phi"), only.phi)
    dt = oracle.time_step(only.params, only.u, only.type)
    assert st["t"] == pytest.approx(2 * dt, rel=1e-15)


@pytest.mark.parametrize("precision", ["FP64", "MIXED", "DF64"])
def test_graph_replay_equals_eager_steps(precision):
    """Steps replayed from captured graphs against the same steps enqueued
    one launch at a time (profiling on disables graphs), bit for bit. A
    FP64 step leaves every buffer pointer where it found it (one graph); a
    mixed or double-float step sorts once, so its pointers alternate and two
    graphs serve the odd and even steps: five steps replay both."""
    from paper_2608_22269_gb300 import wbsph
    sc = S.jitter(S.dam_break_2d(dx=0.01, width=0.8, column=(0.4, 0.25)), 0.3, seed=9)
    sc.u[0, sc.type == 0] = 1.0
    prec = getattr(wbsph, precision)
    out = []
    for eager in (False, True):
        sim = wbsph.Sim(sc.params, precision=prec, water_height=sc.water_height)
        sim.set_scene(sc)
        sim.set_profiling(eager)
        sim.step(5)
        out.append([sim.get(k) for k in ("x", "u", "phi")] + [sim.stats()["t"]])
        sim.close()
    for a, b in zip(out[0], out[1]):
        assert np.array_equal(np.asarray(a), np.asarray(b))
