"""Slab decomposition of the step (paper_2608_22269_gb300/slabs.py) on CPU
ranks, with the oracle as every rank's compute.

The paper runs one domain on one device; a decomposition must not change
the result. After several SSP-RK2 steps the owned particles of all ranks,
put back together, must equal the single-domain oracle step within 1e-12
(they come out bit for bit equal here: each subdomain lists its particles in
ascending global id, so every neighbour sum runs in the same order as in the
single domain, and the time step and shifting take the same global U_max).
Ranks run as threads of this process (several scenes, 1 to 4 slabs) and as
gloo processes (world size 2 and 4), which exercises the torch.distributed
communicator. A one-cell ghost band, too narrow for the wall update's
nearest-fluid search, must visibly change the result."""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

from oracle import oracle as O
from paper_2608_22269_gb300 import scenes as S
from paper_2608_22269_gb300 import slabs

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
from slab_backends import OracleBackend, combine, run_threads  # noqa: E402


def _dam_2d(speed=2.5):
    sc = S.jitter(S.dam_break_2d(dx=0.01, width=0.8, column=(0.4, 0.25)), 0.45, seed=3)
    sc.u[0, sc.type == S.FLUID] = speed      # the column thrown at the far wall: particles cross slab faces
    return sc


def _dam_3d():
    sc = S.jitter(S.dam_break_3d(dx=0.03, box=(0.6, 0.25, 0.3), column=(0.3, 0.25, 0.2)), 0.3, seed=5)
    sc.u[0, sc.type == S.FLUID] = 1.0
    return sc


def _slosh_3d():
    """Forced tank: the body force depends on time, so stage 2 must run at
    t + dt on every rank."""
    return S.jitter(S.sloshing_3d(dx=0.04, tank=(0.8, 0.3, 0.4), depth=0.2, amp=0.05, period=0.05), 0.3,
                    seed=6)


def _body_2d():
    return S.jitter(S.moving_body(2, dx=0.01, tank=(1.0, 0.5), depth=0.35, center=(0.46, 0.2),
                                  body_u=(3.0, 0.0)), 0.2, seed=8)


def _run(sc, size, steps, ghost_cells=2):
    def body(rank, comm):
        sl = slabs.Slab(sc, comm, OracleBackend(sc.params), ghost_cells=ghost_cells)
        start = sl.state["gid"].copy()
        for _ in range(steps):
            sl.step()
        return sl.owned(), start, sl.bounds, sl.t

    out = run_threads(size, body)
    x, u, phi = combine([o[0] for o in out], sc.n, sc.params["dim"])
    owner0 = np.empty(sc.n, dtype=np.int64)
    owner1 = np.empty(sc.n, dtype=np.int64)
    for r, o in enumerate(out):
        owner0[o[1]] = r
        owner1[o[0][0]] = r
    return x, u, phi, owner0, owner1, out[0][3]


def _reference(sc, steps):
    ref = O.State(sc)
    ref.step(steps)
    return ref


def _assert_equal(x, u, phi, ref):
    for a, b in ((x, ref.x), (u, ref.u), (phi, ref.phi)):
        err = float(np.abs(a - b).max())
        assert err <= 1e-12 * max(1.0, float(np.abs(b).max())), err


def test_slab_bounds_are_balanced_whole_cells():
    sc = _dam_2d()
    p = sc.params
    R = 2.0 * p["h_over_dx"] * p["dx"]
    ncell = int(np.floor((p["domain_max"][0] - p["domain_min"][0]) / R)) + 1
    for size in (1, 2, 3, 4):
        b = slabs.slab_bounds(p, sc.x, size, 0)
        assert b[0] == 0 and b[-1] == ncell and np.all(np.diff(b) >= 2)
        cell = np.clip(np.floor((sc.x[0] - p["domain_min"][0]) / R).astype(int), 0, ncell - 1)
        counts = [int(((cell >= b[r]) & (cell < b[r + 1])).sum()) for r in range(size)]
        assert sum(counts) == sc.n
        # the cut lands within one cell column of the balanced share
        per_cell = np.bincount(cell, minlength=ncell).max()
        assert max(counts) - min(counts) <= 2 * per_cell
    with pytest.raises(ValueError):
        slabs.slab_bounds(p, sc.x, ncell // 2 + 1, 0)


@pytest.mark.parametrize("scene,size,steps", [
    ("dam_2d", 1, 8), ("dam_2d", 2, 8), ("dam_2d", 4, 8),
    ("dam_3d", 2, 3), ("dam_3d", 4, 3),
    ("slosh_3d", 3, 5),
    ("body_2d", 4, 50),
])
def test_slabs_equal_the_single_domain_oracle(scene, size, steps):
    sc = {"dam_2d": _dam_2d, "dam_3d": _dam_3d, "slosh_3d": _slosh_3d, "body_2d": _body_2d}[scene]()
    ref = _reference(sc, steps)
    x, u, phi, owner0, owner1, t = _run(sc, size, steps)
    _assert_equal(x, u, phi, ref)
    assert t == ref.t
    if scene == "dam_2d" and size > 1:
        assert np.count_nonzero(owner0 != owner1) >= 3            # migration happened
    if scene == "body_2d":
        moved = (owner0 != owner1) & (sc.type == S.BODY)
        assert moved.any()                                         # wall particles of the body migrate too


def test_one_cell_ghost_band_is_too_narrow():
    """A wall particle next to a slab face takes its potential from its
    nearest fluid particle up to 2h (one cell) further out: with only one
    cell of ghosts that particle may be missing and the result changes."""
    sc = _dam_2d()
    ref = _reference(sc, 3)
    x, u, phi, *_ = _run(sc, 4, 3, ghost_cells=1)
    assert float(np.abs(phi - ref.phi).max()) > 1e-9


# -- gloo ranks ---------------------------------------------------------------------------------
def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _gloo_worker(rank, world, port, steps, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    import torch.distributed as dist
    sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
    from slab_backends import OracleBackend as OB
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        sc = _dam_2d()
        sl = slabs.Slab(sc, slabs.TorchComm(), OB(sc.params))
        for _ in range(steps):
            sl.step()
        gid, x, u, phi, typ = sl.owned()
        out[rank] = (gid.tolist(), x.tolist(), u.tolist(), phi.tolist(), sl.t)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 4])
def test_gloo_ranks_equal_the_single_domain_oracle(world):
    steps = 3
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_gloo_worker, args=(r, world, port, steps, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
    for p in procs:
        if p.is_alive():
            p.kill()
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    sc = _dam_2d()
    parts = [(np.array(out[r][0], dtype=np.int64), np.array(out[r][1]), np.array(out[r][2]),
              np.array(out[r][3]), None) for r in range(world)]
    x, u, phi = combine(parts, sc.n, 2)
    ref = _reference(sc, steps)
    _assert_equal(x, u, phi, ref)
    assert all(out[r][4] == ref.t for r in range(world))
