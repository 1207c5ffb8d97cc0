"""Slab decomposition on the CUDA library: every rank a handle of its own
(wbsph_stage, wbsph_update_particles) on this one GPU, the ranks as host
threads that exchange ghosts and U_max between the stages. No kernel waits
on another rank: all coupling goes through the host. After the steps the
combined owned particles must equal the single-domain FP64 step of the
library within 1e-12 of each field's scale, and the oracle's step within
the parity bound of the FP64 path."""
import os
import sys

import numpy as np
import pytest

from paper_2608_22269_gb300 import scenes as S
from paper_2608_22269_gb300 import slabs

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
from slab_backends import combine, run_threads  # noqa: E402

pytestmark = pytest.mark.gpu


def _scenes():
    dam = S.jitter(S.dam_break_2d(dx=0.005, width=0.8, column=(0.4, 0.25)), 0.45, seed=3)
    dam.u[0, dam.type == S.FLUID] = 2.5
    slosh = S.jitter(S.sloshing_3d(dx=0.02, tank=(0.8, 0.3, 0.4), depth=0.2, amp=0.05, period=0.05), 0.3,
                     seed=6)
    body = S.jitter(S.moving_body(2, dx=0.01, tank=(1.0, 0.5), depth=0.35, center=(0.46, 0.2),
                                  body_u=(3.0, 0.0)), 0.2, seed=8)
    return {"dam_2d": dam, "slosh_3d": slosh, "body_2d": body}


@pytest.mark.parametrize("scene,size,steps", [("dam_2d", 1, 6), ("dam_2d", 4, 6), ("slosh_3d", 3, 4),
                                              ("body_2d", 4, 50)])
def test_gpu_slabs_equal_the_single_domain_step(scene, size, steps):
    from oracle import oracle as O
    from paper_2608_22269_gb300 import wbsph
    sc = _scenes()[scene]
    plain = wbsph.Sim(sc.params, water_height=sc.water_height)
    plain.set_scene(sc)
    plain.step(steps)
    ref = {k: plain.get(k) for k in ("x", "u", "phi")}
    t_ref = plain.stats()["t"]
    plain.close()

    def body(rank, comm):
        be = slabs.GpuBackend(sc.params, sc.water_height)
        sl = slabs.Slab(sc, comm, be)
        start = sl.state["gid"].copy()
        for _ in range(steps):
            sl.step()
        be.close()
        return sl.owned(), start, sl.t

    out = run_threads(size, body)
    x, u, phi = combine([o[0] for o in out], sc.n, sc.params["dim"])
    moved = sum(int(np.setdiff1d(o[0][0], o[1]).size) for o in out)
    print(scene, size, "migrated", moved, "t", out[0][2], t_ref)
    for k, a in (("x", x), ("u", u), ("phi", phi)):
        err = float(np.abs(a - ref[k]).max())
        assert err <= 1e-12 * max(1.0, float(np.abs(ref[k]).max())), (k, err)
    assert abs(out[0][2] - t_ref) <= 1e-15 * t_ref
    o = O.State(sc)
    o.step(steps)
    for k, a in (("x", x), ("u", u), ("phi", phi)):
        b = getattr(o, k)
        assert float(np.abs(a - b).max()) <= 1e-10 * max(1.0, float(np.abs(b).max())), k
    if size > 1 and scene != "slosh_3d":
        assert moved > 0
