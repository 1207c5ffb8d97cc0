"""wbsph_sort_cells_noalloc against the regular neighbour build.

The no-allocation entry point exists for callers that cannot let a library
allocate device memory: a framework that owns the whole device memory pool,
or a loop that cannot take the implicit synchronisation of cudaMalloc and
cudaFree. It keeps its scratch in a static device array shared by all calls,
so these tests call it several times in a row (with different inputs in
between) and compare each result, bit for bit, with the keys and sort order
of wbsph_build_neighbors + wbsph_get_cell_keys. This file is collected last.
"""
import numpy as np
import pytest

from paper_2608_22269_gb300 import scenes as S

pytestmark = pytest.mark.gpu


def _regular(sc):
    from paper_2608_22269_gb300 import wbsph
    sim = wbsph.Sim(sc.params)
    sim.set_scene(sc)
    sim.build_neighbors()
    keys, ids = sim.cell_keys()
    sim.close()
    return keys, ids


def _noalloc(sim, sc):
    import torch
    x = torch.from_numpy(np.ascontiguousarray(sc.x)).cuda()
    keys = torch.full((sc.n,), -1, dtype=torch.int32, device="cuda")
    ids = torch.full((sc.n,), -1, dtype=torch.int32, device="cuda")
    sim.sort_cells_noalloc(x, keys, ids)
    return keys.cpu().numpy().view(np.uint32), ids.cpu().numpy().view(np.uint32)


def test_noalloc_sort_equals_regular_build_on_consecutive_calls():
    from paper_2608_22269_gb300 import wbsph
    big = S.random_box(300_000, 3, side=0.6, dx=0.01, seed=31)
    small = S.jitter(S.dam_break_2d(dx=0.01, width=1.0, column=(0.3, 0.2)), 0.2, seed=4)
    ref_big = _regular(big)
    ref_small = _regular(small)
    sim_big = wbsph.Sim(big.params)      # created only: no particles, no device buffers
    sim_small = wbsph.Sim(small.params)
    for sim, sc, ref in [(sim_big, big, ref_big), (sim_big, big, ref_big),
                         (sim_small, small, ref_small), (sim_big, big, ref_big),
                         (sim_small, small, ref_small)]:
        keys, ids = _noalloc(sim, sc)
        assert np.array_equal(keys, ref[0])
        assert np.array_equal(ids, ref[1])
    assert sim_big.stats()["device_bytes"] == 0


def test_noalloc_sort_rejects_sizes_beyond_its_limit():
    import torch
    from paper_2608_22269_gb300 import wbsph
    sc = S.random_box(wbsph.NOALLOC_MAX_N + 1, 2, side=1.0, dx=0.01, seed=2, on_faces=False)
    sim = wbsph.Sim(sc.params)
    x = torch.from_numpy(sc.x).cuda()
    k = torch.empty(sc.n, dtype=torch.int32, device="cuda")
    with pytest.raises(wbsph.WbsphError) as ei:
        sim.sort_cells_noalloc(x, k, k.clone())
    assert ei.value.code == -9 and "WBSPH_NOALLOC_MAX_N" in str(ei.value)
