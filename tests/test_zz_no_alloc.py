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


@pytest.mark.parametrize("dim,n,side,passes", [(2, 3000, 0.2, 1), (3, 400_000, 1.1, 3)])
def test_noalloc_sort_odd_pass_counts(dim, n, side, passes):
    """Grids of at most 256 cells (one 8-bit radix pass) and of more than
    65,536 cells (three passes): with an odd pass count the sorted keys end in
    the static scratch array and are copied to the caller's buffers. Bit for
    bit against the regular build, twice in a row."""
    from paper_2608_22269_gb300 import wbsph
    sc = S.random_box(n, dim, side=side, dx=0.01, seed=40 + dim)
    R = 2.0 * sc.params["h_over_dx"] * sc.params["dx"]
    ncells = int(np.prod([int(np.floor(side / R)) + 1 for _ in range(dim)]))
    bits = max(1, int(np.ceil(np.log2(ncells))))
    assert (bits + 7) // 8 == passes, (ncells, bits)
    ref = _regular(sc)
    sim = wbsph.Sim(sc.params)
    for _ in range(2):
        keys, ids = _noalloc(sim, sc)
        assert np.array_equal(keys, ref[0])
        assert np.array_equal(ids, ref[1])


def test_noalloc_sort_rejects_bad_tensors_before_the_call():
    """A float32 x, a transposed x or a short output raises before any pointer
    reaches the library; the handle stays usable."""
    import torch
    from paper_2608_22269_gb300 import wbsph
    sc = S.random_box(5000, 3, side=0.3, dx=0.01, seed=5)
    sim = wbsph.Sim(sc.params)
    x = torch.from_numpy(sc.x).cuda()
    k = torch.empty(sc.n, dtype=torch.int32, device="cuda")
    i = torch.empty(sc.n, dtype=torch.int32, device="cuda")
    for bad in [(x.float(), k, i), (x.t(), k, i), (x, k[:-1], i), (x, k, k), (x.cpu(), k, i)]:
        with pytest.raises(wbsph.WbsphError) as ei:
            sim.sort_cells_noalloc(*bad)
        assert ei.value.code == -1
    ref = _regular(sc)
    keys, ids = _noalloc(sim, sc)
    assert np.array_equal(keys, ref[0]) and np.array_equal(ids, ref[1])


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


@pytest.mark.parametrize("dim,side", [(2, 1.0), (3, 1.1)])
def test_noalloc_sort_at_its_size_limit(dim, side):
    """Exactly WBSPH_NOALLOC_MAX_N particles, the largest input accepted: the
    static scratch is used to its last element. 2D: two radix passes; 3D:
    more than 65,536 cells, three passes, so the result ends in the scratch
    and is copied out. Bit for bit against the regular build. An empty input
    then returns at once and leaves its outputs as they were."""
    import torch
    from paper_2608_22269_gb300 import wbsph
    sc = S.random_box(wbsph.NOALLOC_MAX_N, dim, side=side, dx=0.01, seed=60 + dim, on_faces=False)
    ref = _regular(sc)
    sim = wbsph.Sim(sc.params)
    keys, ids = _noalloc(sim, sc)
    assert np.array_equal(keys, ref[0])
    assert np.array_equal(ids, ref[1])
    x0 = torch.empty((dim, 0), dtype=torch.float64, device="cuda")
    k0 = torch.full((4,), 7, dtype=torch.int32, device="cuda")
    i0 = torch.full((4,), 7, dtype=torch.int32, device="cuda")
    sim.sort_cells_noalloc(x0, k0, i0)
    assert int(k0.min()) == 7 and int(k0.max()) == 7 and int(i0.min()) == 7 and int(i0.max()) == 7
