"""Host-side checks of the C-ABI library: it builds for sm_103a, loads, and
exports every function that include/wbsph.h declares (no compute calls);
configuration validation; and, emulated in IEEE arithmetic on the host, the
numerical arguments the kernels rely on: the error bound of the cell-key
kernel's FP32 fast path, the exact high-part offset differences of the
double-float pack, and the error bounds of the double-float primitives."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "wbsph.h")).read()
    return sorted(set(re.findall(r"^\s*(?:int64_t|int|void|const char\*)\s+(wbsph_\w+)\s*\(", src,
                                 re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_2608_22269_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 15
    for name in names:
        assert hasattr(lib, name), name


def test_binding_lists_the_same_symbols():
    from paper_2608_22269_gb300 import wbsph
    assert sorted(wbsph.SYMBOLS) == _declared()


def test_noalloc_arguments_are_checked_before_the_call():
    """The binding of wbsph_sort_cells_noalloc checks every tensor before a
    pointer reaches the library (which cannot check bare pointers): each bad
    argument raises WbsphError(WBSPH_E_INVAL) from the tensors' metadata
    alone, so no kernel is launched. Run here on CPU tensors against a CPU
    'device'; the device mismatch is checked against cuda:0."""
    import torch
    from paper_2608_22269_gb300 import wbsph
    cpu = torch.device("cpu")
    n, dim = 100, 3
    x = torch.zeros(dim, n, dtype=torch.float64)
    k = torch.zeros(n, dtype=torch.int32)
    i = torch.zeros(n, dtype=torch.int32)
    assert wbsph.check_noalloc_args(x, k, i, dim, cpu) == n
    big = torch.zeros(2 * n, dtype=torch.int32)
    assert wbsph.check_noalloc_args(x, big[:n], big[n:], dim, cpu) == n
    bad_cases = {
        "float32 x": (x.float(), k, i),
        "transposed x": (x.t(), k, i),
        "(n, dim) x": (x.t().contiguous(), k, i),
        "wrong dim": (torch.zeros(2, n, dtype=torch.float64), k, i),
        "1-D x": (torch.zeros(dim * n, dtype=torch.float64), k, i),
        "short keys": (x, k[:n - 1], i),
        "short ids": (x, k, i[:n - 1]),
        "int64 keys": (x, k.long(), i),
        "float ids": (x, k, i.float()),
        "strided keys": (x, big[::2], i),
        "keys alias ids": (x, k, k),
        "overlapping outputs": (x, big[:n], big[n - 1:2 * n - 1]),
        "keys inside x": (x, x.view(torch.int32)[0, :n], i),
        "numpy keys": (x, k.numpy(), i),
    }
    for what, (xx, kk, ii) in bad_cases.items():
        with pytest.raises(wbsph.WbsphError) as ei:
            wbsph.check_noalloc_args(xx, kk, ii, dim, cpu)
        assert ei.value.code == -1, what
    with pytest.raises(wbsph.WbsphError):
        wbsph.check_noalloc_args(x, k, i, dim, torch.device("cuda", 0))


def test_update_arguments_are_checked_before_the_call():
    """The binding of wbsph_update_particles checks the host arrays before
    the library reads count rows of each through bare pointers: ids distinct
    integers in [0, n), x and u (dim, count), phi (count,). Each bad argument
    raises WbsphError(WBSPH_E_INVAL); a good call returns the arrays as the
    library takes them, and an empty update passes."""
    from paper_2608_22269_gb300 import wbsph
    n, dim = 50, 2
    ids = np.array([3, 0, 49, 7])
    x, u, phi = np.zeros((dim, 4)), np.ones((dim, 4)), np.arange(4.0)
    i2, x2, u2, p2 = wbsph.check_update_args(ids, x, u, phi, dim, n)
    assert i2.dtype == np.uint32 and i2.flags.c_contiguous and list(i2) == [3, 0, 49, 7]
    assert x2.shape == (dim, 4) and u2.dtype == np.float64 and p2.shape == (4,)
    e = wbsph.check_update_args([], np.zeros((dim, 0)), np.zeros((dim, 0)), np.zeros(0), dim, n)
    assert e[0].size == 0
    bad_cases = {
        "repeated id": ([3, 0, 3, 7], x, u, phi),
        "negative id": ([3, -1, 4, 7], x, u, phi),
        "id = n": ([3, 0, 50, 7], x, u, phi),
        "float ids": (ids.astype(float), x, u, phi),
        "2-D ids": (ids.reshape(2, 2), x, u, phi),
        "x of (count, dim)": (ids, x.T, u, phi),
        "short u": (ids, x, u[:, :3], phi),
        "long phi": (ids, x, u, np.arange(5.0)),
        "x of another dim": (ids, np.zeros((3, 4)), u, phi),
    }
    for what, args in bad_cases.items():
        with pytest.raises(wbsph.WbsphError) as ei:
            wbsph.check_update_args(*args, dim, n)
        assert ei.value.code == -1, what


def test_status_strings_and_config_defaults(lib):
    from paper_2608_22269_gb300 import wbsph
    L = wbsph.load()
    assert L.wbsph_status_string(0) == b"ok"
    assert L.wbsph_status_string(-4) == b"particle outside the domain"
    cfg = wbsph.Config()
    assert L.wbsph_config_default(ctypes.byref(cfg), 3) == 0
    assert cfg.h_over_dx == 1.5 and cfg.c0 == 30.0 and cfg.cfl == 0.2 and cfg.g[2] == -9.81
    assert L.wbsph_config_default(ctypes.byref(cfg), 4) == -1


def test_create_rejects_bad_configs_without_a_gpu(lib):
    from paper_2608_22269_gb300 import wbsph
    L = wbsph.load()
    cfg = wbsph.Config()
    L.wbsph_config_default(ctypes.byref(cfg), 2)
    h = ctypes.c_void_p()
    cfg.dx = -1.0
    assert L.wbsph_create(ctypes.byref(cfg), ctypes.byref(h)) == -1
    cfg.dx = 0.01
    cfg.eos = 5
    assert L.wbsph_create(ctypes.byref(cfg), ctypes.byref(h)) == -1
    cfg.eos = 0
    cfg.domain_max[0] = cfg.domain_min[0]
    assert L.wbsph_create(ctypes.byref(cfg), ctypes.byref(h)) == -1
    cfg.domain_max[0] = 1.0
    assert cfg.scheme == 0 and cfg.art_alpha == 0.02
    cfg.scheme = 2
    assert L.wbsph_create(ctypes.byref(cfg), ctypes.byref(h)) == -1
    # the conventional foil: FP64 only, no delta-SPH, shifting or TIC
    cfg.scheme = 1
    assert L.wbsph_create(ctypes.byref(cfg), ctypes.byref(h)) == -1  # defaults have them on
    cfg.use_delta = cfg.use_pst = cfg.use_tic = 0
    cfg.precision = 1
    assert L.wbsph_create(ctypes.byref(cfg), ctypes.byref(h)) == -1
    cfg.precision = 2  # the double-float path runs the well-balanced scheme only
    assert L.wbsph_create(ctypes.byref(cfg), ctypes.byref(h)) == -1
    cfg.scheme = 0
    cfg.precision = 3  # FP64 = 0, MIXED = 1, DF64 = 2
    assert L.wbsph_create(ctypes.byref(cfg), ctypes.byref(h)) == -1
    assert L.wbsph_step(None, 1) == -1


def test_binding_kernel_classes_match_the_header():
    """The profile arrays the binding passes hold WBSPH_K_COUNT entries, in
    the order of the wbsph_kernel_class enum."""
    from paper_2608_22269_gb300 import wbsph
    src = open(os.path.join(ROOT, "include", "wbsph.h")).read()
    enum = dict((k, int(v)) for k, v in re.findall(r"WBSPH_K_(\w+)\s*=\s*(\d+)", src))
    count = enum.pop("COUNT")
    assert len(wbsph.KERNEL_CLASSES) == count
    assert sorted(enum, key=enum.get) == [k.upper() for k in wbsph.KERNEL_CLASSES]


def _trunc32(x):
    """FP32 value of doubles with the mantissa truncated to 23 bits."""
    b = np.asarray(x, dtype=np.float64).view(np.uint64) & np.uint64(0xFFFFFFFFE0000000)
    return b.view(np.float64).astype(np.float32)


@pytest.mark.parametrize("lo,hi,R", [(0.0, 3.2, 0.02184), (-0.03, 4.03, 0.02), (-1.5, 2.0, 0.0044),
                                     (0.0, 0.2, 0.026)])
def test_cell_key_estimate_error_bound(lo, hi, R):
    """The cell-key kernel trusts floor of an FP32 estimate of (x - min)/R
    when its fractional part is more than 2E from 0 and 1, with
    E = 1.6 A 2^-23 / R + 3.1 N 2^-24 + N 2^-50 (A = max(|min|, |max|), N the
    cells on the axis). The estimate, emulated operation by operation, stays
    within E of the FP64 quotient of the definition, on random positions and
    on positions next to every cell boundary."""
    rng = np.random.default_rng(1)
    N = int(np.floor((hi - lo) / R)) + 1
    A = max(abs(lo), abs(hi))
    E = 1.6 * A * 2.0 ** -23 / R + 3.1 * N * 2.0 ** -24 + N * 2.0 ** -50
    bounds = lo + np.arange(N) * R
    near = np.concatenate([bounds, np.nextafter(bounds, -np.inf), np.nextafter(bounds, np.inf),
                           bounds + R * 1e-9, bounds - R * 1e-9])
    x = np.concatenate([rng.uniform(lo, hi, 200_000), near])
    x = x[(x >= lo) & (x <= hi)]
    q64 = (x - lo) / R  # IEEE FP64 subtraction then division, as the definition
    qf = (_trunc32(x) - np.float32(lo)) * np.float32(1.0 / R)  # float32 arithmetic, round to nearest
    err = np.abs(qf.astype(np.float64) - q64)
    assert err.max() <= E, (err.max(), E)
    # and where the estimate is trusted, it gives the definition's cell
    fr = qf - np.floor(qf)
    m = np.float32(2 * E * 1.001)
    ok = (fr > m) & (fr < 1 - m)
    assert np.array_equal(np.floor(qf[ok]).astype(np.int64), np.floor(q64[ok]).astype(np.int64))


def test_double_float_offsets_subtract_exactly():
    """The double-float pack stores o = (x - cell origin) / R with a high part
    rounded to a multiple of 2^-23 (add and subtract 1.5 * 2^29 in FP64). For
    |o| < 1.5 that high part is an FP32 number, and for every pair closer than
    R the pair pass's FP32 evaluation (cell offset) + (o_hi,j - o_hi,i) is
    exact, so r / R is rounded only in its low parts. Emulated with IEEE FP32
    and FP64 operations on random offsets, including the drift to |o| < 1.5."""
    rng = np.random.default_rng(11)
    o = rng.uniform(-1.5, 1.5, size=(2, 400_000))
    o[:, :64] = [[-1.5 + 2.0 ** -40], [1.5 - 2.0 ** -30]]  # near the ends of the range
    c = 1.5 * 2.0 ** 29
    q = (o + c) - c
    assert np.all(np.abs(o - q) <= 2.0 ** -24)
    assert np.all(np.abs(q * 2.0 ** 23 - np.rint(q * 2.0 ** 23)) == 0)
    hi = q.astype(np.float32)
    assert np.array_equal(hi.astype(np.float64), q)  # the high parts are FP32 numbers
    dc = rng.integers(-1, 2, size=o.shape[1]).astype(np.float32)
    diff = hi[1] - hi[0]  # FP32 subtraction
    rhat = dc + diff      # FP32 addition
    exact = dc.astype(np.float64) + (q[1] - q[0])
    near = np.abs(exact) <= 1.0 + 2.0 ** -22  # pairs within R (plus the low-part slack)
    assert near.sum() > 50_000
    assert np.array_equal(diff[near].astype(np.float64), (q[1] - q[0])[near])
    assert np.array_equal(rhat[near].astype(np.float64), exact[near])


def _f32(x):
    return np.float32(x)


def _fma32(a, b, c):
    """fmaf emulated through FP64: exact for the two-product residual
    a*b - fl(a*b); elsewhere (the cross terms of a product) within one extra
    rounding of a low part, far below the bounds checked here."""
    return np.float32(np.float64(a) * np.float64(b) + np.float64(c))


def _two_sum(a, b):
    s = _f32(a + b)
    bb = _f32(s - a)
    return s, _f32(_f32(a - _f32(s - bb)) + _f32(b - bb))


def _fast_two_sum(a, b):
    s = _f32(a + b)
    return s, _f32(b - _f32(s - a))


def _df_mul(a, b):
    p = _f32(a[0] * b[0])
    e = _fma32(a[0], b[0], -p)
    t = np.float32(np.float64(a[1]) * np.float64(b[0]) + np.float64(_f32(a[0] * b[1])))
    return _fast_two_sum(p, _f32(e + t))


def _df_acc(acc, v):
    s = _two_sum(acc[0], v[0])
    return _fast_two_sum(s[0], _f32(s[1] + _f32(acc[1] + v[1])))


def test_double_float_primitives_meet_their_error_bounds():
    """The double-float arithmetic of the df64 pair pass, emulated operation
    by operation in IEEE FP32 as the device helpers write it, against exact
    rational arithmetic: two-sum is exact; the product has a relative error
    of a few u^2 (u = 2^-24); a running sum of 100 terms of mixed sign stays
    within a few u^2 of the sum of the magnitudes. These bounds are what make
    the double-float pass agree with FP64 to ~1e-13 of a field's scale."""
    from fractions import Fraction as Fr
    rng = np.random.default_rng(3)
    u2 = Fr(1, 2 ** 48)

    def split(x):
        hi = np.float32(x)
        return hi, np.float32(x - np.float64(hi))

    def val(d):
        return Fr(float(d[0])) + Fr(float(d[1]))

    for _ in range(300):
        a, b = (np.float32(v) for v in rng.normal(size=2) * 10.0 ** rng.integers(-3, 4, size=2))
        s = _two_sum(a, b)
        assert Fr(float(s[0])) + Fr(float(s[1])) == Fr(float(a)) + Fr(float(b))
    for _ in range(300):
        x, y = split(rng.normal() * 7.0), split(rng.normal() * 0.3)
        exact = val(x) * val(y)
        err = abs(val(_df_mul(x, y)) - exact)
        assert err <= 6 * u2 * abs(exact)
    for _ in range(20):
        terms = [split(v) for v in rng.normal(size=100) * 10.0 ** rng.integers(-2, 3, size=100)]
        acc = (np.float32(0.0), np.float32(0.0))
        exact, mag = Fr(0), Fr(0)
        for t in terms:
            acc = _df_acc(acc, t)
            exact += val(t)
            mag += abs(val(t))
        assert abs(val(acc) - exact) <= 4 * u2 * mag
