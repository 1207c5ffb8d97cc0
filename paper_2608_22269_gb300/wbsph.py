"""Python binding of the C-ABI in ``include/wbsph.h`` (argument marshalling only).

Every step of the hot path runs in the CUDA library ``libwbsph.so`` built
in-tree by :mod:`paper_2608_22269_gb300.build`; this module only converts
arguments. PyTorch supplies device memory (through its caching allocator,
passed to the library as allocation callbacks) and the CUDA stream. There is
no CPU fallback: if the library is missing, loading fails loudly.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

OK = 0
ERRORS = {-1: "WBSPH_E_INVAL", -2: "WBSPH_E_NOMEM", -3: "WBSPH_E_CUDA", -4: "WBSPH_E_DOMAIN",
          -5: "WBSPH_E_SINGULAR", -6: "WBSPH_E_NAN", -7: "WBSPH_E_TIMEOUT", -8: "WBSPH_E_STATE",
          -9: "WBSPH_E_CAPACITY", -10: "WBSPH_E_NOSYM"}
FP64, MIXED, DF64 = 0, 1, 2
HOST, DEVICE = 0, 1
FIELDS = {"x": 0, "u": 1, "phi": 2, "rho": 3, "p": 4, "dudt": 5, "dphidt": 6, "dushift": 7,
          "lambda": 8, "mass": 9, "vol": 10}
VECTOR_FIELDS = {"x", "u", "dudt", "dushift"}
KERNEL_CLASSES = ["keys", "sort", "reorder", "cells", "prepass", "pair", "update", "other", "nlist"]

#: every symbol declared in include/wbsph.h
SYMBOLS = ["wbsph_config_default", "wbsph_create", "wbsph_set_particles", "wbsph_build_neighbors",
           "wbsph_eval_rates", "wbsph_step", "wbsph_sync", "wbsph_get_fields",
           "wbsph_get_cell_keys", "wbsph_get_neighbors", "wbsph_get_stats", "wbsph_set_profiling",
           "wbsph_get_profile", "wbsph_destroy", "wbsph_last_error", "wbsph_status_string",
           "wbsph_sort_cells_noalloc", "wbsph_test_bounded_wait", "wbsph_stage", "wbsph_update_particles"]
NOALLOC_MAX_N = 524288

ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_void_p)


class Config(C.Structure):
    _fields_ = [("dim", C.c_int), ("dx", C.c_double), ("h_over_dx", C.c_double),
                ("rho0", C.c_double), ("c0", C.c_double), ("nu", C.c_double),
                ("g", C.c_double * 3), ("cfl", C.c_double), ("delta", C.c_double),
                ("pst_R", C.c_double), ("pst_n", C.c_double), ("tic_lambda", C.c_double),
                ("use_delta", C.c_int), ("use_pst", C.c_int), ("use_tic", C.c_int),
                ("use_visc", C.c_int), ("eos", C.c_int), ("tait_gamma", C.c_double),
                ("domain_min", C.c_double * 3), ("domain_max", C.c_double * 3),
                ("force_amp", C.c_double * 3), ("force_period", C.c_double),
                ("fixed_dt", C.c_double), ("precision", C.c_int), ("device", C.c_int),
                ("cuda_stream", C.c_void_p), ("alloc", ALLOC_FN), ("free", FREE_FN),
                ("alloc_ctx", C.c_void_p), ("water_height", C.c_double), ("scheme", C.c_int),
                ("art_alpha", C.c_double), ("wall_bc", C.c_int), ("body_u", C.c_double * 3)]


class Stats(C.Structure):
    _fields_ = [("n", C.c_int64), ("n_fluid", C.c_int64), ("n_dummy", C.c_int64),
                ("ncells", C.c_int64), ("grid", C.c_int64 * 3), ("steps", C.c_int64),
                ("launches", C.c_int64), ("device_bytes", C.c_int64), ("t", C.c_double),
                ("dt", C.c_double), ("pairs", C.c_int64)]


class WbsphError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Load libwbsph.so (raises if it is not built; no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError(f"CUDA library not built: {path} (run __graft_entry__.build())")
        _build.build()
    L = C.CDLL(path)
    P, i64, I = C.c_void_p, C.c_int64, C.c_int
    sig = {
        "wbsph_config_default": (I, [P, I]),
        "wbsph_create": (I, [P, P]),
        "wbsph_set_particles": (I, [P, i64, P, P, P, P, P, P, I]),
        "wbsph_build_neighbors": (I, [P]),
        "wbsph_eval_rates": (I, [P]),
        "wbsph_step": (I, [P, i64]),
        "wbsph_sync": (I, [P]),
        "wbsph_get_fields": (I, [P, I, P, I]),
        "wbsph_get_cell_keys": (I, [P, P, P]),
        "wbsph_get_neighbors": (i64, [P, P, P, i64]),
        "wbsph_get_stats": (I, [P, P]),
        "wbsph_set_profiling": (I, [P, I]),
        "wbsph_get_profile": (I, [P, P, P, I]),
        "wbsph_destroy": (None, [P]),
        "wbsph_last_error": (C.c_char_p, [P]),
        "wbsph_status_string": (C.c_char_p, [I]),
        "wbsph_sort_cells_noalloc": (I, [P, P, i64, P, P]),
        "wbsph_test_bounded_wait": (I, [P, i64]),
        "wbsph_stage": (I, [P, I, C.c_double, C.c_double, C.c_double]),
        "wbsph_update_particles": (I, [P, i64, P, P, P, P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _ptr(a):
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data_as(C.c_void_p)
    return C.c_void_p(a.data_ptr())  # torch tensor


def make_config(params: dict, precision: int = FP64, stream=None, device: int = 0,
                water_height: float = 0.0) -> Config:
    cfg = Config()
    load().wbsph_config_default(C.byref(cfg), int(params["dim"]))
    for name, _ in Config._fields_:
        if name in params and name not in ("alloc", "free", "alloc_ctx", "cuda_stream"):
            v = params[name]
            if isinstance(v, (list, tuple, np.ndarray)):
                arr = getattr(cfg, name)
                for k in range(3):
                    arr[k] = float(v[k]) if k < len(v) else 0.0
            else:
                setattr(cfg, name, v)
    cfg.precision = precision
    cfg.device = device
    cfg.cuda_stream = stream
    cfg.water_height = water_height
    return cfg


class Sim:
    """One simulation handle. ``params`` is a scene parameter dict; device
    memory comes from PyTorch's caching allocator on the current stream.
    ``precision`` selects the pair pass: FP64, MIXED (FP32 sums with Kahan
    compensation, about 1e-5 of the field scale) or DF64 (double-float sums
    on the FP32 pipe, within 1e-12 like FP64); ``water_height`` is the H of
    the hydrostatic split phi_hs = G.x + |G| H that MIXED and DF64 use."""

    def __init__(self, params: dict, precision: int = FP64, water_height: float = 0.0,
                 device: int = 0, use_torch_allocator: bool = True, stream=None, allocator=None):
        """The handle works on its own CUDA stream (a new torch stream unless
        ``stream`` is given), so that its steps can be replayed as CUDA
        graphs; the binding orders that stream against torch's current
        stream wherever device tensors are exchanged. ``allocator``, a pair
        of callables (alloc(size) -> device address or 0, free(address)),
        replaces the device allocator (the C-ABI's alloc/free hooks); an
        address of 0 is an allocation failure, which the library reports as
        WBSPH_E_NOMEM."""
        import torch
        self._torch = torch
        self.lib = load()
        self.dim = int(params["dim"])
        self.device = device
        self.stream = stream if stream is not None else torch.cuda.Stream(device)
        cfg = make_config(params, precision, C.c_void_p(self.stream.cuda_stream), device,
                          water_height)
        if allocator is not None:
            user_alloc, user_free = allocator

            def _alloc(size, stream, ctx):
                return int(user_alloc(int(size))) or None

            def _free(ptr, stream, ctx):
                user_free(int(ptr))

            self._alloc_cb = ALLOC_FN(_alloc)
            self._free_cb = FREE_FN(_free)
            cfg.alloc = self._alloc_cb
            cfg.free = self._free_cb
        elif use_torch_allocator:
            def _alloc(size, stream, ctx):
                return torch.cuda.caching_allocator_alloc(int(size), device, self.stream)

            def _free(ptr, stream, ctx):
                torch.cuda.caching_allocator_delete(int(ptr))

            self._alloc_cb = ALLOC_FN(_alloc)
            self._free_cb = FREE_FN(_free)
            cfg.alloc = self._alloc_cb
            cfg.free = self._free_cb
        self.cfg = cfg
        h = C.c_void_p()
        rc = self.lib.wbsph_create(C.byref(cfg), C.byref(h))
        if rc != OK:
            raise WbsphError(rc, self.lib.wbsph_status_string(rc).decode())
        self.h = h
        self.n = 0

    def _check(self, rc):
        if rc < 0:
            raise WbsphError(int(rc), self.lib.wbsph_last_error(self.h).decode())
        return rc

    def close(self):
        if getattr(self, "h", None):
            self.lib.wbsph_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- C-ABI calls ------------------------------------------------------------------------
    def set_particles(self, x, u, phi, type, normal=None, mass=None, where=None):
        """Host numpy arrays, or torch tensors (float64 SoA, uint8 type) on the
        device or in (pinned) host memory; ``where`` defaults from the arrays."""
        if where is None:
            dev = not isinstance(x, np.ndarray) and x.is_cuda
        else:
            dev = where == DEVICE
        if isinstance(x, np.ndarray):
            x, u, phi = (np.ascontiguousarray(a, dtype=np.float64) for a in (x, u, phi))
            type = np.ascontiguousarray(type, dtype=np.uint8)
            normal = None if normal is None else np.ascontiguousarray(normal, dtype=np.float64)
            mass = None if mass is None else np.ascontiguousarray(mass, dtype=np.float64)
        n = int(phi.shape[0])
        self._keep = (x, u, phi, type, normal, mass)
        if dev:
            self.stream.wait_stream(self._torch.cuda.current_stream(self.device))
        self._check(self.lib.wbsph_set_particles(self.h, n, _ptr(x), _ptr(u), _ptr(phi), _ptr(mass),
                                                 _ptr(type), _ptr(normal), DEVICE if dev else HOST))
        self.n = n
        return self

    def set_scene(self, scene):
        return self.set_particles(scene.x, scene.u, scene.phi, scene.type, scene.normal)

    def build_neighbors(self):
        self._check(self.lib.wbsph_build_neighbors(self.h))

    def eval_rates(self):
        self._check(self.lib.wbsph_eval_rates(self.h))

    def step(self, nsteps=1):
        self._check(self.lib.wbsph_step(self.h, int(nsteps)))

    def sync(self):
        self._check(self.lib.wbsph_sync(self.h))

    def stage(self, stage, t, dt, umax):
        """One SSP-RK2 stage of a subdomain (wbsph_stage): t the step's start
        time, dt the time step (<= 0: from umax in stage 1, kept in stage 2),
        umax the stage's maximum fluid speed over the whole domain."""
        self._check(self.lib.wbsph_stage(self.h, int(stage), float(t), float(dt), float(umax)))

    def update_particles(self, ids, x, u, phi):
        """Overwrite x, U, phi of the particles with these input indices
        (wbsph_update_particles; host arrays, x and u of shape (dim, count)).
        The arguments are checked (check_update_args) before the call."""
        ids, x, u, phi = check_update_args(ids, x, u, phi, self.dim, self.n)
        self._check(self.lib.wbsph_update_particles(self.h, ids.size, _ptr(ids), _ptr(x), _ptr(u), _ptr(phi)))

    def get(self, field: str, out=None):
        """Field in the caller's original order: numpy (host) unless ``out``
        is a device tensor."""
        comps = self.dim if field in VECTOR_FIELDS else 1
        shape = (comps, self.n) if comps > 1 else (self.n,)
        if out is None:
            out = np.empty(shape, dtype=np.float64)
        where = HOST if isinstance(out, np.ndarray) or not out.is_cuda else DEVICE
        if where == DEVICE:
            self.stream.wait_stream(self._torch.cuda.current_stream(self.device))
        self._check(self.lib.wbsph_get_fields(self.h, FIELDS[field], _ptr(out), where))
        if where == DEVICE:
            self._torch.cuda.current_stream(self.device).wait_stream(self.stream)
        return out

    def cell_keys(self):
        k = np.empty(self.n, dtype=np.uint32)
        ids = np.empty(self.n, dtype=np.uint32)
        self._check(self.lib.wbsph_get_cell_keys(self.h, _ptr(k), _ptr(ids)))
        return k, ids

    def neighbors(self):
        row = np.empty(self.n + 1, dtype=np.int64)
        nnz = self._check(self.lib.wbsph_get_neighbors(self.h, _ptr(row), None, 0))
        cols = np.empty(max(nnz, 1), dtype=np.int32)
        self._check(self.lib.wbsph_get_neighbors(self.h, _ptr(row), _ptr(cols), nnz))
        return row, cols[:nnz]

    def stats(self) -> dict:
        s = Stats()
        self._check(self.lib.wbsph_get_stats(self.h, C.byref(s)))
        return {k: (list(getattr(s, k)) if k == "grid" else getattr(s, k)) for k, _ in Stats._fields_}

    def sort_cells_noalloc(self, x, keys_sorted, ids_sorted):
        """wbsph_sort_cells_noalloc on device tensors: x (dim, n) float64,
        keys_sorted / ids_sorted (n,) 32-bit. Allocates no device memory.
        The arguments are checked (check_noalloc_args) before the call, since
        the library receives bare pointers and cannot check them."""
        torch = self._torch
        n = check_noalloc_args(x, keys_sorted, ids_sorted, self.dim,
                               torch.device("cuda", self.device))
        cur = self._torch.cuda.current_stream(self.device)
        self.stream.wait_stream(cur)
        self._check(self.lib.wbsph_sort_cells_noalloc(self.h, _ptr(x), n, _ptr(keys_sorted),
                                                      _ptr(ids_sorted)))
        cur.wait_stream(self.stream)
        return keys_sorted, ids_sorted

    def test_bounded_wait(self, limit=4096):
        """Run the bounded-wait check (wbsph_test_bounded_wait); raises
        WbsphError(WBSPH_E_TIMEOUT) when the first wait gave up and the
        second left on the abort flag, as designed."""
        self._check(self.lib.wbsph_test_bounded_wait(self.h, int(limit)))

    def set_profiling(self, on=True):
        self._check(self.lib.wbsph_set_profiling(self.h, int(on)))

    def profile(self, reset=False) -> dict:
        ms = (C.c_double * len(KERNEL_CLASSES))()
        cnt = (C.c_int64 * len(KERNEL_CLASSES))()
        self._check(self.lib.wbsph_get_profile(self.h, ms, cnt, int(reset)))
        return {k: (ms[i], cnt[i]) for i, k in enumerate(KERNEL_CLASSES)}


def check_update_args(ids, x, u, phi, dim: int, n: int):
    """Argument checks of wbsph_update_particles, on the host arrays before
    the call (the library reads count rows of each array through bare
    pointers): ids a one-dimensional integer array of distinct indices in
    [0, n), n the particle count of the last set_particles; x and u of shape
    (dim, count), phi of shape (count,). Returns the arrays as the library
    takes them (contiguous uint32 ids, float64 fields); raises
    WbsphError(WBSPH_E_INVAL)."""
    def bad(msg):
        raise WbsphError(-1, f"update_particles: {msg}")

    ids = np.asarray(ids)
    if ids.ndim != 1:
        bad(f"ids must be one-dimensional, got shape {ids.shape}")
    if ids.size and not np.issubdtype(ids.dtype, np.integer):
        bad(f"ids must be integers, got {ids.dtype}")
    count = int(ids.size)
    if count and (int(ids.min()) < 0 or int(ids.max()) >= n):
        bad(f"ids must lie in [0, {n})")
    if np.unique(ids).size != count:
        bad("ids must be distinct")
    x, u, phi = (np.ascontiguousarray(a, dtype=np.float64) for a in (x, u, phi))
    for name, a, shape in (("x", x, (dim, count)), ("u", u, (dim, count)), ("phi", phi, (count,))):
        if a.shape != shape:
            bad(f"{name} must have shape {shape}, got {a.shape}")
    return np.ascontiguousarray(ids, dtype=np.uint32), x, u, phi


def check_noalloc_args(x, keys_sorted, ids_sorted, dim: int, device) -> int:
    """Argument checks of wbsph_sort_cells_noalloc, done on the tensors'
    metadata before any pointer reaches the library: x must be a contiguous
    float64 tensor of shape (dim, n) on ``device``; keys_sorted and ids_sorted
    contiguous 32-bit integer tensors of at least n elements on the same
    device, not overlapping each other or x. A float32 or transposed x would
    make the key kernel read past the end of x, and a short output would make
    the sort write past its end. Returns n; raises WbsphError(WBSPH_E_INVAL)."""
    import torch

    def bad(msg):
        raise WbsphError(-1, f"sort_cells_noalloc: {msg}")

    for name, t in (("x", x), ("keys_sorted", keys_sorted), ("ids_sorted", ids_sorted)):
        if not isinstance(t, torch.Tensor):
            bad(f"{name} must be a torch tensor")
        if t.device != torch.device(device):
            bad(f"{name} is on {t.device}, the handle's device is {device}")
        if not t.is_contiguous():
            bad(f"{name} must be contiguous")
    if x.dtype != torch.float64:
        bad(f"x must be float64, got {x.dtype}")
    if x.dim() != 2 or int(x.shape[0]) != int(dim):
        bad(f"x must have shape ({dim}, n), got {tuple(x.shape)}")
    n = int(x.shape[1])
    u32 = getattr(torch, "uint32", None)
    for name, t in (("keys_sorted", keys_sorted), ("ids_sorted", ids_sorted)):
        if t.dtype not in (torch.int32,) + ((u32,) if u32 is not None else ()):
            bad(f"{name} must be a 32-bit integer tensor, got {t.dtype}")
        if t.numel() < n:
            bad(f"{name} holds {t.numel()} elements, {n} are needed")

    def span(t, count):
        return t.data_ptr(), t.data_ptr() + count * t.element_size()

    spans = {"x": span(x, x.numel()), "keys_sorted": span(keys_sorted, n),
             "ids_sorted": span(ids_sorted, n)}
    names = list(spans)
    for a in range(3):
        for b in range(a + 1, 3):
            (a0, a1), (b0, b1) = spans[names[a]], spans[names[b]]
            if n > 0 and a0 < b1 and b0 < a1:
                bad(f"{names[a]} and {names[b]} overlap")
    return n


# ---------------------------------------------------------------------------
# Learned surrogate (wbsph_surrogate_* in include/wbsph.h)
# ---------------------------------------------------------------------------
class SurrogateConfig(C.Structure):
    _fields_ = [("dim", C.c_int), ("hidden", C.c_int), ("layers", C.c_int), ("beta1", C.c_float),
                ("beta2", C.c_float), ("eps", C.c_float), ("device", C.c_int)]


class AnchorStats(C.Structure):
    _fields_ = [("surrogate_steps", C.c_int64), ("plain_steps", C.c_int64), ("anchors", C.c_int64),
                ("fallbacks", C.c_int64), ("last_rel_err", C.c_double), ("max_rel_err", C.c_double)]


SURROGATE_NETWORK, SURROGATE_FROZEN = 0, 1
SURROGATE_SYMBOLS = ["wbsph_surrogate_config_default", "wbsph_surrogate_create",
                     "wbsph_surrogate_num_params", "wbsph_surrogate_set_params",
                     "wbsph_surrogate_get_params", "wbsph_surrogate_set_normalization",
                     "wbsph_surrogate_set_mode",
                     "wbsph_surrogate_train_step", "wbsph_surrogate_eval", "wbsph_surrogate_predict",
                     "wbsph_surrogate_debug", "wbsph_step_surrogate", "wbsph_surrogate_destroy",
                     "wbsph_surrogate_last_error"]
SYMBOLS += SURROGATE_SYMBOLS


def _load_surrogate(L):
    if getattr(L, "_surrogate_sig", False):
        return L
    P, i64, I, F, D = C.c_void_p, C.c_int64, C.c_int, C.c_float, C.c_double
    sig = {
        "wbsph_surrogate_config_default": (I, [P, I]),
        "wbsph_surrogate_create": (I, [P, P]),
        "wbsph_surrogate_num_params": (i64, [P]),
        "wbsph_surrogate_set_params": (I, [P, P]),
        "wbsph_surrogate_get_params": (I, [P, P]),
        "wbsph_surrogate_set_normalization": (I, [P, P, P, P, P, P]),
        "wbsph_surrogate_set_mode": (I, [P, I]),
        "wbsph_surrogate_train_step": (I, [P, P, F, P]),
        "wbsph_surrogate_eval": (I, [P, P, P]),
        "wbsph_surrogate_predict": (I, [P, P]),
        "wbsph_surrogate_debug": (I, [P, P, P, P, P, P, P, P, P, P, P]),
        "wbsph_step_surrogate": (I, [P, P, i64, I, D, P]),
        "wbsph_surrogate_destroy": (None, [P]),
        "wbsph_surrogate_last_error": (C.c_char_p, [P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    L._surrogate_sig = True
    return L


class Surrogate:
    """BF16 message-passing surrogate; parameters live on the device."""

    def __init__(self, dim: int, device: int = 0, layers: int = 3):
        self.lib = _load_surrogate(load())
        cfg = SurrogateConfig()
        self.lib.wbsph_surrogate_config_default(C.byref(cfg), dim)
        cfg.layers = layers
        cfg.device = device
        h = C.c_void_p()
        rc = self.lib.wbsph_surrogate_create(C.byref(cfg), C.byref(h))
        if rc != OK:
            raise WbsphError(rc, "wbsph_surrogate_create failed")
        self.h = h
        self.dim = dim
        self.np = int(self.lib.wbsph_surrogate_num_params(h))

    def _check(self, rc, sim=None):
        if rc < 0:
            msg = self.lib.wbsph_surrogate_last_error(self.h).decode()
            if sim is not None:
                msg += " / " + sim.lib.wbsph_last_error(sim.h).decode()
            raise WbsphError(int(rc), msg)
        return rc

    def close(self):
        if getattr(self, "h", None):
            self.lib.wbsph_surrogate_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, theta):
        theta = np.ascontiguousarray(theta, dtype=np.float32)
        assert theta.size == self.np
        self._check(self.lib.wbsph_surrogate_set_params(self.h, _ptr(theta)))

    def get_params(self):
        out = np.empty(self.np, dtype=np.float32)
        self._check(self.lib.wbsph_surrogate_get_params(self.h, _ptr(out)))
        return out

    def set_normalization(self, node_mean, node_std, edge_std, out_mean, out_std):
        """Scales of the inputs and outputs: node (dim + 2 means and stds of
        U, rho/rho0 - 1, phi'), edge (s_U, s_phi) and output (dim + 1)."""
        a = [np.ascontiguousarray(v, dtype=np.float32)
             for v in (node_mean, node_std, edge_std, out_mean, out_std)]
        self._check(self.lib.wbsph_surrogate_set_normalization(self.h, *[_ptr(v) for v in a]))

    def set_mode(self, mode):
        """SURROGATE_NETWORK, or SURROGATE_FROZEN: the control whose surrogate
        stages replay the rates of the rollout's last plain stage."""
        self._check(self.lib.wbsph_surrogate_set_mode(self.h, int(mode)))

    def train_step(self, sim, lr):
        loss = C.c_double()
        self._check(self.lib.wbsph_surrogate_train_step(self.h, sim.h, float(lr), C.byref(loss)), sim)
        return loss.value

    def eval(self, sim):
        loss = C.c_double()
        self._check(self.lib.wbsph_surrogate_eval(self.h, sim.h, C.byref(loss)), sim)
        return loss.value

    def predict(self, sim):
        self._check(self.lib.wbsph_surrogate_predict(self.h, sim.h), sim)

    def edges(self, sim):
        """Number of graph edges (fluid receivers and their neighbours) at the
        sim's current state."""
        ne = C.c_int64()
        self._check(self.lib.wbsph_surrogate_debug(self.h, sim.h, C.byref(ne), None, None, None, None,
                                                   None, None, None, None), sim)
        return ne.value

    def debug(self, sim):
        ne = C.c_int64()
        self._check(self.lib.wbsph_surrogate_debug(self.h, sim.h, C.byref(ne), None, None, None, None,
                                                   None, None, None, None), sim)
        E = ne.value
        st = sim.stats()
        n, nf = st["n"], st["n_fluid"]
        recv = np.empty(E, np.uint32)
        send = np.empty(E, np.uint32)
        ef = np.empty((E, 8), np.float32)
        nfe = np.empty((n, 8), np.float32)
        fid = np.empty(nf, np.uint32)
        out = np.empty((nf, self.dim + 1), np.float32)
        grad = np.empty(self.np, np.float32)
        loss = C.c_double()
        self._check(self.lib.wbsph_surrogate_debug(self.h, sim.h, C.byref(ne), _ptr(recv), _ptr(send),
                                                   _ptr(ef), _ptr(nfe), _ptr(fid), _ptr(out), _ptr(grad),
                                                   C.byref(loss)), sim)
        return dict(recv=recv, send=send, edge_feat=ef, node_feat=nfe, fluid_ids=fid, out=out,
                    grad=grad, loss=loss.value)

    def step(self, sim, nsteps, anchor_every=10, tau=0.1):
        stats = AnchorStats()
        self._check(self.lib.wbsph_step_surrogate(sim.h, self.h, int(nsteps), int(anchor_every),
                                                  float(tau), C.byref(stats)), sim)
        return {k: getattr(stats, k) for k, _ in AnchorStats._fields_}
