"""ctypes wrapper of the FP64 CPU oracle (test infrastructure only).

``build()`` compiles ``wbsph_oracle.c`` with gcc into ``oracle/_build``;
the wrapper functions take numpy arrays in structure-of-arrays layout
(``x[k, i]``) and a parameter dict as produced by the scene generators.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "wbsph_oracle.c")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "liboracle.so")

NSUMS = 31
ERRORS = {-1: "invalid argument", -2: "out of memory", -4: "particle outside the domain",
          -5: "singular renormalisation matrix", -6: "non-finite value",
          -9: "output capacity too small"}


class OracleError(RuntimeError):
    def __init__(self, code, what):
        super().__init__(f"{what}: {ERRORS.get(code, 'error')} ({code})")
        self.code = code


class Config(C.Structure):
    _fields_ = [("dim", C.c_int), ("dx", C.c_double), ("h_over_dx", C.c_double),
                ("rho0", C.c_double), ("c0", C.c_double), ("nu", C.c_double),
                ("g", C.c_double * 3), ("cfl", C.c_double), ("delta", C.c_double),
                ("pst_R", C.c_double), ("pst_n", C.c_double), ("tic_lambda", C.c_double),
                ("use_delta", C.c_int), ("use_pst", C.c_int), ("use_tic", C.c_int),
                ("use_visc", C.c_int), ("eos", C.c_int), ("tait_gamma", C.c_double),
                ("domain_min", C.c_double * 3), ("domain_max", C.c_double * 3),
                ("force_amp", C.c_double * 3), ("force_period", C.c_double),
                ("fixed_dt", C.c_double), ("umax_override", C.c_double),
                ("scheme", C.c_int), ("art_alpha", C.c_double), ("wall_bc", C.c_int),
                ("body_u", C.c_double * 3)]

# parameters with defaults when a parameter set does not name them
_DEFAULTS = {"umax_override": -1.0, "scheme": 0, "art_alpha": 0.02, "wall_bc": 0, "body_u": [0.0, 0.0, 0.0]}


_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle (gcc, -O2, OpenMP, no floating-point contraction)."""
    os.makedirs(BUILD, exist_ok=True)
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < max(
            os.path.getmtime(SRC), os.path.getmtime(os.path.join(HERE, "wbsph_oracle.h"))):
        tmp = LIB + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
               "-fno-fast-math", "-Wall", "-o", tmp, SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, LIB)
    return LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(LIB)
            P = C.c_void_p
            i64 = C.c_int64
            L.orc_neighbors.restype = i64
            for name, args in {
                "orc_kernel_eval": [P, i64, P, P, P],
                "orc_cell_keys": [P, i64, P, P],
                "orc_sort_by_key": [i64, P, P],
                "orc_neighbors": [P, i64, P, C.c_int, P, P, i64],
                "orc_mass": [P, i64, P, P],
                "orc_density": [P, i64, P, P],
                "orc_pressure": [P, i64, P, P],
                "orc_eig_min_sym": [C.c_int, P, P],
                "orc_dummy_update": [P, i64, P, P, P, P, P, C.c_double],
                "orc_pair_sums": [P, i64, P, P, P, P, P, C.c_int, P],
                "orc_stage_rates": [P, i64, P, P, P, P, P, P, C.c_double, P, P, P, P, P],
                "orc_time_step": [P, i64, P, P, P],
                "orc_step": [P, i64, P, P, P, P, P, P, P, i64, P, P, P, P, P],
                "orc_l2_velocity": [P, i64, P, P, P, P, P, P],
                "orc_num_threads": [],
            }.items():
                f = getattr(L, name)
                f.argtypes = args
                if name != "orc_neighbors":
                    f.restype = C.c_int
            _lib = L
    return _lib


def make_config(params: dict) -> Config:
    c = Config()
    for name, _ in Config._fields_:
        v = params.get(name, _DEFAULTS[name]) if name in _DEFAULTS else params[name]
        if isinstance(v, (list, tuple, np.ndarray)):
            arr = getattr(c, name)
            for k in range(3):
                arr[k] = float(v[k]) if k < len(v) else 0.0
        else:
            setattr(c, name, v)
    return c


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _check(rc, what):
    if rc < 0:
        raise OracleError(int(rc), what)
    return rc


def num_threads() -> int:
    return int(lib().orc_num_threads())


def kernel(params, r):
    r = _f64(r)
    w = np.empty_like(r)
    dw = np.empty_like(r)
    c = make_config(params)
    _check(lib().orc_kernel_eval(C.byref(c), r.size, _p(r), _p(w), _p(dw)), "kernel")
    return w, dw


def cell_keys(params, x):
    x = _f64(x)
    n = x.shape[1]
    k = np.empty(n, dtype=np.uint32)
    c = make_config(params)
    _check(lib().orc_cell_keys(C.byref(c), n, _p(x), _p(k)), "cell_keys")
    return k


def sort_by_key(keys):
    keys = np.ascontiguousarray(keys, dtype=np.uint32)
    perm = np.empty(keys.size, dtype=np.uint32)
    _check(lib().orc_sort_by_key(keys.size, _p(keys), _p(perm)), "sort_by_key")
    return perm


def neighbors(params, x, brute=False):
    """CSR neighbour lists (row_ptr int64, cols int32), rows ascending."""
    x = _f64(x)
    n = x.shape[1]
    c = make_config(params)
    row = np.empty(n + 1, dtype=np.int64)
    nnz = _check(lib().orc_neighbors(C.byref(c), n, _p(x), int(brute), _p(row), None, 0),
                 "neighbors")
    cols = np.empty(max(nnz, 1), dtype=np.int32)
    _check(lib().orc_neighbors(C.byref(c), n, _p(x), int(brute), _p(row), _p(cols), nnz),
           "neighbors")
    return row, cols[:nnz]


def mass(params, phi):
    phi = _f64(phi)
    m = np.empty_like(phi)
    c = make_config(params)
    _check(lib().orc_mass(C.byref(c), phi.size, _p(phi), _p(m)), "mass")
    return m


def density(params, phi):
    phi = _f64(phi)
    r = np.empty_like(phi)
    c = make_config(params)
    _check(lib().orc_density(C.byref(c), phi.size, _p(phi), _p(r)), "density")
    return r


def pressure(params, phi):
    phi = _f64(phi)
    r = np.empty_like(phi)
    c = make_config(params)
    _check(lib().orc_pressure(C.byref(c), phi.size, _p(phi), _p(r)), "pressure")
    return r


def eig_min_sym(dim, a):
    a = _f64(np.asarray(a).reshape(-1))
    m = np.zeros(9)
    d = dim
    m.reshape(3, 3)[:d, :d] = a.reshape(d, d)
    lam = np.zeros(1)
    _check(lib().orc_eig_min_sym(d, _p(m), _p(lam)), "eig_min_sym")
    return float(lam[0])


def dummy_update(params, x, u, phi, typ, normal, t=0.0):
    x, u, phi, normal = _f64(x), _f64(u).copy(), _f64(phi).copy(), _f64(normal)
    typ = np.ascontiguousarray(typ, dtype=np.uint8)
    c = make_config(params)
    _check(lib().orc_dummy_update(C.byref(c), phi.size, _p(x), _p(u), _p(phi), _p(typ),
                                  _p(normal), float(t)), "dummy_update")
    return u, phi


def pair_sums(params, x, u, phi, m, typ, all_types=False):
    """Raw pair sums per particle, shape (n, 31): L(9) S(3) M(9) C(3) D P(3) Lambda(3)."""
    x, u, phi, m = _f64(x), _f64(u), _f64(phi), _f64(m)
    typ = np.ascontiguousarray(typ, dtype=np.uint8)
    n = phi.size
    out = np.zeros((n, NSUMS))
    c = make_config(params)
    _check(lib().orc_pair_sums(C.byref(c), n, _p(x), _p(u), _p(phi), _p(m), _p(typ),
                               int(all_types), _p(out)), "pair_sums")
    return out


class Rates(dict):
    pass


def stage_rates(params, x, u, phi, m, typ, normal, t=0.0, umax=None):
    """One stage of rates at the given state (dummy update applied to
    copies of u and phi). ``umax`` (optional) replaces the U_max of the
    shifting term, for rates of a patch cut from a larger scene. Returns
    dict with dudt, dphidt, dushift, lam, umax, u, phi (after the dummy
    update)."""
    x, u, phi, m, normal = _f64(x), _f64(u).copy(), _f64(phi).copy(), _f64(m), _f64(normal)
    typ = np.ascontiguousarray(typ, dtype=np.uint8)
    d, n = x.shape
    dudt = np.zeros((d, n))
    dushift = np.zeros((d, n))
    dphidt = np.zeros(n)
    lam = np.zeros(n)
    params = dict(params, umax_override=-1.0 if umax is None else float(umax))
    umax = np.zeros(1)
    c = make_config(params)
    _check(lib().orc_stage_rates(C.byref(c), n, _p(x), _p(u), _p(phi), _p(m), _p(typ),
                                 _p(normal), float(t), _p(dudt), _p(dphidt), _p(dushift),
                                 _p(lam), _p(umax)), "stage_rates")
    return Rates(dudt=dudt, dphidt=dphidt, dushift=dushift, lam=lam, umax=float(umax[0]),
                 u=u, phi=phi)


def time_step(params, u, typ):
    u = _f64(u)
    typ = np.ascontiguousarray(typ, dtype=np.uint8)
    dt = np.zeros(1)
    c = make_config(params)
    _check(lib().orc_time_step(C.byref(c), u.shape[1], _p(u), _p(typ), _p(dt)), "time_step")
    return float(dt[0])


class State:
    """Oracle particle state in the caller's order (the oracle never reorders)."""

    def __init__(self, scene, mass_override=None):
        self.params = dict(scene.params)
        self.x = _f64(scene.x).copy()
        self.u = _f64(scene.u).copy()
        self.phi = _f64(scene.phi).copy()
        self.type = np.ascontiguousarray(scene.type, dtype=np.uint8).copy()
        self.normal = _f64(scene.normal).copy()
        self.m = mass(self.params, self.phi) if mass_override is None else _f64(mass_override)
        self.t = 0.0
        d, n = self.x.shape
        self.dudt = np.zeros((d, n))
        self.dushift = np.zeros((d, n))
        self.dphidt = np.zeros(n)
        self.lam = np.zeros(n)
        self.dt = 0.0

    def step(self, nsteps=1):
        c = make_config(self.params)
        t = np.array([self.t])
        dt = np.zeros(1)
        _check(lib().orc_step(C.byref(c), self.phi.size, _p(self.x), _p(self.u), _p(self.phi),
                              _p(self.m), _p(self.type), _p(self.normal), _p(t), int(nsteps),
                              _p(dt), _p(self.dudt), _p(self.dphidt), _p(self.dushift),
                              _p(self.lam)), "step")
        self.t = float(t[0])
        self.dt = float(dt[0])
        return self

    def l2_velocity(self):
        l2 = np.zeros(1)
        um = np.zeros(1)
        c = make_config(self.params)
        _check(lib().orc_l2_velocity(C.byref(c), self.phi.size, _p(self.u), _p(self.phi),
                                     _p(self.m), _p(self.type), _p(l2), _p(um)), "l2_velocity")
        return float(l2[0]), float(um[0])
