"""Host-side checks of the C-ABI library: it builds for sm_103a, loads, and
exports every function that include/wbsph.h declares (no compute calls)."""
import ctypes
import os
import re

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
