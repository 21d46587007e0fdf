"""CPU-side checks of the C-ABI library: it builds, loads, and exports every
symbol that include/fde.h declares.  No compute call is made without a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fde.h")


@pytest.fixture(scope="module")
def lib():
    from paper_1305_6653_gb300 import _lib
    if not os.path.exists(_lib.LIB_PATH):
        from paper_1305_6653_gb300 import build
        build.build()
    return ctypes.CDLL(_lib.LIB_PATH)


def _declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:int|void|long long|const char\*|fde_problem\*)\s+\**(\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("fde_problem_create", "bvm_assemble", "strang_precond_factor", "pgmres_solve",
                     "fde_problem_destroy", "fde_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared_functions():
        assert hasattr(lib, name), name


def test_binding_lists_every_declared_symbol():
    from paper_1305_6653_gb300 import _lib
    assert sorted(_lib.EXPORTED) == _declared_functions()


def test_struct_layouts_match_header():
    from paper_1305_6653_gb300 import _lib
    # fde_problem_desc: 2 ints, 5 doubles, 2 pointers, 2 doubles, 2 ints, 2 pointers, 1 int (+ padding),
    # 2 pointers (time-dependent coefficients)
    assert ctypes.sizeof(_lib.FdeProblemDesc) == 8 + 40 + 16 + 16 + 8 + 16 + 8 + 16
    assert _lib.FdeProblemDesc.dplus_t.offset == 112 and _lib.FdeProblemDesc.dminus_t.offset == 120
    assert ctypes.sizeof(_lib.FdePgmresOpts) == 24
    assert ctypes.sizeof(_lib.FdeStats) == 16 + 24 + 8


def test_argument_validation_needs_no_gpu(lib):
    """fde_problem_create rejects bad arguments before touching the device."""
    from paper_1305_6653_gb300 import _lib
    L = _lib.load()
    d = _lib.FdeProblemDesc()
    d.m, d.s, d.alpha, d.xL, d.xR, d.t0, d.T, d.family, d.mu = 63, 32, 2.5, 0.0, 1.0, 0.0, 1.0, 1, 3
    h = ctypes.c_void_p()
    assert L.fde_problem_create(ctypes.byref(d), None, ctypes.byref(h)) == _lib.FDE_ERR_ARG
    assert b"alpha" in L.fde_last_error()
    d.alpha = 1.5
    d.s = 30  # not a power of two
    assert L.fde_problem_create(ctypes.byref(d), None, ctypes.byref(h)) == _lib.FDE_ERR_ARG
    d.s, d.family = 32, 9
    assert L.fde_problem_create(ctypes.byref(d), None, ctypes.byref(h)) == _lib.FDE_ERR_ARG
    d.family, d.mu = 3, 4  # ETR needs odd mu
    assert L.fde_problem_create(ctypes.byref(d), None, ctypes.byref(h)) == _lib.FDE_ERR_ARG
    d.family, d.mu = 1, 3
    one = (ctypes.c_double * 1)(1.0)
    d.u0 = d.f = ctypes.cast(one, ctypes.c_void_p)
    d.dplus_t = ctypes.cast(one, ctypes.c_void_p)  # d+(x, t) without d-(x, t)
    assert L.fde_problem_create(ctypes.byref(d), None, ctypes.byref(h)) == _lib.FDE_ERR_ARG
    assert b"dminus_t" in L.fde_last_error()
    d.dplus_t = None
    assert L.bvm_assemble(None) == _lib.FDE_ERR_ARG
    assert L.strang_precond_factor(None, 0) == _lib.FDE_ERR_ARG


def test_release_of_an_empty_device_cache_needs_no_gpu(lib):
    """With nothing cached, fde_release_cached_memory makes no CUDA call and succeeds."""
    from paper_1305_6653_gb300 import _lib, fde_release_cached_memory
    assert _lib.load().fde_release_cached_memory() == _lib.FDE_OK
    fde_release_cached_memory()
