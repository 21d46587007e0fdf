"""fde_precond_apply_noalloc: the allocation-free preconditioner apply.

Some callers cannot allocate device memory when they apply the preconditioner
(an application whose memory manager owns the device after start-up, or code
that must not risk cudaMalloc's implicit synchronisation).  The entry point keeps
its frequency-domain scratch in a static device array instead.  These tests call
it through the C ABI and compare it with fde_precond_apply, whose scratch the
library allocates, on two calls in a row (the static array keeps the previous
call's contents, so the second call checks that nothing stale leaks in).

This file is collected last on purpose; it also passes when run alone.
"""
import ctypes

import numpy as np
import pytest

import fde_inputs as fi

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    from paper_1305_6653_gb300 import _lib
    return _lib.load()


def _apply(lib, name, h, r):
    z = torch.empty_like(r)
    rc = getattr(lib, name)(h, ctypes.c_void_p(r.data_ptr()), ctypes.c_void_p(z.data_ptr()))
    assert rc == 0, lib.fde_last_error()
    return z


def _m64():
    # m = 64 = mp: no padding column, so the transform fills the whole block row
    return fi.manufactured(64, 32, 1.4, "GAM4")


@pytest.mark.parametrize("precision", ["fp64", "fp32", "tf32"])
@pytest.mark.parametrize("make", [fi.config_small,
                                  lambda: fi.manufactured(100, 16, 1.8, "GBDF5", dplus_fn=lambda x: 1 + x,
                                                          dminus_fn=lambda x: 2 - x),
                                  _m64],
                         ids=["m63_s32", "m100_s16", "m64_s32"])
def test_noalloc_matches_precond_apply(lib, precision, make):
    from paper_1305_6653_gb300 import FDEProblem
    prob = make()
    rng = np.random.default_rng(21)
    with FDEProblem.from_inputs(prob) as p:
        p.assemble().factor(precision)
        for call in range(2):  # two calls in a row: the shared array keeps the last call's contents
            r = torch.as_tensor(rng.standard_normal(prob.n), device="cuda")
            z_ref = _apply(lib, "fde_precond_apply", p.h, r)
            z_new = _apply(lib, "fde_precond_apply_noalloc", p.h, r)
            torch.cuda.synchronize()
            err = (z_new - z_ref).norm().item() / z_ref.norm().item()
            assert err <= 1e-10, (call, err)


def test_noalloc_stale_scratch_never_reaches_the_result(lib):
    """Back to back through the shared array: an FP64 problem with a wide block row,
    then an FP32 problem with a narrower one (other mp, other element size), then the
    FP64 problem again.  Each result must equal fde_precond_apply's."""
    from paper_1305_6653_gb300 import FDEProblem
    rng = np.random.default_rng(5)
    wide = fi.manufactured(190, 64, 1.6, "GBDF3")   # mp = 192, FP64
    narrow = fi.manufactured(70, 16, 1.3, "ETR3")   # mp = 128, FP32
    with FDEProblem.from_inputs(wide) as pw, FDEProblem.from_inputs(narrow) as pn:
        pw.assemble().factor("fp64")
        pn.assemble().factor("fp32")
        for p, prob in ((pw, wide), (pn, narrow), (pw, wide), (pn, narrow)):
            r = torch.as_tensor(rng.standard_normal(prob.n), device="cuda")
            z_new = _apply(lib, "fde_precond_apply_noalloc", p.h, r)
            z_ref = _apply(lib, "fde_precond_apply", p.h, r)
            torch.cuda.synchronize()
            err = (z_new - z_ref).norm().item() / z_ref.norm().item()
            assert err <= 1e-10, (prob.m, err)


def _call(lib, p, n):
    r = torch.ones(n, dtype=torch.float64, device="cuda")
    z = torch.empty_like(r)
    return lib.fde_precond_apply_noalloc(p.h, ctypes.c_void_p(r.data_ptr()), ctypes.c_void_p(z.data_ptr()))


def test_noalloc_rejects_unfactored_problems(lib):
    from paper_1305_6653_gb300 import FDEProblem, _lib
    prob = fi.manufactured(2047, 1024, 1.5, "GBDF3")  # would also exceed the scratch: the state comes first
    with FDEProblem.from_inputs(prob) as p:
        p.assemble()
        assert _call(lib, p, prob.n) == _lib.FDE_ERR_STATE


@pytest.mark.parametrize("precision,m,fits", [
    ("fp64", 960, True),    # 513 * 960 = 492,480 <= 524,288 complex FP64 values
    ("fp64", 1024, False),  # 513 * 1024 = 525,312
    ("tf32", 1984, True),   # 513 * 1984 = 1,017,792 <= 1,048,576 complex FP32 values
    ("tf32", 1985, False),  # mp = 2048: 513 * 2048 = 1,050,624
])
def test_noalloc_size_limit_follows_the_factor_precision(lib, precision, m, fits):
    from paper_1305_6653_gb300 import FDEProblem, _lib
    prob = fi.manufactured(m, 1024, 1.5, "GBDF3")
    with FDEProblem.from_inputs(prob) as p:
        p.assemble().factor(precision)
        rc = _call(lib, p, prob.n)
        if fits:
            assert rc == 0, lib.fde_last_error()
            r = torch.as_tensor(np.random.default_rng(8).standard_normal(prob.n), device="cuda")
            z_new = _apply(lib, "fde_precond_apply_noalloc", p.h, r)
            z_ref = _apply(lib, "fde_precond_apply", p.h, r)
            torch.cuda.synchronize()
            assert (z_new - z_ref).norm().item() <= 1e-10 * z_ref.norm().item()
        else:
            assert rc == _lib.FDE_ERR_ARG
            assert b"8 MiB" in lib.fde_last_error()
    from paper_1305_6653_gb300 import _lib as L
    L.load().fde_release_cached_memory()
