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


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("make", [fi.config_small,
                                  lambda: fi.manufactured(100, 16, 1.8, "GBDF5", dplus_fn=lambda x: 1 + x,
                                                          dminus_fn=lambda x: 2 - x)],
                         ids=["m63_s32", "m100_s16"])
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


def test_noalloc_rejects_problems_beyond_the_static_scratch(lib):
    from paper_1305_6653_gb300 import FDEProblem, _lib
    prob = fi.manufactured(2047, 1024, 1.5, "GBDF3")  # 513 * 2048 complex FP64 values > 8 MiB
    with FDEProblem.from_inputs(prob) as p:
        r = torch.zeros(prob.n, dtype=torch.float64, device="cuda")
        z = torch.empty_like(r)
        rc = lib.fde_precond_apply_noalloc(p.h, ctypes.c_void_p(r.data_ptr()), ctypes.c_void_p(z.data_ptr()))
        assert rc == _lib.FDE_ERR_ARG
        assert b"8 MiB" in lib.fde_last_error()
