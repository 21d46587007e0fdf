"""GB300-native Strang-preconditioned BVM/GMRES solver for space-fractional diffusion.

Method: Gu, Huang, Zhao, Li & Li, "Strang-type preconditioners for solving
fractional diffusion equations by boundary value methods" (arXiv:1305.6653).

The compute path is libfde.so (CUDA, sm_103a) behind the C ABI of include/fde.h.
This package is the thin Python binding: it marshals arguments (PyTorch only
provides device memory and the CUDA stream) and calls the library with the same
entry-point names.  Importing the package does not load the library; the first
call does, and fails loudly if it is missing.
"""
from __future__ import annotations

import ctypes as C

from . import _lib
from ._lib import (FDE_BF16, FDE_ETR, FDE_FP32, FDE_FP64, FDE_GAM, FDE_GBDF, FDE_TF32, FdeError,  # noqa: F401
                   FdePgmresOpts, FdeProblemDesc, FdeStats, PRECISIONS, FAMILIES)

__all__ = ["FDEProblem", "FDEBatch", "FDENop", "fde_problem_create", "bvm_assemble", "strang_precond_factor",
           "bccb_precond_setup", "pgmres_solve",
           "fde_problem_destroy", "fde_matvec", "fde_precond_apply", "fde_release_cached_memory", "FdeError",
           "PRECISIONS"]


def _torch():
    import torch
    return torch


def _stream_handle(stream):
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


# ---- thin wrappers with the C-ABI names ------------------------------------

def fde_problem_create(desc: FdeProblemDesc, stream=None) -> C.c_void_p:
    h = C.c_void_p()
    _lib.check(_lib.load().fde_problem_create(C.byref(desc), _stream_handle(stream), C.byref(h)),
               "fde_problem_create")
    return h


def bvm_assemble(h) -> None:
    _lib.check(_lib.load().bvm_assemble(h), "bvm_assemble")


def strang_precond_factor(h, precision) -> None:
    prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    _lib.check(_lib.load().strang_precond_factor(h, prec), "strang_precond_factor")


def bccb_precond_setup(h, modified: bool = False, precision="fp64") -> None:
    prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    _lib.check(_lib.load().bccb_precond_setup(h, 1 if modified else 0, prec), "bccb_precond_setup")


def pgmres_solve(h, opts: FdePgmresOpts, x0_ptr: int | None, x_ptr: int, raise_on_error: bool = True) -> FdeStats:
    st = FdeStats()
    rc = _lib.load().pgmres_solve(h, C.byref(opts), C.c_void_p(x0_ptr) if x0_ptr else None, C.c_void_p(x_ptr),
                                  C.byref(st))
    if raise_on_error:
        _lib.check(rc, "pgmres_solve")
    return st


def fde_launch_count() -> int:
    return int(_lib.load().fde_launch_count())


def fde_release_cached_memory() -> None:
    """Return the library's cached device buffers to the CUDA driver."""
    _lib.check(_lib.load().fde_release_cached_memory(), "fde_release_cached_memory")


def fde_tune_set(kernel: int, variant: int) -> None:
    """Force a launch-shape variant of a tuned kernel family (-1: autotune)."""
    _lib.check(_lib.load().fde_tune_set(int(kernel), int(variant)), "fde_tune_set")


def fde_tune_cache(path: str | None) -> None:
    """Use `path` for the tuning table (None or "": memory only)."""
    _lib.check(_lib.load().fde_tune_cache(path.encode() if path else None), "fde_tune_cache")


def fde_tune_query(kernel: int, mp: int, nb: int, precision) -> int:
    prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    v = C.c_int()
    _lib.check(_lib.load().fde_tune_query(int(kernel), int(mp), int(nb), prec, C.byref(v)), "fde_tune_query")
    return v.value


def fde_problem_destroy(h) -> None:
    if h:
        _lib.load().fde_problem_destroy(h)


def fde_matvec(h, z_ptr: int, y_ptr: int) -> None:
    _lib.check(_lib.load().fde_matvec(h, C.c_void_p(z_ptr), C.c_void_p(y_ptr)), "fde_matvec")


def fde_precond_apply(h, r_ptr: int, z_ptr: int) -> None:
    _lib.check(_lib.load().fde_precond_apply(h, C.c_void_p(r_ptr), C.c_void_p(z_ptr)), "fde_precond_apply")


# ---- convenience object ------------------------------------------------------

def _as_host_vector(a, n):
    """A contiguous float64 CPU tensor of length n (moved from the device if needed)."""
    torch = _torch()
    t = torch.as_tensor(a, dtype=torch.float64)
    if t.is_cuda:
        t = t.cpu()
    t = t.contiguous().reshape(-1)
    if t.numel() != n:
        raise ValueError(f"expected {n} values, got {t.numel()}")
    return t


class FDEProblem:
    """One instance of eq. (1.1) on the device.

    Inputs (dplus, dminus, u0, f) may be numpy arrays (host, copied by the
    library) or CUDA float64 tensors (device).  The solve vectors follow the
    inputs (the desc's device_ptrs): a problem built from device tensors takes
    and returns CUDA float64 tensors, one built from host arrays takes and
    returns CPU float64 tensors (the library copies them on its stream).  The
    step-level vectors (matvec, precond_apply, rhs) are CUDA tensors; all are
    length s*m, time-major (u_1 .. u_s).
    """

    def __init__(self, *, m, s, alpha, xL, xR, t0, T, dplus, dminus, u0, f, family, mu, stream=None,
                 device_inputs: bool | None = None, dplus_t=None, dminus_t=None):
        torch = _torch()
        self.m, self.s = int(m), int(s)
        self.n = self.m * self.s
        self.stream = stream
        fam = FAMILIES[family] if isinstance(family, str) else int(family)
        keep = []

        def ptr(a):
            if a is None:
                return None
            if isinstance(a, torch.Tensor):
                t = a.contiguous().to(torch.float64)
                keep.append(t)
                return t.data_ptr()
            import numpy as np
            arr = np.ascontiguousarray(a, dtype=np.float64)
            keep.append(arr)
            return arr.ctypes.data

        if device_inputs is None:
            device_inputs = isinstance(u0, torch.Tensor) and u0.is_cuda
        self.device_ptrs = bool(device_inputs)
        self.desc = FdeProblemDesc(self.m, self.s, float(alpha), float(xL), float(xR), float(t0), float(T),
                                   ptr(dplus), ptr(dminus), 0.0, 0.0, fam, int(mu), ptr(u0), ptr(f),
                                   1 if device_inputs else 0, ptr(dplus_t), ptr(dminus_t))
        self.h = fde_problem_create(self.desc, stream)
        del keep

    @classmethod
    def from_inputs(cls, prob, stream=None, device_inputs: bool = False):
        """Build from an fde_inputs.Problem (host arrays unless device_inputs)."""
        torch = _torch()
        fam, mu = prob.family, prob.mu
        arrays = dict(dplus=prob.dplus, dminus=prob.dminus, u0=prob.u0, f=prob.f)
        if getattr(prob, "dplus_t", None) is not None:
            arrays.update(dplus_t=prob.dplus_t, dminus_t=prob.dminus_t)
        if device_inputs:
            arrays = {k: torch.as_tensor(v, dtype=torch.float64, device="cuda") for k, v in arrays.items()}
        return cls(m=prob.m, s=prob.s, alpha=prob.alpha, xL=prob.xL, xR=prob.xR, t0=prob.t0, T=prob.T,
                   family=fam, mu=mu, stream=stream, device_inputs=device_inputs, **arrays)

    def assemble(self):
        bvm_assemble(self.h)
        return self

    def factor(self, precision="fp64", storage="fp32"):
        """Strang-block LU in `precision`; `storage` ("fp32" or "bf16") is the storage of
        the copy of the factors the block solves stream (tensor-core precisions)."""
        _lib.check(_lib.load().fde_factor_storage(self.h, _lib.STORAGES[storage]), "fde_factor_storage")
        strang_precond_factor(self.h, precision)
        return self

    def no_precond(self):
        """Plain GMRES (no preconditioner) for the solves."""
        _lib.check(_lib.load().fde_precond_none(self.h), "fde_precond_none")
        return self

    def bccb(self, modified=False, precision="fp64"):
        """Select the Strang-type BCCB preconditioner S^(2) (or S~^(2)) for the solves."""
        bccb_precond_setup(self.h, modified, precision)
        return self

    def solve(self, tol=1e-10, restart=20, maxit=1000, reorth=1, x0=None, out=None, raise_on_error=True,
              matvec="fp64", relax=0.0):
        """pgmres_solve (matvec="fp32": the Arnoldi products' Toeplitz apply in FP32 while
        the residual estimate is above relax, see fde_pgmres_opts).  Device problems: x0 / out are CUDA tensors.  Host problems:
        x0 / out are CPU tensors (a CUDA x0 is copied to the host first, so that the
        library receives the host pointer its desc declared)."""
        torch = _torch()
        if self.device_ptrs:
            x = out if out is not None else torch.empty(self.n, dtype=torch.float64, device="cuda")
            if not x.is_cuda:
                raise ValueError("this problem was created from device inputs: out must be a CUDA tensor")
            if x0 is not None:
                x0 = torch.as_tensor(x0, dtype=torch.float64, device="cuda").contiguous()
        else:
            x = out if out is not None else torch.empty(self.n, dtype=torch.float64)
            if x.is_cuda:
                raise ValueError("this problem was created from host inputs: its solve writes host memory, "
                                 "pass a CPU tensor as out")
            if x0 is not None:
                x0 = _as_host_vector(x0, self.n)
        opts = FdePgmresOpts(float(tol), int(restart), int(maxit), int(reorth), PRECISIONS[matvec], float(relax))
        st = pgmres_solve(self.h, opts, x0.data_ptr() if x0 is not None else None, x.data_ptr(),
                          raise_on_error=raise_on_error)
        return x, st.as_dict()

    def matvec(self, z):
        torch = _torch()
        y = torch.empty(self.n, dtype=torch.float64, device="cuda")
        fde_matvec(self.h, z.data_ptr(), y.data_ptr())
        return y

    def matvec_fp32(self, z):
        """y = M z with the Toeplitz apply in FP32 (fde_matvec_fp32)."""
        torch = _torch()
        y = torch.empty(self.n, dtype=torch.float64, device="cuda")
        _lib.check(_lib.load().fde_matvec_fp32(self.h, C.c_void_p(z.data_ptr()), C.c_void_p(y.data_ptr())),
                   "fde_matvec_fp32")
        return y

    def precond_apply(self, r):
        torch = _torch()
        z = torch.empty(self.n, dtype=torch.float64, device="cuda")
        fde_precond_apply(self.h, r.data_ptr(), z.data_ptr())
        return z

    def rhs(self):
        torch = _torch()
        b = torch.empty(self.n, dtype=torch.float64, device="cuda")
        _lib.check(_lib.load().fde_get_rhs(self.h, C.c_void_p(b.data_ptr())), "fde_get_rhs")
        return b

    def grunwald(self):
        import numpy as np
        g = np.empty(self.m + 2)
        _lib.check(_lib.load().fde_get_grunwald(self.h, C.c_void_p(g.ctypes.data)), "fde_get_grunwald")
        return g

    def factor_block(self, k):
        import numpy as np
        re = np.empty((self.m, self.m))
        im = np.empty((self.m, self.m))
        _lib.check(_lib.load().fde_get_factor_block(self.h, int(k), C.c_void_p(re.ctypes.data),
                                                     C.c_void_p(im.ctypes.data)), "fde_get_factor_block")
        return re + 1j * im

    def profile(self, on: bool = True):
        _lib.check(_lib.load().fde_profile_enable(self.h, 1 if on else 0), "fde_profile_enable")
        return self

    def profile_select(self, stages=()):
        """Time only the named stages (e.g. ["trsv"]) and keep the iteration graphs
        (fde_profile_select); an empty list stops recording."""
        mask = 0
        for name in stages:
            mask |= 1 << _lib.STAGES.index(name)
        _lib.check(_lib.load().fde_profile_select(self.h, C.c_uint(mask)), "fde_profile_select")
        return self

    def profile_read(self) -> dict:
        out = {}
        for i, name in enumerate(_lib.STAGES):
            ms = C.c_double()
            cnt = C.c_int()
            _lib.check(_lib.load().fde_profile_read(self.h, i, C.byref(ms), C.byref(cnt)), "fde_profile_read")
            out[name] = (ms.value, cnt.value)
        return out

    def close(self):
        if getattr(self, "h", None):
            fde_problem_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class FDEBatch:
    """A batch of independent instances solved together (fde_batch_* entry points).

    problems: list of fde_inputs.Problem (or objects with the same fields).  With
    device_inputs the arrays are first placed in device memory (desc device_ptrs = 1)
    and the solutions are CUDA tensors; otherwise the library copies host arrays and
    the solutions are CPU tensors."""

    def __init__(self, problems, stream=None, device_inputs: bool = False):
        import numpy as np
        torch = _torch()
        self.count = len(problems)
        self.sizes = [(p.m, p.s) for p in problems]
        self.device_ptrs = bool(device_inputs)
        self._keep = []
        descs = (FdeProblemDesc * self.count)()

        def ptr(a):
            if device_inputs:
                t = torch.as_tensor(np.asarray(a, dtype=np.float64), device="cuda").contiguous()
                self._keep.append(t)
                return t.data_ptr()
            arr = np.ascontiguousarray(a, dtype=np.float64)
            self._keep.append(arr)
            return arr.ctypes.data

        for i, p in enumerate(problems):
            arrs = [ptr(a) for a in (p.dplus, p.dminus, p.u0, p.f)]
            descs[i] = FdeProblemDesc(p.m, p.s, float(p.alpha), float(p.xL), float(p.xR), float(p.t0), float(p.T),
                                      arrs[0], arrs[1], 0.0, 0.0, FAMILIES[p.family],
                                      int(p.mu), arrs[2], arrs[3], 1 if device_inputs else 0)
            if getattr(p, "dplus_t", None) is not None:  # rejected by the library: not batched
                tv = [np.ascontiguousarray(a, dtype=np.float64) for a in (p.dplus_t, p.dminus_t)]
                self._keep.extend(tv)
                descs[i].dplus_t, descs[i].dminus_t = tv[0].ctypes.data, tv[1].ctypes.data
        self.h = C.c_void_p()
        _lib.check(_lib.load().fde_batch_create(descs, self.count, _stream_handle(stream), C.byref(self.h)),
                   "fde_batch_create")
        self._keep = []

    def share_operator(self):
        """All instances have one operator (only u0 and f differ): factor once, share the factors."""
        _lib.check(_lib.load().fde_batch_share_operator(self.h), "fde_batch_share_operator")
        return self

    def block_solver(self, kind="auto"):
        """Block solves of a shared-operator batch: "cuda_cores" (FP32, groups of 8),
        "tensor_cores" (TF32 tcgen05 products, groups of 16) or "auto"; before factor()."""
        _lib.check(_lib.load().fde_batch_block_solver(self.h, _lib.BLOCK_SOLVERS[kind]), "fde_batch_block_solver")
        return self

    def assemble(self):
        _lib.check(_lib.load().fde_batch_assemble(self.h), "fde_batch_assemble")
        return self

    def factor(self, precision="fp32", storage="fp32"):
        """Factor every instance; `storage` ("fp32" or "bf16") is set on each instance
        (fde_factor_storage) before the batched LU."""
        L = _lib.load()
        for i in range(L.fde_batch_size(self.h)):
            _lib.check(L.fde_factor_storage(C.c_void_p(L.fde_batch_problem(self.h, i)), _lib.STORAGES[storage]),
                       "fde_factor_storage")
        prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        _lib.check(L.fde_batch_factor(self.h, prec), "fde_batch_factor")
        return self

    def solve(self, tol=1e-10, restart=20, maxit=1000, reorth=1, outs=None, raise_on_error=True):
        torch = _torch()
        dev = "cuda" if self.device_ptrs else "cpu"
        if outs is None:
            outs = [torch.empty(m * s, dtype=torch.float64, device=dev) for m, s in self.sizes]
        if any(o.is_cuda != self.device_ptrs for o in outs):
            raise ValueError(f"this batch's solutions are {'device' if self.device_ptrs else 'host'} memory: "
                             f"pass {dev} tensors as outs")
        ptrs = (C.c_void_p * self.count)(*[o.data_ptr() for o in outs])
        stats = (FdeStats * self.count)()
        opts = FdePgmresOpts(float(tol), int(restart), int(maxit), int(reorth))
        rc = _lib.load().fde_batch_solve(self.h, C.byref(opts), ptrs, stats)
        if raise_on_error:
            _lib.check(rc, "fde_batch_solve")
        return outs, [st.as_dict() for st in stats]

    def problem(self, i):
        """Problem handle of instance i (owned by the batch)."""
        return C.c_void_p(_lib.load().fde_batch_problem(self.h, int(i)))

    def close(self):
        if getattr(self, "h", None):
            _lib.load().fde_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class FDENop:
    """Learned warm start (fde_nop_* entry points): a 1-D convolutional neural
    operator along the sine-mode axis, trained and run by the library's own kernels."""

    def __init__(self, m, s, modes=16, width=64, layers=6, ksize=5, seed=1305, stream=None):
        self.m, self.s, self.modes = int(m), int(s), int(modes)
        self.h = C.c_void_p()
        _lib.check(_lib.load().fde_nop_create(self.m, self.s, self.modes, int(width), int(layers), int(ksize),
                                              int(seed), _stream_handle(stream), C.byref(self.h)), "fde_nop_create")
        self.nparam = int(_lib.load().fde_nop_num_params(self.h))
        self.cin = int(_lib.load().fde_nop_in_channels(self.h))

    def set_params(self, params):
        import numpy as np
        a = np.ascontiguousarray(params, dtype=np.float32)
        assert a.size == self.nparam
        _lib.check(_lib.load().fde_nop_set_params(self.h, C.c_void_p(a.ctypes.data)), "fde_nop_set_params")

    def get_params(self):
        import numpy as np
        a = np.empty(self.nparam, dtype=np.float32)
        _lib.check(_lib.load().fde_nop_get_params(self.h, C.c_void_p(a.ctypes.data)), "fde_nop_get_params")
        return a

    def forward(self, x, batch):
        torch = _torch()
        out = torch.empty(batch * self.s * self.modes, dtype=torch.float32, device="cuda")
        _lib.check(_lib.load().fde_nop_forward(self.h, C.c_void_p(x.data_ptr()), C.c_void_p(out.data_ptr()),
                                                int(batch)), "fde_nop_forward")
        return out

    def loss_grad(self, x, target, batch, want_grad=False):
        import numpy as np
        loss = C.c_double()
        g = np.empty(self.nparam, dtype=np.float32) if want_grad else None
        _lib.check(_lib.load().fde_nop_loss_grad(self.h, C.c_void_p(x.data_ptr()), C.c_void_p(target.data_ptr()),
                                                  int(batch), C.byref(loss),
                                                  C.c_void_p(g.ctypes.data) if want_grad else None),
                   "fde_nop_loss_grad")
        return loss.value, g

    def adam_step(self, lr):
        _lib.check(_lib.load().fde_nop_adam_step(self.h, C.c_float(lr)), "fde_nop_adam_step")

    def features(self, problem_handle, out):
        _lib.check(_lib.load().fde_nop_features(self.h, problem_handle, C.c_void_p(out.data_ptr())),
                   "fde_nop_features")

    def coefficients(self, x, out):
        _lib.check(_lib.load().fde_nop_coefficients(self.h, C.c_void_p(x.data_ptr()), C.c_void_p(out.data_ptr())),
                   "fde_nop_coefficients")

    def synthesize(self, coef, out):
        _lib.check(_lib.load().fde_nop_synthesize(self.h, C.c_void_p(coef.data_ptr()), C.c_void_p(out.data_ptr())),
                   "fde_nop_synthesize")

    def warm_start(self, problem_handle, x0):
        _lib.check(_lib.load().fde_nop_warm_start(self.h, problem_handle, C.c_void_p(x0.data_ptr())),
                   "fde_nop_warm_start")

    def close(self):
        if getattr(self, "h", None):
            _lib.load().fde_nop_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
