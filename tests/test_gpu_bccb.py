"""GPU parity of the Strang-type BCCB preconditioners S^(2) (eq. x1) and S~^(2)
(eq. xc) against the FP64 oracle's two-dimensional DFT apply (Sec. 3.3).

Tolerances (derived from the arithmetic): the GPU applies C_k^{-1} as a cyclic
convolution by length-L FFTs (L >= 2m) after the FFT along time, with the first
column of C_k^{-1} from a direct length-m DFT in FP64.  Each transform contributes
O(eps log2 L) relative error, amplified by the condition number kappa =
max|lambda| / min|lambda| of the preconditioner's eigenvalues (eq. 1.13; the
smallest sit at j = 0, where phi_0 = 0 and the partial sums of g are small):
FP64 tolerance kappa * 2.2e-16 * log2(2m) relative to ||z|| (kappa reaches 5e6 at
m = 2047); FP32 apply: 1e-4 relative on the small cases.  Solutions:
||x - x_oracle|| / ||x_oracle|| <= 1e-8.
"""
import numpy as np
import pytest

import fde_inputs as fi
import oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1305_6653_gb300 import _lib
    _lib.load()  # fails loudly if the library is missing
    torch.cuda.set_device(0)


def _variable(m, s, scheme, alpha=1.5):
    return fi.manufactured(m, s, alpha, scheme, dplus_fn=lambda x: 1.0 + x, dminus_fn=lambda x: 2.0 - x)


def _tol64(P, m):
    a = np.abs(P.D)
    return a.max() / a.min() * 2.2e-16 * np.log2(2 * m + 2)


def _gpu_bccb(prob, modified=False, precision="fp64"):
    from paper_1305_6653_gb300 import FDEProblem
    p = FDEProblem.from_inputs(prob)
    p.assemble()
    p.bccb(modified=modified, precision=precision)
    return p


CASES = [
    ("small", lambda: fi.config_small()),
    ("ragged_gbdf5", lambda: _variable(100, 16, "GBDF5", 1.8)),
    ("gam4_ex41", lambda: fi.example_4_1(1.2, 48, 32)),
    ("etr3_odd_m", lambda: _variable(37, 8, "ETR3", 1.3)),
    ("tiny_m1", lambda: _variable(1, 4, "GBDF1", 1.5)),
    ("m64_pow2", lambda: _variable(64, 16, "GAM4", 1.9)),
    ("m255_s64", lambda: _variable(255, 64, "GBDF3", 1.7)),
]


@pytest.mark.parametrize("modified", [False, True])
@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_apply_fp64(name, make, modified):
    prob = make()
    r = np.random.default_rng(7).standard_normal(prob.n)
    P = O.BCCBPreconditioner(prob, modified=modified)
    ref = P.apply(r)
    with _gpu_bccb(prob, modified) as p:
        z = p.precond_apply(torch.as_tensor(r, device="cuda")).cpu().numpy()
    assert np.linalg.norm(z - ref) <= _tol64(P, prob.m) * np.linalg.norm(ref)


@pytest.mark.parametrize("name,make", CASES[:4], ids=[c[0] for c in CASES[:4]])
def test_apply_fp32(name, make):
    prob = make()
    r = np.random.default_rng(8).standard_normal(prob.n)
    ref = O.BCCBPreconditioner(prob).apply(r)
    with _gpu_bccb(prob, precision="fp32") as p:
        z = p.precond_apply(torch.as_tensor(r, device="cuda")).cpu().numpy()
    assert np.linalg.norm(z - ref) <= 1e-4 * np.linalg.norm(ref)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("modified", [False, True])
def test_solve_matches_direct_solution(modified, precision):
    prob = _variable(100, 16, "GBDF5", 1.8)
    ref = O.direct_solve(prob)
    with _gpu_bccb(prob, modified, precision) as p:
        x, st = p.solve(tol=1e-11, maxit=2000)
        x = x.cpu().numpy()
    assert st["status"] == 0 and st["rel_residual"] <= 1e-11
    assert np.linalg.norm(x - ref) <= 1e-8 * np.linalg.norm(ref)


@pytest.mark.parametrize("alpha,n,s", [(1.2, 24, 16), (1.5, 48, 32), (1.5, 96, 64)])
def test_iterations_match_the_oracle(alpha, n, s):
    # the same right-preconditioned flexible GMRES(20) with the true-residual test
    prob = fi.example_4_1(alpha, n, s)
    _, its, ok, _ = O.solve_bccb_gmres(prob, tol=1e-10, restart=20)
    with _gpu_bccb(prob) as p:
        _, st = p.solve(tol=1e-10, restart=20, maxit=2000)
    assert ok and st["status"] == 0
    assert abs(st["iterations"] - its) <= 1, (st["iterations"], its)


def test_fullsize_apply():
    # the benchmark workload (m = 2047, s = 256) against the oracle's 2-D FFT apply
    prob = fi.config_scale(2047, 256)
    r = np.random.default_rng(9).standard_normal(prob.n)
    P = O.BCCBPreconditioner(prob)
    ref = P.apply(r)
    from paper_1305_6653_gb300 import FDEProblem
    with FDEProblem.from_inputs(prob) as p:
        p.assemble().bccb()
        z = p.precond_apply(torch.as_tensor(r, device="cuda")).cpu().numpy()
    assert np.linalg.norm(z - ref) <= _tol64(P, prob.m) * np.linalg.norm(ref)


def test_switch_back_to_the_block_preconditioner():
    # strang_precond_factor after bccb_precond_setup selects S (eq. 1.11) again
    prob = _variable(100, 16, "GBDF5", 1.8)
    r = np.random.default_rng(10).standard_normal(prob.n)
    ref_s = O.StrangPreconditioner(prob).apply(r)
    Pb, Pm = O.BCCBPreconditioner(prob), O.BCCBPreconditioner(prob, modified=True)
    ref_b = Pb.apply(r)
    from paper_1305_6653_gb300 import FDEProblem
    with FDEProblem.from_inputs(prob) as p:
        p.assemble().bccb()
        zb = p.precond_apply(torch.as_tensor(r, device="cuda")).cpu().numpy()
        p.factor("fp64")
        zs = p.precond_apply(torch.as_tensor(r, device="cuda")).cpu().numpy()
        p.bccb(modified=True)
        zm = p.precond_apply(torch.as_tensor(r, device="cuda")).cpu().numpy()
    assert np.linalg.norm(zb - ref_b) <= _tol64(Pb, prob.m) * np.linalg.norm(ref_b)
    assert np.linalg.norm(zs - ref_s) <= 1e-10 * np.linalg.norm(ref_s)
    ref_m = Pm.apply(r)
    assert np.linalg.norm(zm - ref_m) <= _tol64(Pm, prob.m) * np.linalg.norm(ref_m)


def test_state_errors():
    from paper_1305_6653_gb300 import FDEProblem, FdeError, _lib
    prob = _variable(37, 8, "GBDF3", 1.4)
    with FDEProblem.from_inputs(prob) as p:
        with pytest.raises(FdeError):
            p.bccb()  # before bvm_assemble
        p.assemble()
        with pytest.raises(FdeError):
            p.bccb(precision="tf32")  # the BCCB apply is FP64 or FP32
        p.bccb()
        with pytest.raises(FdeError):
            p.factor_block(0)  # no block LU under the BCCB preconditioner
        r = torch.zeros(prob.n, dtype=torch.float64, device="cuda")
        z = torch.empty_like(r)
        import ctypes as C
        rc = _lib.load().fde_precond_apply_noalloc(p.h, C.c_void_p(r.data_ptr()), C.c_void_p(z.data_ptr()))
        assert rc == _lib.FDE_ERR_STATE


def test_no_preconditioner_is_plain_gmres():
    # column I of Tables 1-2: fde_precond_none gives plain restarted GMRES; the iteration
    # count follows the oracle's unpreconditioned GMRES(20) with the same true-residual test
    prob = fi.example_4_1(1.2, 24, 16)
    _, its, ok, _ = O.gmres(lambda z: O.matvec(prob, z), O.reduced_rhs(prob), side="none", restart=20, tol=1e-10,
                            reference="b", maxit=5000)
    ref = O.direct_solve(prob)
    from paper_1305_6653_gb300 import FDEProblem
    with FDEProblem.from_inputs(prob) as p:
        p.assemble().no_precond()
        x, st = p.solve(tol=1e-10, restart=20, maxit=5000)
        x = x.cpu().numpy()
    assert ok and st["status"] == 0
    assert abs(st["iterations"] - its) <= max(2, 0.05 * its), (st["iterations"], its)
    assert np.linalg.norm(x - ref) <= 1e-7 * np.linalg.norm(ref)
