"""GPU parity for time-dependent coefficients d+-(x, t) (eq. (1.1)): the matvec applies
J_n = dx^-alpha (D+(t_n) G + D-(t_n) G^T) at every time level and combines the BVM
band afterwards; the right-hand side uses J_0; the Strang preconditioner is built
from the time-averaged coefficients.  Tolerances as in test_gpu_parity.py (the
same FFT Toeplitz apply, bounded by the largest coefficient over all time levels)."""
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


CASES = [
    ("gbdf3_m63_s16", lambda: fi.manufactured_time_varying(63, 16, 1.5, "GBDF3")),
    ("gbdf5_m100_s32", lambda: fi.manufactured_time_varying(100, 32, 1.8, "GBDF5")),
    ("gam4_m37_s8", lambda: fi.manufactured_time_varying(37, 8, 1.3, "GAM4")),
    ("etr3_m255_s64", lambda: fi.manufactured_time_varying(255, 64, 1.7, "ETR3")),
]


def _gpu(prob, precision=None, device_inputs=False):
    from paper_1305_6653_gb300 import FDEProblem
    p = FDEProblem.from_inputs(prob, device_inputs=device_inputs)
    p.assemble()
    if precision:
        p.factor(precision)
    return p


def _jscale(prob):
    return 2 * prob.alpha * (prob.dplus_t + prob.dminus_t).max() * prob.dx ** (-prob.alpha)


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_rhs_and_matvec(name, make):
    prob = make()
    z = np.random.default_rng(21).standard_normal(prob.n)
    with _gpu(prob) as p:
        b = p.rhs().cpu().numpy()
        y = p.matvec(torch.as_tensor(z, device="cuda")).cpu().numpy()
    ref_b = O.reduced_rhs(prob)
    scale_b = np.abs(ref_b).max() + prob.h * _jscale(prob) * np.abs(prob.u0).max()
    assert np.abs(b - ref_b).max() <= 1e-12 * scale_b
    ref_y = O.matvec(prob, z)
    scale_y = prob.h * _jscale(prob) * np.abs(z).max() + 4 * np.abs(z).max()
    assert np.abs(y - ref_y).max() <= 1e-12 * scale_y


@pytest.mark.parametrize("device_inputs", [False, True])
@pytest.mark.parametrize("precision", ["fp64", "tf32"])
def test_solve_matches_direct_solution(precision, device_inputs):
    prob = fi.manufactured_time_varying(63, 32, 1.6, "GBDF5")
    ref = O.direct_solve(prob)
    with _gpu(prob, precision, device_inputs) as p:
        x, st = p.solve(tol=1e-11, maxit=400)
        xs = x.cpu().numpy()
    assert st["status"] == 0, st
    assert np.linalg.norm(xs - ref) <= 1e-8 * np.linalg.norm(ref)
    b = O.reduced_rhs(prob)
    res = np.linalg.norm(b - O.matvec(prob, xs)) / np.linalg.norm(b)
    assert res <= 1e-10 and abs(res - st["rel_residual"]) <= 1e-11


def test_larger_instance_true_residual():
    # m = 1023, s = 128: no dense solve; the oracle's time-dependent matvec judges the residual
    prob = fi.manufactured_time_varying(1023, 128, 1.8, "GBDF5")
    with _gpu(prob, "tf32") as p:
        x, st = p.solve(tol=1e-10, maxit=400)
        xs = x.cpu().numpy()
    assert st["status"] == 0, st
    b = O.reduced_rhs(prob)
    res = np.linalg.norm(b - O.matvec(prob, xs)) / np.linalg.norm(b)
    assert res <= 2e-10, res
    # against the manufactured solution: first-order spatial error
    err = np.abs(xs.reshape(prob.s, prob.m) - fi.manufactured_exact(prob.x, prob.t)[1:]).max()
    assert err < 2e-4, err


def test_batches_reject_time_dependent_coefficients():
    from paper_1305_6653_gb300 import FDEBatch, FdeError
    with pytest.raises(FdeError):
        FDEBatch([fi.manufactured_time_varying(63, 16, 1.5, "GBDF3")])
