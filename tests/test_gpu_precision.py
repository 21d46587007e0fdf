"""Precision study (m=4095, s=128, alpha=1.9, d+=d-=1, 3-step GBDF, manufactured
solution; 524,160 unknowns, 65 complex 4095 x 4095 Strang blocks): every
preconditioner precision inside the FP64 flexible GMRES against the oracle's
FP64 Strang-preconditioned FGMRES solution.

The bar is the same as everywhere else: rel.err <= 1e-8 against the oracle and a
true FP64 residual <= 1e-10 under the oracle's Kronecker matvec.  The oracle's
own FGMRES floors a little above 1e-11 at this size, so its reference is taken at
3e-11 (its error against the exact discrete solution is then ~1e-10 or less).
Each variant prints one line (iterations, true residual, error, solve time) so a
run with -s records the per-precision table.
"""
import numpy as np
import pytest

import fde_inputs as fi
import oracle as O

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    prob = fi.config_precision()
    J = O.j_of(prob)
    b = O.reduced_rhs(prob, J=J)
    return prob, J, b


@pytest.fixture(scope="module")
def oracle_solution(setup):
    prob, _, _ = setup
    x, its, ok, _ = O.solve_strang_gmres(prob, side="right", tol=3e-11, maxit=100)
    assert ok, its
    return x


@pytest.mark.parametrize("precision", ["fp64", "fp32", "tf32", "tf32x3", "bf16"])
def test_precision_variant(setup, oracle_solution, precision):
    from paper_1305_6653_gb300 import FDEProblem
    prob, J, b = setup
    with FDEProblem.from_inputs(prob, device_inputs=True) as p:
        p.assemble().factor(precision)
        x, st = p.solve(tol=1e-10, restart=20, maxit=400)
        xs = x.cpu().numpy()
    assert st["status"] == 0, st
    res = np.linalg.norm(b - O.matvec(prob, xs, J=J)) / np.linalg.norm(b)
    err = np.linalg.norm(xs - oracle_solution) / np.linalg.norm(oracle_solution)
    print(f"\nprecision m={prob.m} s={prob.s} {precision}: iterations={st['iterations']} "
          f"true_res={res:.3e} rel_err_vs_oracle={err:.3e} solve_ms={st['ms_solve']:.1f}")
    assert res <= 1e-10, res
    assert err <= 1e-8, err
    assert st["iterations"] <= 2 * prob.m * prob.mu + 1  # Theorem 3.3 bound
