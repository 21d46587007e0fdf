"""CPU check of the bfloat16 factor copy's effect on the method (no GPU).

The block solves can stream a copy of the Strang blocks' LU factors rounded to
bfloat16 (8-bit significand, rounding to nearest even), while the diagonal 32 x 32
tiles enter through their FP32 inverses.  The preconditioner is then the exact
inverse of slightly perturbed factors, and the flexible outer iteration (Sec. 3.2
GMRES, right-preconditioned, stopping on the true residual) absorbs the perturbation
at the cost of a few iterations.  Here the exact factors of the oracle's blocks are
rounded the same way in plain numpy, and the oracle's FGMRES is run with the
perturbed preconditioner: it must still reach the tolerance, with at most three more
iterations than the exact preconditioner, and its solution must match the direct
solve.  (Rounding the diagonal tiles as well makes ||S z - r|| four to ten times
larger and costs one more iteration in these cases; the design keeps them in FP32.)
"""
import numpy as np
import pytest
import scipy.linalg as sla

import fde_inputs as fi
import oracle as O


def _lu_nopivot(B):
    """Doolittle LU without pivoting (the Strang blocks are strictly row diagonally
    dominant): returns the unit lower L and the upper U."""
    A = B.astype(np.complex128).copy()
    n = A.shape[0]
    for k in range(n - 1):
        A[k + 1:, k] /= A[k, k]
        A[k + 1:, k + 1:] -= np.outer(A[k + 1:, k], A[k, k + 1:])
    return np.tril(A, -1) + np.eye(n), np.triu(A)


def _bf16(x):
    """Round float values to bfloat16 (to nearest even), returned as float64."""
    u = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def _round_off_diagonal_tiles(F, tile=32):
    """bfloat16 copy of a factor, the diagonal tile x tile blocks kept exact."""
    G = _bf16(F.real) + 1j * _bf16(F.imag)
    for t in range(0, F.shape[0], tile):
        G[t:t + tile, t:t + tile] = F[t:t + tile, t:t + tile]
    return G


class _RoundedStrang:
    """S^{-1} r as StrangPreconditioner.apply, with each block's unpivoted LU factors
    replaced by their bfloat16 copy (diagonal tiles exact)."""

    def __init__(self, prob, J):
        self.s, self.m = prob.s, prob.m
        phi, psi = O.strang_symbols(prob.family, prob.mu, prob.s)
        n = np.arange(prob.s)
        self.F = np.exp(-2j * np.pi * np.outer(n, n) / prob.s)
        self.Finv = np.exp(2j * np.pi * np.outer(n, n) / prob.s) / prob.s
        self.fac = {}
        for k in range(prob.s // 2 + 1):
            L, U = _lu_nopivot(phi[k] * np.eye(prob.m) - prob.h * psi[k] * J)
            self.fac[k] = (_round_off_diagonal_tiles(L), _round_off_diagonal_tiles(U))

    def _solve(self, k, v):
        L, U = self.fac[k]
        y = sla.solve_triangular(L, v, lower=True, unit_diagonal=True, check_finite=False)
        return sla.solve_triangular(U, y, lower=False, check_finite=False)

    def apply(self, r):
        s = self.s
        Rhat = self.F @ r.reshape(s, self.m)
        Xhat = np.empty_like(Rhat)
        for k in range(s):
            Xhat[k] = self._solve(k, Rhat[k]) if k in self.fac else np.conj(self._solve(s - k, np.conj(Rhat[k])))
        return (self.Finv @ Xhat).real.reshape(-1)


def test_bf16_rounding_of_a_value():
    # 1 + 2^-8 is a tie between 1 and 1 + 2^-7: to even (1); 1 + 3 * 2^-8 rounds up
    v = _bf16(np.array([1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, -2.5, 1.0 + 2.0 ** -7]))
    assert list(v) == [1.0, 1.0, 1.0 + 2.0 ** -6, -2.5, 1.0 + 2.0 ** -7]


@pytest.mark.parametrize("m,s,scheme,alpha", [(127, 16, "GBDF5", 1.8), (95, 32, "GBDF3", 1.5)])
def test_rounded_factor_copy_costs_a_few_iterations(m, s, scheme, alpha):
    prob = fi.manufactured(m, s, alpha, scheme, dplus_fn=lambda x: 1 + x, dminus_fn=lambda x: 2 - x)
    J = O.j_of(prob)
    AB = O.bvm_matrices(prob.family, prob.mu, prob.s)
    b = O.reduced_rhs(prob, J=J)
    mv = lambda z: O.matvec(prob, z, J=J, AB=AB)  # noqa: E731
    exact = O.StrangPreconditioner(prob, J=J)
    rounded = _RoundedStrang(prob, J)
    x0, its0, ok0, _ = O.gmres(mv, b, precond=exact.apply, side="right", restart=20, tol=1e-10, maxit=200,
                               reference="b")
    x1, its1, ok1, _ = O.gmres(mv, b, precond=rounded.apply, side="right", restart=20, tol=1e-10, maxit=200,
                               reference="b")
    assert ok0 and ok1
    assert its1 <= its0 + 3, (its0, its1)
    ref = O.direct_solve(prob)
    assert np.linalg.norm(x1 - ref) <= 1e-8 * np.linalg.norm(ref)
    # the copy does perturb the preconditioner: S z = r no longer holds exactly
    r = np.random.default_rng(3).standard_normal(prob.n)
    srel = np.linalg.norm(O.strang_matvec(prob, rounded.apply(r), J=J) - r) / np.linalg.norm(r)
    assert 1e-6 < srel < 0.5, srel
