"""Pins of the oracle's time-dependent coefficients d+-(x, t) (eq. (1.1) allows them; the
paper's experiments use d+-(x)): the BVM applied to u' = J(t) u + f(t) gives the block
(B (x) I) blkdiag(J_0, .., J_s) in place of B (x) J, and the Strang preconditioner uses
the time-averaged J."""
import numpy as np
import pytest

import fde_inputs as fi
import oracle as O


def test_constant_in_time_reduces_to_the_time_independent_system():
    p = fi.manufactured(9, 8, 1.6, "GBDF3", dplus_fn=lambda x: 1.0 + x, dminus_fn=lambda x: 2.0 - x)
    q = fi.manufactured(9, 8, 1.6, "GBDF3", dplus_fn=lambda x: 1.0 + x, dminus_fn=lambda x: 2.0 - x)
    q.dplus_t = np.tile(q.dplus, (q.s + 1, 1))
    q.dminus_t = np.tile(q.dminus, (q.s + 1, 1))
    Mp, bp = O.reduced_system(p)
    Mq, bq = O.reduced_system(q)
    np.testing.assert_allclose(Mq, Mp, rtol=1e-13, atol=1e-13 * np.abs(Mp).max())
    np.testing.assert_allclose(bq, bp, rtol=1e-13, atol=1e-15)
    z = np.random.default_rng(1).standard_normal(p.n)
    np.testing.assert_allclose(O.matvec(q, z), O.matvec(p, z), rtol=1e-12, atol=1e-12 * np.abs(Mp).max())


@pytest.mark.parametrize("m,s,scheme", [(7, 8, "GBDF3"), (12, 16, "GBDF5"), (9, 10, "GAM4")])
def test_block_matvec_and_rhs_match_the_dense_system(m, s, scheme):
    p = fi.manufactured_time_varying(m, s, 1.7, scheme)
    M, b = O.reduced_system(p)
    z = np.random.default_rng(2).standard_normal(p.n)
    np.testing.assert_allclose(O.matvec(p, z), M @ z, rtol=1e-12, atol=1e-12 * np.abs(M).max())
    np.testing.assert_allclose(O.reduced_rhs(p), b, rtol=1e-12, atol=1e-13)
    # the time levels differ: J_1 != J_s
    assert np.abs(O.j_at(p, 1) - O.j_at(p, s)).max() > 1e-3 * np.abs(O.j_at(p, 1)).max()


def test_manufactured_error_first_order_in_space():
    errs = []
    for m in (15, 31, 63):
        p = fi.manufactured_time_varying(m, 16, 1.5, "GBDF5")
        u = O.direct_solve(p).reshape(p.s, p.m)
        errs.append(np.abs(u - fi.manufactured_exact(p.x, p.t)[1:]).max())
    assert 1.6 < errs[0] / errs[1] < 2.6 and 1.6 < errs[1] / errs[2] < 2.6, errs


def test_time_averaged_strang_preconditioner_converges():
    p = fi.manufactured_time_varying(31, 16, 1.7, "GBDF3")
    x, its, ok, _ = O.solve_strang_gmres(p, tol=1e-12)
    u = O.direct_solve(p)
    assert ok and its < 40
    assert np.linalg.norm(x - u) / np.linalg.norm(u) < 1e-10
    # the preconditioner's J is the mean of J_1..J_s
    Jbar = np.mean([O.j_at(p, n) for n in range(1, p.s + 1)], axis=0)
    np.testing.assert_allclose(O.j_of(p), Jbar, rtol=1e-12, atol=1e-12 * np.abs(Jbar).max())


def test_time_level_matvec_matches_fft_toeplitz_products():
    """J_n z_n = dx^-alpha (D+(t_n) G z_n + D-(t_n) G^T z_n) (eq. (1.4) at each time
    level), with G z and G^T z taken as Toeplitz products by scipy's FFT route and
    the BVM band applied after: an evaluation independent of the oracle's dense J_n."""
    from scipy.linalg import matmul_toeplitz

    prob = fi.manufactured_time_varying(255, 32, 1.6, "GBDF3")
    m, s = prob.m, prob.s
    z = np.random.default_rng(5).standard_normal(m * s)
    g = O.grunwald_weights(prob.alpha, m + 1)
    col = g[1:m + 1]
    row = np.zeros(m)
    row[0], row[1] = g[1], g[0]
    Z = z.reshape(s, m)
    GZ = matmul_toeplitz((col, row), Z.T).T
    GtZ = matmul_toeplitz((row, col), Z.T).T
    JZ = (prob.dplus_t[1:] * GZ + prob.dminus_t[1:] * GtZ) / prob.dx ** prob.alpha
    A, B = O.bvm_matrices(prob.family, prob.mu, s)
    ref = (A[1:, 1:] @ Z - prob.h * (B[1:, 1:] @ JZ)).reshape(-1)
    got = O.matvec(prob, z)
    assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref)
