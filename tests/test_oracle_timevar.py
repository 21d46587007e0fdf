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
