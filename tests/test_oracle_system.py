"""Pins of the oracle's all-at-once system (eq. (1.10)), its reduced form, the
Strang preconditioner (eq. (1.11), Sec. 3.2), Theorem 3.3 and GMRES."""
import os

import numpy as np
import pytest

import fde_inputs as fi
import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_tables_its.txt")


def _tiny(m, s, scheme, alpha=1.5, variable=True):
    if variable:
        return fi.manufactured(m, s, alpha, scheme, dplus_fn=lambda x: 1.0 + x, dminus_fn=lambda x: 2.0 - x)
    return fi.manufactured(m, s, alpha, scheme)


@pytest.mark.parametrize("m,s,scheme", [(5, 12, "GBDF3"), (6, 16, "GBDF5"), (5, 12, "GAM4"), (7, 9, "ETR3")])
def test_reduced_system_has_the_full_solution(m, s, scheme):
    # eq. (1.10) solved as printed ((s+1) m unknowns) vs the reduced system (u_0 eliminated)
    p = _tiny(m, s, scheme)
    M, rhs = O.full_system(p)
    u_full = np.linalg.solve(M, rhs)
    np.testing.assert_allclose(u_full[:m], p.u0, rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(u_full[m:], O.direct_solve(p), rtol=1e-11, atol=1e-14)


@pytest.mark.parametrize("m,s,scheme", [(9, 12, "GBDF3"), (6, 16, "GBDF5"), (11, 10, "GAM4")])
def test_kronecker_matvec_and_rhs_match_dense(m, s, scheme):
    p = _tiny(m, s, scheme)
    M, b = O.reduced_system(p)
    z = np.random.default_rng(0).standard_normal(m * s)
    np.testing.assert_allclose(O.matvec(p, z), M @ z, rtol=1e-12, atol=1e-12 * np.abs(M).max())
    np.testing.assert_allclose(O.reduced_rhs(p), b, rtol=1e-12, atol=1e-13)


def test_manufactured_solution_small_config():
    # m = 63, s = 32, GBDF3: max error ~7.5e-4 against u = exp(-t) x^2 (1-x)^2
    p = fi.config_small()
    u = O.direct_solve(p).reshape(p.s, p.m)
    exact = fi.manufactured_exact(p.x, p.t)[1:]
    err = np.abs(u - exact).max()
    assert 1e-4 < err < 1e-3


def test_manufactured_error_first_order_in_space():
    # shifted Grunwald is first order in dx; the GBDF5 time error (h^5) is negligible here
    errs = []
    for m in (15, 31, 63):
        p = fi.manufactured(m, 16, 1.5, "GBDF5", dplus_fn=lambda x: 1.0 + x, dminus_fn=lambda x: 2.0 - x)
        u = O.direct_solve(p).reshape(p.s, p.m)
        errs.append(np.abs(u - fi.manufactured_exact(p.x, p.t)[1:]).max())
    assert 1.6 < errs[0] / errs[1] < 2.6 and 1.6 < errs[1] / errs[2] < 2.6, errs


@pytest.mark.parametrize("m,s,scheme,sym", [(5, 12, "GBDF3", True), (6, 16, "GBDF5", False), (5, 12, "GAM4", True),
                                            (4, 7, "ETR3", True), (6, 16, "GBDF5", True)])
def test_strang_apply_equals_dense_inverse(m, s, scheme, sym):
    p = _tiny(m, s, scheme)
    S = O.strang_matrix(p)
    P = O.StrangPreconditioner(p, conjugate_symmetry=sym)
    r = np.random.default_rng(1).standard_normal(m * s)
    np.testing.assert_allclose(P.apply(r), np.linalg.solve(S, r), rtol=1e-11, atol=1e-13)


@pytest.mark.parametrize("m,s,scheme", [(5, 12, "GBDF3"), (6, 16, "GBDF5"), (7, 8, "GAM4")])
def test_strang_matvec_matches_dense(m, s, scheme):
    p = _tiny(m, s, scheme)
    z = np.random.default_rng(4).standard_normal(m * s)
    np.testing.assert_allclose(O.strang_matvec(p, z), O.strang_matrix(p) @ z, rtol=1e-12, atol=1e-10)


@pytest.mark.parametrize("m,s,scheme", [(5, 12, "GBDF3"), (6, 16, "GBDF5"), (5, 12, "GAM4"), (4, 10, "ETR3")])
def test_theorem_3_3_rank_and_iterations(m, s, scheme):
    """S^{-1} M = I + L with rank L <= 2 m mu; full GMRES converges in <= rank + 1 steps."""
    p = _tiny(m, s, scheme)
    M, b = O.reduced_system(p)
    S = O.strang_matrix(p)
    L = np.linalg.solve(S, M) - np.eye(m * s)
    rank = np.linalg.matrix_rank(L, tol=1e-9 * np.abs(L).max())
    mu = p.mu
    assert rank <= 2 * m * mu
    assert rank == mu * m  # tighter count: corrections live on nu + (mu - nu) block rows
    P = O.StrangPreconditioner(p)
    _, its, ok, _ = O.gmres(lambda z: M @ z, b, precond=P.apply, side="left", restart=m * s,
                            tol=1e-10, maxit=m * s)
    assert ok and its <= rank + 1


def test_strang_blocks_are_nonsingular_and_diagonally_dominant():
    # Theorem 3.1 / Corollary 3.2: S invertible for A_{nu,mu-nu}-stable BVMs and Re lambda(J) < 0;
    # the blocks phi_k I - h psi_k J are strictly row diagonally dominant (derived).
    for scheme in ("GBDF3", "GBDF5", "GAM4", "ETR3"):
        p = _tiny(31, 32, scheme, alpha=1.9)
        P = O.StrangPreconditioner(p)
        for k in range(p.s // 2 + 1):
            Bk = P.block(k)
            d = np.abs(np.diag(Bk))
            off = np.abs(Bk).sum(axis=1) - d
            assert np.all(d > off), (scheme, k)


def test_gmres_unpreconditioned_matches_numpy_solve():
    rng = np.random.default_rng(3)
    n = 60
    A = np.eye(n) * 4 + rng.standard_normal((n, n)) / np.sqrt(n)
    b = rng.standard_normal(n)
    x, its, ok, _ = O.gmres(lambda v: A @ v, b, side="none", restart=7, tol=1e-13, reference="b")
    assert ok
    np.testing.assert_allclose(x, np.linalg.solve(A, b), rtol=1e-11, atol=1e-12)


@pytest.mark.parametrize("side", ["left", "right"])
def test_strang_gmres_matches_direct_solve(side):
    p = fi.config_small()
    u = O.direct_solve(p)
    x, its, ok, _ = O.solve_strang_gmres(p, side=side, tol=1e-12)
    assert ok and its < 40
    assert np.linalg.norm(x - u) / np.linalg.norm(u) < 1e-10


def _golden():
    rows = []
    for line in open(GOLDEN):
        if line.strip() and not line.startswith("#"):
            a, n, s, i_its, s_its = line.split()
            rows.append((float(a), int(n), int(s), int(i_its), int(s_its)))
    return rows


@pytest.mark.parametrize("row", _golden(), ids=lambda r: f"a{r[0]}-n{r[1]}-s{r[2]}")
def test_paper_tables_iteration_counts(row):
    """Tables 1-2 of Sec. 4: ITS of GMRES(20) for the I and S columns of Example 4.1.

    Tolerance: S within +-1 iteration; I within 15% (the printed counts come from
    MATLAB's gmres, whose Householder Arnoldi and restart bookkeeping differ)."""
    alpha, n, s, its_I, its_S = row
    p = fi.example_4_1(alpha, n, s)
    J = O.j_of(p)
    AB = O.bvm_matrices(p.family, p.mu, p.s)
    mv = lambda z: O.matvec(p, z, J=J, AB=AB)  # noqa: E731
    b = O.reduced_rhs(p, J=J)
    P = O.StrangPreconditioner(p, J=J)
    _, got_S, okS, _ = O.gmres(mv, b, precond=P.apply, side="left", restart=20, tol=1e-8)
    _, got_I, okI, _ = O.gmres(mv, b, side="none", restart=20, tol=1e-8)
    assert okS and okI
    assert abs(got_S - its_S) <= 1, (got_S, its_S)
    assert abs(got_I - its_I) <= 0.15 * its_I, (got_I, its_I)
