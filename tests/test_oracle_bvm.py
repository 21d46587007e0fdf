"""Pins of the oracle's BVM coefficients, matrices A/B and Strang symbols (Sec. 2.2,
Sec. 3.1) against order conditions checked on polynomials, consistency, A_{nu,mu-nu}
stability, the displayed circulant s(A) and an FFT of its first column."""
from fractions import Fraction

import numpy as np
import pytest

import oracle as O

SCHEMES = [("GBDF", 1), ("GBDF", 2), ("GBDF", 3), ("GBDF", 4), ("GBDF", 5),
           ("GAM", 1), ("GAM", 2), ("GAM", 3), ("GAM", 4), ("GAM", 5), ("ETR", 3), ("ETR", 5)]


def _order(family, mu):
    return mu if family == "GBDF" else mu + 1


def _exact_on_poly(a, b, ell_pts, q):
    # formula sum_i a_i p(i) = sum_i b_i p'(i) for p(t) = t^q, exact rational arithmetic
    lhs = sum(ai * Fraction(i) ** q for i, ai in enumerate(a))
    rhs = sum(bi * (q * Fraction(i) ** (q - 1) if q > 0 else 0) for i, bi in enumerate(b))
    return lhs == rhs


@pytest.mark.parametrize("family,mu", SCHEMES)
def test_every_formula_has_the_stated_order(family, mu):
    p = _order(family, mu)
    for ell in range(1, mu + 1):
        a, b = O.lmf_coefficients(family, mu, ell)
        for q in range(p + 1):
            assert _exact_on_poly(a, b, None, q), (family, mu, ell, q)
        # structure of the family
        if family == "GBDF":
            assert b == [Fraction(int(i == ell)) for i in range(mu + 1)]
        else:
            assert a == [Fraction(1 if i == ell else (-1 if i == ell - 1 else 0)) for i in range(mu + 1)]


def test_textbook_coefficients():
    # classical values of the generalised BDF / Adams formulas used in the paper's experiments
    F = Fraction
    a, b = O.lmf_coefficients("GBDF", 3, 2)
    assert a == [F(1, 6), F(-1), F(1, 2), F(1, 3)]
    a, b = O.lmf_coefficients("GAM", 4, 2)  # fifth-order GAM, Sec. 4
    assert b == [F(-19, 720), F(346, 720), F(456, 720), F(-74, 720), F(11, 720)]
    a, b = O.lmf_coefficients("GAM", 1, 1)  # trapezoidal rule
    assert b == [F(1, 2), F(1, 2)]
    a, b = O.lmf_coefficients("GBDF", 1, 1)  # implicit Euler
    assert a == [F(-1), F(1)]
    a, b = O.lmf_coefficients("ETR", 3, 2)
    assert b == b[::-1]  # symmetric


@pytest.mark.parametrize("family,mu", SCHEMES)
def test_consistency_rho_sigma(family, mu):
    # Sec. 3.1: rho(1) = 0 and rho'(1) = sigma(1), rho/sigma of eq. (1.12)
    nu = O.nu_of(family, mu)
    a, b = O.lmf_coefficients(family, mu, nu)
    assert sum(a) == 0
    assert sum(i * ai for i, ai in enumerate(a)) == sum(b)


@pytest.mark.parametrize("family,mu", [("GBDF", 3), ("GBDF", 5), ("GAM", 4), ("ETR", 3), ("GAM", 2), ("GBDF", 1)])
def test_a_nu_mu_minus_nu_stability(family, mu):
    # Definition 3.1: rho(z) - q sigma(z) has nu zeros inside |z| = 1 and mu - nu outside, Re q < 0
    nu = O.nu_of(family, mu)
    a, b = O.lmf_coefficients(family, mu, nu)
    a = np.array([float(v) for v in a])
    b = np.array([float(v) for v in b])
    rng = np.random.default_rng(1)
    qs = np.concatenate([-rng.exponential(3.0, 200) + 1j * rng.normal(0, 5, 200),
                         -np.logspace(-3, 4, 50) + 0j, -1e-3 + 1j * np.logspace(-2, 3, 50)])
    for q in qs:
        poly = (a - q * b)[::-1]  # highest power first
        poly = np.trim_zeros(poly, "f")
        roots = np.roots(poly)
        inside = np.sum(np.abs(roots) < 1)
        outside = np.sum(np.abs(roots) > 1)
        # leading coefficient may vanish (GBDF: beta_mu = 0 ...) -> a root at infinity counts as outside
        outside += mu - len(roots)
        assert inside == nu and outside == mu - nu, (family, mu, q, roots)


@pytest.mark.parametrize("family,mu,s", [("GBDF", 3, 9), ("GBDF", 5, 12), ("GAM", 4, 10), ("ETR", 3, 7), ("GBDF", 1, 4)])
def test_matrices_integrate_polynomials_exactly(family, mu, s):
    """Every row t = 1..s of (A, B) is exact on t^q, q <= order, on the grid t_n = n h:
    sum_j A[t,j] p(t_j) = h sum_j B[t,j] p'(t_j).  This pins the column placement
    of the main, initial and final formulas (eqs. (1.7)-(1.9))."""
    A, B = O.bvm_matrices(family, mu, s, exact=True)
    nu = O.nu_of(family, mu)
    p = _order(family, mu)
    h = Fraction(1, s)
    for t in range(1, s + 1):
        for q in range(p + 1):
            lhs = sum(A[t][j] * (j * h) ** q for j in range(s + 1))
            rhs = h * sum(B[t][j] * (q * (j * h) ** (q - 1) if q else 0) for j in range(s + 1))
            assert lhs == rhs, (t, q)
        nz = [j for j in range(s + 1) if A[t][j] != 0 or B[t][j] != 0]
        start = 0 if t < nu else (t - nu if t <= s - mu + nu else s - mu)
        assert min(nz) >= start and max(nz) <= start + mu
    assert A[0][0] == 1 and all(v == 0 for v in A[0][1:]) and all(v == 0 for v in B[0])


def test_strang_circulant_first_row_as_displayed():
    # eq. (1.11) display: first row alpha_nu .. alpha_mu, zeros, alpha_0 .. alpha_{nu-1}
    a, _ = O.lmf_coefficients("GBDF", 5, 3)
    s, nu, mu = 11, 3, 5
    C = O.strang_circulant(a, nu, s)
    row = [float(v) for v in a[nu:]] + [0.0] * (s - mu - 1) + [float(v) for v in a[:nu]]
    np.testing.assert_array_equal(C[0], row)
    # last row: alpha_{nu+1} .. alpha_mu, zeros, alpha_0 .. alpha_nu
    last = [float(v) for v in a[nu + 1:]] + [0.0] * (s - mu - 1) + [float(v) for v in a[:nu + 1]]
    np.testing.assert_array_equal(C[-1], last)


@pytest.mark.parametrize("family,mu,s", [("GBDF", 3, 16), ("GBDF", 5, 32), ("GAM", 4, 64), ("ETR", 3, 8)])
def test_strang_symbols(family, mu, s):
    phi, psi = O.strang_symbols(family, mu, s)
    nu = O.nu_of(family, mu)
    a, b = O.lmf_coefficients(family, mu, nu)
    assert abs(phi[0]) < 1e-14  # phi_0 = rho(1) = 0 (Sec. 3.1)
    assert psi[0] == pytest.approx(float(sum(b)))  # psi_0 = sigma(1) = rho'(1)
    # eigenvalues of a circulant are the DFT of its first column (library FFT vs direct sum)
    C = O.strang_circulant(a, nu, s)
    np.testing.assert_allclose(phi, np.fft.fft(C[:, 0]), atol=1e-13)
    # and C v_k = phi_k v_k for the Fourier vectors v_k[n] = exp(2 pi i n k / s)
    n = np.arange(s)
    for k in range(s):
        v = np.exp(2j * np.pi * n * k / s)
        np.testing.assert_allclose(C @ v, phi[k] * v, atol=1e-12)
    Cb = O.strang_circulant(b, nu, s)
    np.testing.assert_allclose(psi, np.fft.fft(Cb[:, 0]), atol=1e-13)
    # conjugate symmetry of the symbols of real circulants
    np.testing.assert_allclose(phi[1:], np.conj(phi[1:][::-1]), atol=1e-14)
