"""Pins of the oracle's Grunwald weights and the matrix J (Sec. 2.1) against closed
forms, Proposition 2.1, Proposition 2.2 / Remark 2.1 and the fractional derivative
the shifted Grunwald formula approximates."""
import math

import numpy as np
import pytest
from scipy.special import binom, gamma

import oracle as O


@pytest.mark.parametrize("alpha", [1.1, 1.2, 1.5, 1.8, 1.9])
def test_weights_match_product_definition(alpha):
    # eq. (1.2): g_k = (-1)^k / k! * alpha (alpha-1) ... (alpha-k+1) = (-1)^k binom(alpha, k)
    g = O.grunwald_weights(alpha, 40)
    for k in range(41):
        prod = 1.0
        for i in range(k):
            prod *= (alpha - i)
        ref = (-1) ** k * prod / math.factorial(k)
        assert g[k] == pytest.approx(ref, rel=1e-13, abs=1e-300)
        assert g[k] == pytest.approx((-1) ** k * binom(alpha, k), rel=1e-12)


@pytest.mark.parametrize("alpha", [1.2, 1.5, 1.8])
def test_weights_match_gamma_closed_form_large_k(alpha):
    # g_k = Gamma(k - alpha) / (Gamma(-alpha) Gamma(k + 1)), checked far out (k = 4096)
    g = O.grunwald_weights(alpha, 4096)
    for k in (2, 10, 100, 1000, 4096):
        ref = math.exp(math.lgamma(k - alpha) - math.lgamma(k + 1)) / gamma(-alpha)
        assert g[k] == pytest.approx(ref, rel=1e-11)


@pytest.mark.parametrize("alpha", [1.05, 1.3, 1.5, 1.7, 1.95])
def test_proposition_2_1(alpha):
    g = O.grunwald_weights(alpha, 20000)
    assert g[0] == 1.0
    assert g[1] == pytest.approx(-alpha, rel=1e-15)
    assert np.all(g[2:] > 0)
    assert np.all(np.diff(g[2:]) < 0)  # g_2 > g_3 > ... > 0
    partial = np.cumsum(g)
    assert np.all(partial[1:] < 0)  # sum_{k=0}^n g_k < 0 for n >= 1
    # sum_{k=0}^inf g_k = 0: the partial sums are g_n^(alpha-1) ~ n^-alpha / Gamma(1-alpha) -> 0
    assert abs(partial[-1]) < 5.0 * 20000 ** (-alpha)


@pytest.mark.parametrize("alpha", [1.2, 1.5, 1.9])
def test_partial_sum_identity(alpha):
    # sum_{k=0}^n g_k^(alpha) = g_n^(alpha-1) (Vandermonde convolution with (1-z)^-1)
    g = O.grunwald_weights(alpha, 300)
    g1 = O.grunwald_weights(alpha - 1.0, 300)
    np.testing.assert_allclose(np.cumsum(g), g1, rtol=1e-11, atol=1e-16)


@pytest.mark.parametrize("alpha", [1.2, 1.5, 1.8])
def test_absolute_sum_is_two_alpha(alpha):
    # Sec. 3.2 (Wiener class proof): sum_k |g_k| = -2 g_1 + sum_k g_k = 2 alpha
    g = O.grunwald_weights(alpha, 200000)
    tail = abs(np.cumsum(g)[-1])
    assert np.sum(np.abs(g)) == pytest.approx(2 * alpha, abs=2 * tail + 1e-9)


def _g_matrix_as_displayed(alpha, N):
    # eq. (1.5): first row g1 g0 0 ...; row i: g_{i+1} ... g_1 g_0 (lower Hessenberg Toeplitz)
    g = O.grunwald_weights(alpha, N + 1)
    G = np.zeros((N, N))
    for i in range(N):
        for j in range(N):
            if j <= i + 1:
                G[i, j] = g[i - j + 1]
    return G


@pytest.mark.parametrize("alpha,m", [(1.5, 7), (1.2, 13), (1.8, 31)])
def test_j_entries_match_matrix_form(alpha, m):
    # eq. (1.10t) entries vs eq. (1.4) J = dx^-alpha (D+ G + D- G^T) with G of eq. (1.5)
    rng = np.random.default_rng(5)
    dp, dm = rng.uniform(0, 2, m), rng.uniform(0, 2, m)
    dx = 1.0 / (m + 1)
    G = _g_matrix_as_displayed(alpha, m)
    ref = (np.diag(dp) @ G + np.diag(dm) @ G.T) / dx ** alpha
    np.testing.assert_allclose(O.j_matrix(alpha, dx, dp, dm), ref, rtol=1e-14, atol=0)
    np.testing.assert_allclose(O.j_matrix_from_g(alpha, dx, dp, dm), ref, rtol=1e-14, atol=0)


@pytest.mark.parametrize("alpha", [1.1, 1.5, 1.9])
def test_proposition_2_2_gershgorin(alpha):
    m = 40
    x = np.arange(1, m + 1) / (m + 1)
    dp, dm = 1.0 + x, 2.0 - x
    J = O.j_matrix(alpha, 1.0 / (m + 1), dp, dm)
    off = J - np.diag(np.diag(J))
    # The proof of Proposition 2.2 prints "p_ij <= 0 for i != j"; with g_0 = 1 and g_k > 0
    # (k >= 2) the off-diagonal entries are in fact >= 0.  Only |p_ij| enters the radii.
    assert np.all(off >= 0)
    gam = np.diag(J)
    radius = np.sum(np.abs(off), axis=1)
    assert np.all(gam < 0)
    assert np.all(radius < -gam)  # strict row diagonal dominance
    lam = np.linalg.eigvals(J)
    inside = np.abs(lam[:, None] - gam[None, :]) < -gam[None, :]
    assert np.all(inside.any(axis=1))
    assert np.all(lam.real < 0)  # Remark 2.1 (i)
    assert np.all(np.abs(lam) <= 2 * np.max(np.abs(gam)) * (1 + 1e-12))  # Remark 2.1 (ii)


def _rl_poly(coeffs, y, alpha):
    # Riemann-Liouville derivative of sum_p c_p y^p with lower terminal 0
    return sum(c * gamma(p + 1) / gamma(p + 1 - alpha) * y ** (p - alpha) for p, c in coeffs.items() if c)


@pytest.mark.parametrize("alpha", [1.3, 1.7])
def test_j_approximates_two_sided_fractional_derivative(alpha):
    """J u(x_i) -> d+ D^a_+ u + d- D^a_- u at first order (Sec. 2.1, shifted Grunwald).

    u = x^3 (1-x)^2 is not symmetric and d+ != d-, so a transposed G or swapped
    coefficients would converge to a different function and fail."""
    left = {3: 1.0, 4: -2.0, 5: 1.0}  # x^3 - 2x^4 + x^5
    right = {2: 1.0, 3: -3.0, 4: 3.0, 5: -1.0}  # same in y = 1-x: y^2 (1-y)^3
    errs = []
    for m in (127, 255, 511, 1023):
        dx = 1.0 / (m + 1)
        x = dx * np.arange(1, m + 1)
        dp, dm = 1.0 + x, 2.0 - x
        J = O.j_matrix_from_g(alpha, dx, dp, dm)
        u = x ** 3 * (1 - x) ** 2
        exact = dp * _rl_poly(left, x, alpha) + dm * _rl_poly(right, 1 - x, alpha)
        probe = [(m + 1) // 4 - 1, (m + 1) // 2 - 1, 3 * (m + 1) // 4 - 1]  # x = 1/4, 1/2, 3/4
        errs.append(np.max(np.abs((J @ u - exact)[probe])))
    ratios = [errs[i] / errs[i + 1] for i in range(len(errs) - 1)]
    assert errs[-1] < 0.05
    for r in ratios:
        assert 1.6 < r < 2.6, (errs, ratios)
