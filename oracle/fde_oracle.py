"""Plain FP64 CPU oracle of the Strang-preconditioned BVM/GMRES method.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.  The
CUDA library never calls it, and it shares no code with the CUDA library.

Source: X.-M. Gu, T.-Z. Huang, X.-L. Zhao, H.-B. Li, L. Li, "Strang-type
preconditioners for solving fractional diffusion equations by boundary value
methods" (arXiv:1305.6653).  Equation numbers below are the paper's equation
labels: (1.1) the problem, (1.2) Grunwald weights, (1.4)/(1.5) the matrix J,
(1.10t) the entries of J, (1.7)-(1.9) the BVM formulae, (1.10) the all-at-once
system, (1.11) the Strang preconditioner S, (1.12) the characteristic
polynomials; Theorem 3.3 is the rank / GMRES-iteration bound; Sec. 4 holds the
experiments.

Everything here is written to be checked against the paper by eye: dense
matrices, explicit loops or vectorised one-line formulas, exact rational BVM
coefficients, an explicit DFT matrix along time, one dense complex LU (LAPACK,
partial pivoting) per frequency, and textbook restarted GMRES (modified
Gram-Schmidt Arnoldi + Givens rotations).

Readings of points the paper leaves open (each is listed in the design notes):

* The unknowns are u_1..u_s; the given u_0 is eliminated from (1.10).  The
  Strang circulants are then s x s and use omega = exp(2 pi i / s).
* The additional initial / final formulas (1.8)/(1.9) are the same family as
  the main formula, written on the first / last mu+1 time points with the
  "current" point moved to the row being approximated; their coefficients solve
  the order conditions in exact rational arithmetic.
* GBDF: beta = e_nu, order mu.  GAM: rho(z) = z^nu - z^(nu-1), order mu+1.
  ETR: the GAM with an odd number of steps (symmetric beta).
* The paper's iteration count ITS (Sec. 4) is the total number of inner GMRES
  iterations across restarts; the stopping test there is the preconditioned
  residual relative to the initial one.

Strang-type BCCB preconditioners (eqs. x1 and xc, Sec. 3.1), readings:

* s(G) is the circulant whose first column the paper displays: g_1 .. g_K on
  the diagonal and the first K-1 subdiagonals (K = floor((N+1)/2)), g_0 on the
  superdiagonal that wraps to the last row; s(G^T) is its transpose (the
  display of its first column is garbled in its last entry).
* The modified preconditioner replaces the zero eigenvalue phi_0 of s(A) by
  Re(phi_{s-1}) (the paper's "phi_s", the last eigenvalue in its indexing).

Parity pins: every function below is checked in ``tests/test_oracle_*.py``
against something other than itself (closed forms, invariants, the paper's
printed tables, brute force); there is no "parity unpinned" function.
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np
import scipy.linalg as sla

__all__ = [
    "grunwald_weights",
    "j_matrix",
    "j_of",
    "j_matrix_from_g",
    "time_varying",
    "j_at",
    "nu_of",
    "lmf_coefficients",
    "bvm_matrices",
    "full_system",
    "reduced_system",
    "reduced_rhs",
    "matvec",
    "direct_solve",
    "strang_symbols",
    "strang_circulant",
    "strang_matrix",
    "strang_matvec",
    "StrangPreconditioner",
    "gmres",
    "solve_strang_gmres",
    "strang_g_column",
    "circulant",
    "strang_j_matrix",
    "bccb_matrix",
    "BCCBPreconditioner",
    "solve_bccb_gmres",
]


# ---------------------------------------------------------------------------
# Sec. 2.1: shifted Grunwald discretisation
# ---------------------------------------------------------------------------

def grunwald_weights(alpha: float, n: int) -> np.ndarray:
    """g_0..g_n of eq. (1.2) by the recurrence g_{k+1} = (1 - (alpha+1)/(k+1)) g_k."""
    g = np.empty(n + 1, dtype=np.float64)
    g[0] = 1.0
    for k in range(n):
        g[k + 1] = (1.0 - (alpha + 1.0) / (k + 1)) * g[k]
    return g


def j_matrix(alpha: float, dx: float, dplus: np.ndarray, dminus: np.ndarray) -> np.ndarray:
    """Dense J (m x m) from its entries p_ij, eq. (1.10t) (Proposition 2.2 proof).

    With r_{+,i} = d_{+,i}/dx^alpha, r_{-,i} = d_{-,i}/dx^alpha (1-based i, j):
      j == i   : (r_+ + r_-) g_1
      j == i-1 : r_+ g_2 + r_- g_0
      j == i+1 : r_+ g_0 + r_- g_2
      j <  i-1 : r_+ g_{i-j+1}
      j >  i+1 : r_- g_{j-i+1}
    """
    m = len(dplus)
    g = grunwald_weights(alpha, m + 1)
    rp = np.asarray(dplus, dtype=np.float64) / dx ** alpha
    rm = np.asarray(dminus, dtype=np.float64) / dx ** alpha
    P = np.zeros((m, m), dtype=np.float64)
    for i in range(m):
        for j in range(m):
            if j == i:
                P[i, j] = (rp[i] + rm[i]) * g[1]
            elif j == i - 1:
                P[i, j] = rp[i] * g[2] + rm[i] * g[0]
            elif j == i + 1:
                P[i, j] = rp[i] * g[0] + rm[i] * g[2]
            elif j < i - 1:
                P[i, j] = rp[i] * g[i - j + 1]
            else:
                P[i, j] = rm[i] * g[j - i + 1]
    return P


def j_matrix_from_g(alpha: float, dx: float, dplus: np.ndarray, dminus: np.ndarray) -> np.ndarray:
    """Same matrix as j_matrix, built as dx^-alpha (D+ G + D- G^T) with G of eq. (1.5).

    Used for large m where the double loop of j_matrix is too slow in Python;
    the tests check that both constructions agree.
    """
    m = len(dplus)
    g = grunwald_weights(alpha, m + 1)
    i = np.arange(m)[:, None]
    j = np.arange(m)[None, :]
    k = i - j + 1  # G[i][j] = g_{i-j+1} for j <= i+1, zero above the first superdiagonal
    G = np.where(k >= 0, g[np.clip(k, 0, m)], 0.0)
    return (np.asarray(dplus)[:, None] * G + np.asarray(dminus)[:, None] * G.T) / dx ** alpha


def j_of(prob) -> np.ndarray:
    """J of eq. (1.4)/(1.5) with the problem's d+, d- (for time-dependent coefficients:
    their means over the unknown time levels, the J of the Strang preconditioner)."""
    if prob.m <= 160:
        return j_matrix(prob.alpha, prob.dx, prob.dplus, prob.dminus)
    return j_matrix_from_g(prob.alpha, prob.dx, prob.dplus, prob.dminus)


def time_varying(prob) -> bool:
    return getattr(prob, "dplus_t", None) is not None


def j_at(prob, n: int) -> np.ndarray:
    """J_n = dx^-alpha (D+(t_n) G + D-(t_n) G^T): eq. (1.4) at time level n, for
    coefficients d+-(x, t) (eq. (1.1)); the time-independent J otherwise."""
    if not time_varying(prob):
        return j_of(prob)
    dp, dm = prob.dplus_t[n], prob.dminus_t[n]
    if prob.m <= 160:
        return j_matrix(prob.alpha, prob.dx, dp, dm)
    return j_matrix_from_g(prob.alpha, prob.dx, dp, dm)


# ---------------------------------------------------------------------------
# Sec. 2.2: boundary value methods
# ---------------------------------------------------------------------------

def nu_of(family: str, mu: int) -> int:
    """Number nu of initial conditions of the main formula (1.7) for each family."""
    if family == "GBDF":
        return (mu + 1) // 2 if mu % 2 == 1 else mu // 2 + 1
    if family == "GAM":
        return (mu + 1) // 2 if mu % 2 == 1 else mu // 2
    if family == "ETR":
        if mu % 2 != 1:
            raise ValueError("ETR needs an odd number of steps")
        return (mu + 1) // 2
    raise ValueError(f"unknown BVM family {family!r}")


def _solve_rational(a: list[list[Fraction]], b: list[Fraction]) -> list[Fraction]:
    """Gaussian elimination in exact rational arithmetic."""
    n = len(b)
    M = [row[:] + [b[i]] for i, row in enumerate(a)]
    for c in range(n):
        p = next(r for r in range(c, n) if M[r][c] != 0)
        M[c], M[p] = M[p], M[c]
        for r in range(n):
            if r != c and M[r][c] != 0:
                fac = M[r][c] / M[c][c]
                M[r] = [M[r][k] - fac * M[c][k] for k in range(n + 1)]
    return [M[i][n] / M[i][i] for i in range(n)]


def lmf_coefficients(family: str, mu: int, ell: int) -> tuple[list[Fraction], list[Fraction]]:
    """Coefficients (alpha_0..alpha_mu, beta_0..beta_mu) of a mu-step formula on the
    points 0..mu that approximates u' at the point ``ell`` (exact rationals).

    Order conditions of a linear multistep formula: sum_i alpha_i i^q = q sum_i beta_i i^(q-1).
    * GBDF: beta = e_ell, conditions q = 0..mu (order mu).
    * GAM / ETR: alpha = e_ell - e_(ell-1), conditions q = 1..mu+1 (order mu+1).
    """
    F = Fraction
    pts = [F(i) for i in range(mu + 1)]
    if family == "GBDF":
        beta = [F(0)] * (mu + 1)
        beta[ell] = F(1)
        rows = [[p ** q for p in pts] for q in range(mu + 1)]
        rhs = [F(q) * F(ell) ** (q - 1) if q > 0 else F(0) for q in range(mu + 1)]
        alpha = _solve_rational(rows, rhs)
        return alpha, beta
    if family in ("GAM", "ETR"):
        alpha = [F(0)] * (mu + 1)
        alpha[ell] = F(1)
        alpha[ell - 1] = F(-1)
        rows = [[F(q) * p ** (q - 1) for p in pts] for q in range(1, mu + 2)]
        rhs = [sum(alpha[i] * pts[i] ** q for i in range(mu + 1)) for q in range(1, mu + 2)]
        beta = _solve_rational(rows, rhs)
        return alpha, beta
    raise ValueError(f"unknown BVM family {family!r}")


def bvm_matrices(family: str, mu: int, s: int, exact: bool = False):
    """A and B of eq. (1.10), size (s+1) x (s+1).

    Row 0 is the initial condition (A: e_0, B: 0).  Row t = 1..s holds the formula
    approximating the ODE at t_t: the main formula (1.7) with its mu+1 points
    t-nu..t-nu+mu for nu <= t <= s-mu+nu, the additional initial formulas (1.8)
    on the points 0..mu for t < nu, and the additional final formulas (1.9) on the
    points s-mu..s for t > s-mu+nu.
    """
    nu = nu_of(family, mu)
    if s < mu:
        raise ValueError("need s >= mu")
    Z = Fraction(0)
    A = [[Z] * (s + 1) for _ in range(s + 1)]
    B = [[Z] * (s + 1) for _ in range(s + 1)]
    A[0][0] = Fraction(1)
    for t in range(1, s + 1):
        if t < nu:  # (1.8)
            start = 0
        elif t <= s - mu + nu:  # (1.7)
            start = t - nu
        else:  # (1.9)
            start = s - mu
        a, b = lmf_coefficients(family, mu, t - start)
        for i in range(mu + 1):
            A[t][start + i] = a[i]
            B[t][start + i] = b[i]
    if exact:
        return A, B
    return (np.array([[float(v) for v in row] for row in A]),
            np.array([[float(v) for v in row] for row in B]))


# ---------------------------------------------------------------------------
# The all-at-once system (1.10)
# ---------------------------------------------------------------------------

def full_system(prob):
    """(A (x) I - h B (x) J) u = e_1 (x) u_0 + h (B (x) I) f, eq. (1.10); size (s+1) m.

    With time-dependent coefficients the BVM is applied to u' = J(t) u + f(t): the
    term B (x) J becomes (B (x) I) blkdiag(J_0, .., J_s)."""
    m, s, h = prob.m, prob.s, prob.h
    A, B = bvm_matrices(prob.family, prob.mu, s)
    I = np.eye(m)
    if time_varying(prob):
        JB = np.zeros(((s + 1) * m, (s + 1) * m))
        for n in range(s + 1):
            JB[n * m:(n + 1) * m, n * m:(n + 1) * m] = j_at(prob, n)
        M = np.kron(A, I) - h * np.kron(B, I) @ JB
    else:
        J = j_of(prob)
        M = np.kron(A, I) - h * np.kron(B, J)
    e1 = np.zeros(s + 1)
    e1[0] = 1.0
    rhs = np.kron(e1, prob.u0) + h * np.kron(B, I) @ prob.f.reshape(-1)
    return M, rhs


def reduced_system(prob):
    """Eliminate the known block u_0 from (1.10): unknowns u_1..u_s (size s m).

    M_red = M[m:, m:], b_red = rhs[m:] - M[m:, :m] u_0.
    """
    m = prob.m
    M, rhs = full_system(prob)
    return M[m:, m:].copy(), rhs[m:] - M[m:, :m] @ prob.u0


def reduced_rhs(prob, J=None) -> np.ndarray:
    """b_red without forming M: b_t = h sum_j B[t,j] f_j - A[t,0] u_0 + h B[t,0] J u_0."""
    h = prob.h
    A, B = bvm_matrices(prob.family, prob.mu, prob.s)
    if time_varying(prob):
        J0 = j_at(prob, 0)
    else:
        J0 = j_of(prob) if J is None else J
    b = h * (B[1:, :] @ prob.f) - np.outer(A[1:, 0], prob.u0) + h * np.outer(B[1:, 0], J0 @ prob.u0)
    return b.reshape(-1)


def matvec(prob, z: np.ndarray, J=None, AB=None) -> np.ndarray:
    """M_red z = (A_1 (x) I - h B_1 (x) J) z with z ordered time-major (u_1, ..., u_s)."""
    if J is None:
        J = j_of(prob)
    if AB is None:
        AB = bvm_matrices(prob.family, prob.mu, prob.s)
    A, B = AB
    Z = z.reshape(prob.s, prob.m)
    if time_varying(prob):  # (A_1 (x) I) z - h (B_1 (x) I) [J_1 z_1; ..; J_s z_s]
        JZ = np.stack([j_at(prob, n + 1) @ Z[n] for n in range(prob.s)])
        return (A[1:, 1:] @ Z - prob.h * (B[1:, 1:] @ JZ)).reshape(-1)
    Y = A[1:, 1:] @ Z - prob.h * (B[1:, 1:] @ Z) @ J.T
    return Y.reshape(-1)


def direct_solve(prob) -> np.ndarray:
    """Exact discrete solution of the reduced system by dense LU (partial pivoting)."""
    M, b = reduced_system(prob)
    return np.linalg.solve(M, b)


# ---------------------------------------------------------------------------
# Sec. 3.1: Strang block-circulant preconditioner (1.11)
# ---------------------------------------------------------------------------

def strang_symbols(family: str, mu: int, s: int):
    """Eigenvalues phi_k of s(A) and psi_k of s(B), k = 0..s-1 (Sec. 3.1).

    phi_k = sum_{r=-nu}^{mu-nu} alpha_{r+nu} omega^{r k}, omega = exp(2 pi i / s),
    psi_k likewise with beta.  They diagonalise the circulants in the DFT
    convention Rhat_k = sum_n R_n exp(-2 pi i k n / s).
    """
    nu = nu_of(family, mu)
    a, b = lmf_coefficients(family, mu, nu)
    k = np.arange(s)
    phi = np.zeros(s, dtype=np.complex128)
    psi = np.zeros(s, dtype=np.complex128)
    for r in range(-nu, mu - nu + 1):
        w = np.exp(2j * np.pi * r * k / s)
        phi += float(a[r + nu]) * w
        psi += float(b[r + nu]) * w
    return phi, psi


def strang_circulant(coeffs, nu: int, s: int) -> np.ndarray:
    """s x s Strang circulant of eq. (1.11): C[n, (n+r) mod s] = c_{r+nu}, r = -nu..mu-nu."""
    mu = len(coeffs) - 1
    C = np.zeros((s, s))
    for n in range(s):
        for r in range(-nu, mu - nu + 1):
            C[n, (n + r) % s] += float(coeffs[r + nu])
    return C


def strang_matrix(prob) -> np.ndarray:
    """Dense S = s(A) (x) I - h s(B) (x) J, eq. (1.11), for small sizes."""
    nu = nu_of(prob.family, prob.mu)
    a, b = lmf_coefficients(prob.family, prob.mu, nu)
    sA = strang_circulant(a, nu, prob.s)
    sB = strang_circulant(b, nu, prob.s)
    J = j_of(prob)
    return np.kron(sA, np.eye(prob.m)) - prob.h * np.kron(sB, J)


def strang_matvec(prob, z: np.ndarray, J=None) -> np.ndarray:
    """S z with S = s(A) (x) I - h s(B) (x) J of eq. (1.11), by its Kronecker form."""
    if J is None:
        J = j_of(prob)
    nu = nu_of(prob.family, prob.mu)
    a, b = lmf_coefficients(prob.family, prob.mu, nu)
    sA = strang_circulant(a, nu, prob.s)
    sB = strang_circulant(b, nu, prob.s)
    Z = z.reshape(prob.s, prob.m)
    return (sA @ Z - prob.h * (sB @ Z) @ J.T).reshape(-1)


class StrangPreconditioner:
    """S^{-1} r by the DFT diagonalisation of Sec. 3.2:

        S^{-1} = (F^* (x) I) (Lambda_A (x) I - h Lambda_B (x) J)^{-1} (F (x) I)

    F is applied as an explicit DFT matrix along time; the s blocks
    phi_k I - h psi_k J are factored once by dense complex LU with partial
    pivoting.  With ``conjugate_symmetry`` only k = 0..s/2 are factored and the
    block for s-k is used as the complex conjugate (J, u real).
    """

    def __init__(self, prob, J=None, conjugate_symmetry: bool = True):
        self.m, self.s, self.h = prob.m, prob.s, prob.h
        self.J = j_of(prob) if J is None else J
        self.phi, self.psi = strang_symbols(prob.family, prob.mu, prob.s)
        s = self.s
        n = np.arange(s)
        self.F = np.exp(-2j * np.pi * np.outer(n, n) / s)
        self.Finv = np.exp(2j * np.pi * np.outer(n, n) / s) / s
        self.sym = conjugate_symmetry
        kmax = s // 2 if conjugate_symmetry else s - 1
        I = np.eye(self.m)
        self.lu = {}
        for k in range(kmax + 1):
            Bk = self.phi[k] * I - self.h * self.psi[k] * self.J
            self.lu[k] = sla.lu_factor(Bk, check_finite=False)

    def block(self, k: int) -> np.ndarray:
        return self.phi[k] * np.eye(self.m) - self.h * self.psi[k] * self.J

    def apply(self, r: np.ndarray) -> np.ndarray:
        s, m = self.s, self.m
        R = r.reshape(s, m)
        Rhat = self.F @ R
        Xhat = np.empty_like(Rhat)
        for k in range(s):
            if k in self.lu:
                Xhat[k] = sla.lu_solve(self.lu[k], Rhat[k], check_finite=False)
            else:
                Xhat[k] = np.conj(sla.lu_solve(self.lu[s - k], np.conj(Rhat[k]), check_finite=False))
        return (self.Finv @ Xhat).real.reshape(-1)


# ---------------------------------------------------------------------------
# GMRES(restart) (Saad), as used in Sec. 4
# ---------------------------------------------------------------------------

def gmres(mv, b: np.ndarray, *, precond=None, side: str = "left", restart: int = 20,
          tol: float = 1e-8, maxit: int = 10000, x0: np.ndarray | None = None,
          reference: str = "r0"):
    """Restarted GMRES with modified Gram-Schmidt Arnoldi and Givens rotations.

    side = "none"  : GMRES on M x = b.
    side = "left"  : GMRES on P^{-1} M x = P^{-1} b (the form of Theorem 3.3 and
                     Sec. 4); the residual is the preconditioned one.
    side = "right" : flexible GMRES, x = x0 + Z y with z_j = P^{-1} v_j; the
                     residual is the true one, b - M x.
    reference = "r0": stop when ||r_q|| / ||r_0|| < tol (Sec. 4);
    reference = "b" : stop when ||r_q|| / ||b|| <= tol (||P^{-1} b|| for "left").

    Returns (x, its, converged, history) where its is the total number of inner
    iterations and history the residual ratio after each inner iteration.
    """
    n = b.size
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64)

    def residual(xv):
        r = b - mv(xv)
        return precond(r) if side == "left" else r

    r = residual(x)
    beta = np.linalg.norm(r)
    if reference == "r0":
        ref = beta
    else:
        ref = np.linalg.norm(precond(b) if side == "left" else b)
    hist = []
    if ref == 0.0 or beta / ref < tol:
        return x, 0, True, hist
    its = 0
    while its < maxit:
        V = np.zeros((restart + 1, n))
        Zs = np.zeros((restart, n)) if side == "right" else None
        H = np.zeros((restart + 1, restart))
        cs = np.zeros(restart)
        sn = np.zeros(restart)
        g = np.zeros(restart + 1)
        g[0] = beta
        V[0] = r / beta
        j_last = -1
        done = False
        for j in range(restart):
            if side == "right":
                Zs[j] = precond(V[j])
                w = mv(Zs[j])
            elif side == "left":
                w = precond(mv(V[j]))
            else:
                w = mv(V[j])
            for i in range(j + 1):
                H[i, j] = V[i] @ w
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            breakdown = H[j + 1, j] == 0.0
            if not breakdown:
                V[j + 1] = w / H[j + 1, j]
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            rr = np.hypot(H[j, j], H[j + 1, j])
            cs[j] = H[j, j] / rr
            sn[j] = H[j + 1, j] / rr
            H[j, j] = rr
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            its += 1
            j_last = j
            hist.append(abs(g[j + 1]) / ref)
            if abs(g[j + 1]) / ref < tol or breakdown or its >= maxit:
                done = True
                break
        k = j_last + 1
        y = sla.solve_triangular(H[:k, :k], g[:k])
        if side == "right":
            x = x + Zs[:k].T @ y
        else:
            x = x + V[:k].T @ y
        r = residual(x)
        beta = np.linalg.norm(r)
        if beta / ref < tol:
            return x, its, True, hist
        if done and its >= maxit:
            break
    return x, its, False, hist


def solve_strang_gmres(prob, *, side: str = "right", restart: int = 20, tol: float = 1e-12,
                       maxit: int = 2000, reference: str = "b", x0=None):
    """Strang-preconditioned GMRES solve of the reduced system (FP64 throughout)."""
    J = j_of(prob)
    AB = bvm_matrices(prob.family, prob.mu, prob.s)
    P = StrangPreconditioner(prob, J=J)
    b = reduced_rhs(prob, J=J)
    x, its, ok, hist = gmres(lambda z: matvec(prob, z, J=J, AB=AB), b, precond=P.apply,
                             side=side, restart=restart, tol=tol, maxit=maxit,
                             reference=reference, x0=x0)
    return x, its, ok, hist


# ---------------------------------------------------------------------------
# Sec. 3.1, eqs. (x1) and (xc): Strang-type BCCB preconditioners
# ---------------------------------------------------------------------------

def strang_g_column(alpha: float, m: int) -> np.ndarray:
    """First column of the m x m Strang circulant s(G_alpha) as the paper displays it:
    [g_1, ..., g_K, 0, ..., 0, g_0] with K = floor((m+1)/2)."""
    g = grunwald_weights(alpha, m + 1)
    c = np.zeros(m)
    K = (m + 1) // 2
    for i in range(K):
        c[i] += g[i + 1]
    c[m - 1] += g[0]
    return c


def circulant(c: np.ndarray) -> np.ndarray:
    """Dense circulant with first column c: C[i, j] = c[(i - j) mod n]."""
    n = len(c)
    C = np.empty((n, n), dtype=np.result_type(c, np.float64))
    for i in range(n):
        for j in range(n):
            C[i, j] = c[(i - j) % n]
    return C


def strang_j_matrix(prob) -> np.ndarray:
    """Dense s(J_N) = dx^-alpha (mean(d+) s(G) + mean(d-) s(G)^T) (Sec. 3.1, below eq. x1)."""
    m = prob.m
    dp = float(np.mean(np.broadcast_to(np.asarray(prob.dplus, dtype=np.float64), (m,))))
    dm = float(np.mean(np.broadcast_to(np.asarray(prob.dminus, dtype=np.float64), (m,))))
    sG = circulant(strang_g_column(prob.alpha, m))
    return prob.dx ** (-prob.alpha) * (dp * sG + dm * sG.T)


def _s_of_a_modified(prob) -> np.ndarray:
    """s~(A) (eq. xc): s(A) with its eigenvalue phi_0 = 0 moved to Re(phi_{s-1}).
    As a matrix: s(A) + (phi~_0 - phi_0) / s * ones (the rank-one change of the
    eigenvalue that belongs to the constant eigenvector)."""
    nu = nu_of(prob.family, prob.mu)
    a, _ = lmf_coefficients(prob.family, prob.mu, nu)
    sA = strang_circulant(a, nu, prob.s)
    phi, _ = strang_symbols(prob.family, prob.mu, prob.s)
    return sA + (phi[-1].real - phi[0].real) / prob.s * np.ones((prob.s, prob.s))


def bccb_matrix(prob, modified: bool = False) -> np.ndarray:
    """Dense S^(2) = s(A) (x) I - h s(B) (x) s(J) (eq. x1), or S~^(2) with s~(A) (eq. xc)."""
    nu = nu_of(prob.family, prob.mu)
    a, b = lmf_coefficients(prob.family, prob.mu, nu)
    sA = _s_of_a_modified(prob) if modified else strang_circulant(a, nu, prob.s)
    sB = strang_circulant(b, nu, prob.s)
    return np.kron(sA, np.eye(prob.m)) - prob.h * np.kron(sB, strang_j_matrix(prob))


class BCCBPreconditioner:
    """(S^(2))^{-1} r or (S~^(2))^{-1} r by the two-dimensional DFT diagonalisation
    of Sec. 3.3: F along time and F_N along space, division by the eigenvalues
    phi_j - h psi_j lambda_k(s(J)) (eq. 1.13), inverse transforms.

    lambda_k(s(J)) = sum_i c_i exp(-2 pi i i k / N) for the first column c of
    s(J); numpy.fft uses the same sign, so fft(c) pairs with fft(x) along space.
    """

    def __init__(self, prob, modified: bool = False):
        self.s, self.m, self.h = prob.s, prob.m, prob.h
        phi, psi = strang_symbols(prob.family, prob.mu, prob.s)
        if modified:
            phi = phi.copy()
            phi[0] = phi[-1].real
        m = prob.m
        dp = float(np.mean(np.broadcast_to(np.asarray(prob.dplus, dtype=np.float64), (m,))))
        dm = float(np.mean(np.broadcast_to(np.asarray(prob.dminus, dtype=np.float64), (m,))))
        cG = strang_g_column(prob.alpha, m)
        cGT = np.roll(cG[::-1], 1)  # first column of s(G)^T: c[(-i) mod m]
        self.lam_J = np.fft.fft(prob.dx ** (-prob.alpha) * (dp * cG + dm * cGT))
        self.D = phi[:, None] - prob.h * psi[:, None] * self.lam_J[None, :]

    def apply(self, r: np.ndarray) -> np.ndarray:
        R = r.reshape(self.s, self.m)
        X = np.fft.fft2(R) / self.D
        return np.fft.ifft2(X).real.reshape(-1)


def solve_bccb_gmres(prob, *, modified: bool = False, side: str = "right", restart: int = 20,
                     tol: float = 1e-12, maxit: int = 5000, reference: str = "b", x0=None):
    """GMRES on the reduced system with the BCCB preconditioner (FP64 throughout)."""
    J = j_of(prob)
    AB = bvm_matrices(prob.family, prob.mu, prob.s)
    P = BCCBPreconditioner(prob, modified=modified)
    b = reduced_rhs(prob, J=J)
    return gmres(lambda z: matvec(prob, z, J=J, AB=AB), b, precond=P.apply, side=side, restart=restart,
                 tol=tol, maxit=maxit, reference=reference, x0=x0)
