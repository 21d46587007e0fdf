"""GPU parity of the CUDA path (through the C ABI) against the FP64 CPU oracle.

Tolerances (derived from the arithmetic):
* Grunwald weights: the same factors (1 - (alpha+1)/(k+1)) multiplied in FP64 in a
  different association (warp scan): relative difference <= ~(m+2) eps.
* M z: J is applied through length-L FFTs (L = 2^k >= 2m).  The FFT's error is
  O(eps log2 L) relative to ||lambda||_inf ||z||, and ||lambda||_inf <= sum|t_k|
  = 2 alpha (d+ + d-) dx^-alpha (Sec. 3.2, Wiener class).  With eps = 1.1e-16
  and log2 L <= 13 the bound is below 1e-12 * h * 2 alpha (d+ + d-) dx^-alpha
  ||z||_inf, the scale used in the test.
* S^{-1} r: FP64 LU without pivoting of strictly diagonally dominant blocks
  (growth factor <= 2), backward stable; forward error <= cond(B_k) * eps * c.
  cond(B_k) <= 1e4 on these sizes, so 1e-10 relative.
* Solutions: the accuracy target of the solver, ||x - x_oracle|| / ||x_oracle|| <= 1e-8.
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


def _gpu(prob, precision="fp64", device_inputs=False):
    from paper_1305_6653_gb300 import FDEProblem
    p = FDEProblem.from_inputs(prob, device_inputs=device_inputs)
    p.assemble()
    if precision:
        p.factor(precision)
    return p


def _variable(m, s, scheme, alpha=1.5):
    return fi.manufactured(m, s, alpha, scheme, dplus_fn=lambda x: 1.0 + x, dminus_fn=lambda x: 2.0 - x)


CASES = [
    ("small", lambda: fi.config_small()),
    ("ragged_gbdf5", lambda: _variable(100, 16, "GBDF5", 1.8)),
    ("gam4_ex41", lambda: fi.example_4_1(1.2, 48, 32)),
    ("etr3", lambda: _variable(37, 8, "ETR3", 1.3)),
    ("tiny_m1", lambda: _variable(1, 4, "GBDF1", 1.5)),
    ("m64_exact_tile", lambda: _variable(64, 16, "GAM4", 1.9)),
    ("m255_s64", lambda: _variable(255, 64, "GBDF3", 1.7)),
]


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_grunwald_and_rhs(name, make):
    prob = make()
    with _gpu(prob, precision=None) as p:
        g = p.grunwald()
        # the device forms the same product of the same factors, associated by a warp scan:
        # relative difference bounded by ~(m+2) eps in the worst case, a few eps in practice
        np.testing.assert_allclose(g, O.grunwald_weights(prob.alpha, prob.m + 1), rtol=max(1e-14, 4e-16 * (prob.m + 2)),
                                   atol=0)
        b = p.rhs().cpu().numpy()
    ref = O.reduced_rhs(prob)
    scale = np.abs(ref).max() + prob.h * O.j_of(prob).__abs__().sum(axis=1).max() * np.abs(prob.u0).max()
    np.testing.assert_allclose(b, ref, rtol=0, atol=1e-12 * max(scale, 1e-300))


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_matvec(name, make):
    prob = make()
    rng = np.random.default_rng(11)
    z = rng.standard_normal(prob.n)
    with _gpu(prob, precision=None) as p:
        y = p.matvec(torch.as_tensor(z, device="cuda")).cpu().numpy()
    ref = O.matvec(prob, z)
    jscale = 2 * prob.alpha * (prob.dplus + prob.dminus).max() * prob.dx ** (-prob.alpha)
    scale = prob.h * jscale * np.abs(z).max() + 4 * np.abs(z).max()
    assert np.abs(y - ref).max() <= 1e-12 * scale


# FP32 Toeplitz apply (fde_matvec_fp32).  Only J w runs in FP32 (w = the B-band sum of a
# time row, rounded once to FP32; a length-L/2 complex FFT and its split, the product with
# the FP32 symbol, a length-L inverse FFT; twiddles accurate to FP32).  The 2-norm error
# bound of an FFT with twiddle error mu is log2(n) eta / (1 - log2(n) eta) ||x||, eta =
# mu + gamma_4 (sqrt 2 + mu) ~ 6.7 u (Higham, Accuracy and Stability, Thm. 24.2); two
# transforms, the split and the symbol product give ||C w - fl(C w)||_2 <=
# (2 log2(L) 6.7 + 4) u_32 ||lambda_C||_inf ||w||_2 for the complex circulant C = G + i G^T
# that yields G w and G^T w together, ||lambda_C||_inf <= 2 sum |g_k| = 4 alpha (Wiener
# bound of Sec. 3.2), and J w = dx^-alpha (D+ Re + D- Im) adds the factor max(d+ + d-)
# dx^-alpha; u_32 = 2^-24.  Every entry of row t is held to h times that bound for w_t
# (the A-band part and the output are FP64).
@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_matvec_fp32(name, make):
    prob = make()
    rng = np.random.default_rng(13)
    z = rng.standard_normal(prob.n)
    with _gpu(prob, precision=None) as p:
        zt = torch.as_tensor(z, device="cuda")
        y = p.matvec_fp32(zt).cpu().numpy().reshape(prob.s, prob.m)
        y64 = p.matvec(zt).cpu().numpy().reshape(prob.s, prob.m)
    ref = O.matvec(prob, z).reshape(prob.s, prob.m)
    _, B = O.bvm_matrices(prob.family, prob.mu, prob.s)
    W = B[1:, 1:] @ z.reshape(prob.s, prob.m)  # the input of the Toeplitz apply, row by row
    L = 2
    while L < 2 * prob.m:
        L *= 2
    lam = 4 * prob.alpha * (prob.dplus + prob.dminus).max() * prob.dx ** (-prob.alpha)
    u32 = 2.0 ** -24
    bound = (2 * np.log2(L) * 6.7 + 4) * u32 * prob.h * lam * np.linalg.norm(W, axis=1)
    err = np.abs(y - ref).max(axis=1)
    jscale = 2 * prob.alpha * (prob.dplus + prob.dminus).max() * prob.dx ** (-prob.alpha)
    fp64_floor = 1e-12 * (prob.h * jscale * np.abs(z).max() + 4 * np.abs(z).max())
    assert np.all(err <= bound + fp64_floor), (err / (bound + fp64_floor)).max()
    if prob.m >= 63:  # and it is the FP32 path: far above the FP64 product's error
        assert np.abs(y - ref).max() > 100 * np.abs(y64 - ref).max()


@pytest.mark.parametrize("relax", [0.0, 1e-4])
@pytest.mark.parametrize("name,make", [c for c in CASES if c[0] in ("small", "ragged_gbdf5", "m255_s64")],
                         ids=["small", "ragged_gbdf5", "m255_s64"])
def test_solve_with_fp32_arnoldi_products(name, make, relax):
    """Flexible GMRES with the FP32 Toeplitz apply in the Arnoldi products (all of them, or
    while the residual estimate is above 1e-4): the FP64 true residual at every restart still
    drives the solution to the oracle's within 1e-8."""
    prob = make()
    if prob.n <= 5000:
        ref = O.direct_solve(prob)
    else:
        ref, _, ok, _ = O.solve_strang_gmres(prob, side="right", tol=1e-12)
        assert ok
    with _gpu(prob, "tf32") as p:
        x, st = p.solve(tol=1e-11, restart=20, maxit=400, matvec="fp32", relax=relax)
        xs = x.cpu().numpy()
    assert st["status"] == 0, st
    assert st["matvecs_fp32"] >= 1
    if relax == 0.0:
        assert st["matvecs_fp32"] == st["iterations"]
    assert np.linalg.norm(xs - ref) <= 1e-8 * np.linalg.norm(ref), st


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_precond_apply_fp64(name, make):
    prob = make()
    rng = np.random.default_rng(12)
    r = rng.standard_normal(prob.n)
    with _gpu(prob, "fp64") as p:
        z = p.precond_apply(torch.as_tensor(r, device="cuda")).cpu().numpy()
    ref = O.StrangPreconditioner(prob).apply(r)
    # elementwise, against the largest entry (the bound above is normwise; the FP64
    # differences are ~1e-14 of max|z|)
    assert np.abs(z - ref).max() <= 1e-10 * np.abs(ref).max()


# Reconstruction tolerance of L U against B_k, relative to max|B_k|: FP64 and FP32
# factors carry their unit roundoff times a small growth factor; TF32 (10-bit
# mantissa) and BF16 (7-bit) inputs to the trailing updates carry 2^-11 and 2^-8
# per product, accumulated over the m/NB updates; split TF32 (hi + lo) is FP32-level.
FACTOR_TOL = {"fp64": 1e-12, "fp32": 2e-5, "tf32": 5e-3, "bf16": 5e-2, "tf32x3": 2e-5}


@pytest.mark.parametrize("precision", ["fp64", "fp32", "tf32", "bf16", "tf32x3"])
def test_factor_reconstructs_strang_blocks(precision):
    """Sampled check: L_k U_k equals phi_k I - h psi_k J of the oracle (Sec. 3.2)."""
    prob = _variable(300, 16, "GBDF5", 1.8)  # several 128-row tensor-core tiles plus a ragged tail
    P = O.StrangPreconditioner(prob)
    tol = FACTOR_TOL[precision]
    with _gpu(prob, precision) as p:
        for k in (0, 1, prob.s // 4, prob.s // 2):
            F = p.factor_block(k)
            L = np.tril(F, -1) + np.eye(prob.m)
            U = np.triu(F)
            B = P.block(k)
            assert np.abs(L @ U - B).max() <= tol * np.abs(B).max(), k


@pytest.mark.parametrize("precision", ["fp64", "fp32", "tf32", "bf16", "tf32x3"])
@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_solve_matches_direct_solution(name, make, precision):
    prob = make()
    if prob.n <= 5000:
        ref = O.direct_solve(prob)
    else:
        ref, _, ok, _ = O.solve_strang_gmres(prob, side="right", tol=1e-12)
        assert ok
    with _gpu(prob, precision) as p:
        x, st = p.solve(tol=1e-11, restart=20, maxit=400)
        xs = x.cpu().numpy()
    err = np.linalg.norm(xs - ref) / np.linalg.norm(ref)
    assert st["status"] == 0, st
    assert err <= 1e-8, (err, st)
    # Theorem 3.3: with S, GMRES needs at most 2 m mu + 1 iterations (exact arithmetic)
    assert st["iterations"] <= 2 * prob.m * prob.mu + 1
    # the true residual reported by the library agrees with the oracle's
    M_b = O.reduced_rhs(prob)
    res = np.linalg.norm(M_b - O.matvec(prob, xs)) / np.linalg.norm(M_b)
    assert res <= 1e-10 and abs(res - st["rel_residual"]) <= 1e-11


@pytest.mark.parametrize("precision", ["tf32", "bf16", "tf32x3"])
@pytest.mark.parametrize("name,make", [("m255_s64", lambda: _variable(255, 64, "GBDF3", 1.7)),
                                       ("m500_s16", lambda: _variable(500, 16, "GBDF3", 1.8))],
                         ids=["m255_s64", "m500_s16"])
def test_bf16_factor_storage(name, make, precision):
    """Block solves from the bfloat16 copy of the factors (fde_factor_storage; m_p = 256 and
    512, whole 128-wide panels, where the tensor-core LU writes the copy).  The solution
    against the oracle (1e-8) and the true residual through the oracle's matvec; the
    preconditioner is the exact inverse of the factors perturbed by bfloat16 rounding
    (2^-9 relative per entry), so S z = r holds only to the factors' accuracy, and the
    outer iteration pays at most a few iterations for it."""
    from paper_1305_6653_gb300 import FDEProblem
    prob = make()
    if prob.n <= 5000:
        ref = O.direct_solve(prob)
    else:
        ref, _, ok, _ = O.solve_strang_gmres(prob, side="right", tol=1e-12)
        assert ok
    J = O.j_of(prob)
    r = np.random.default_rng(8).standard_normal(prob.n)
    out = {}
    for storage in ("fp32", "bf16"):
        with FDEProblem.from_inputs(prob, device_inputs=True) as p:
            p.assemble().factor(precision, storage=storage)
            z = p.precond_apply(torch.as_tensor(r, device="cuda")).cpu().numpy()
            x, st = p.solve(tol=1e-11, restart=20, maxit=400)
            out[storage] = (z, x.cpu().numpy(), st)
    zf, _, stf = out["fp32"]
    zb, xb, stb = out["bf16"]
    assert stb["status"] == 0, stb
    assert np.linalg.norm(xb - ref) <= 1e-8 * np.linalg.norm(ref)
    M_b = O.reduced_rhs(prob, J=J)
    assert np.linalg.norm(M_b - O.matvec(prob, xb, J=J)) <= 1e-10 * np.linalg.norm(M_b)
    assert not np.array_equal(zb, zf)
    sf = np.linalg.norm(O.strang_matvec(prob, zf, J=J) - r) / np.linalg.norm(r)
    sb = np.linalg.norm(O.strang_matvec(prob, zb, J=J) - r) / np.linalg.norm(r)
    print(name, precision, "S z = r:", sf, sb, "iterations", stf["iterations"], stb["iterations"])
    assert sb <= 0.2, (sf, sb)
    assert stb["iterations"] <= stf["iterations"] + 3, (stf, stb)


def test_small_config_iterations_are_paper_like():
    prob = fi.config_small()
    with _gpu(prob, "fp64") as p:
        _, st = p.solve(tol=1e-10)
    _, its_oracle, _, _ = O.solve_strang_gmres(prob, side="right", tol=1e-10)
    assert abs(st["iterations"] - its_oracle) <= 1


def test_device_inputs_and_warm_start():
    prob = fi.config_small()
    ref = O.direct_solve(prob)
    with _gpu(prob, "fp64", device_inputs=True) as p:
        x0 = torch.as_tensor(ref, device="cuda")
        x, st = p.solve(tol=1e-10, x0=x0)
        assert st["iterations"] <= 1
        np.testing.assert_allclose(x.cpu().numpy(), ref, rtol=0, atol=1e-8 * np.abs(ref).max())


def test_host_solution_vectors_through_the_abi():
    """desc->device_ptrs = 0: pgmres_solve takes x0 and writes x_out in host memory
    (the library copies them on its stream).  Raw C-ABI call with numpy buffers."""
    import ctypes as C

    from paper_1305_6653_gb300 import FdePgmresOpts, FdeStats, _lib
    prob = fi.config_small()
    ref = O.direct_solve(prob)
    lib = _lib.load()
    with _gpu(prob, "fp64") as p:
        assert not p.device_ptrs
        opts = FdePgmresOpts(1e-11, 20, 400, 1)
        x = np.full(prob.n, np.nan)
        st = FdeStats()
        assert lib.pgmres_solve(p.h, C.byref(opts), None, C.c_void_p(x.ctypes.data), C.byref(st)) == 0
        assert np.linalg.norm(x - ref) <= 1e-8 * np.linalg.norm(ref)
        # a host initial guess, aliased with the output: the exact solution needs no iteration
        x2 = ref.copy()
        assert lib.pgmres_solve(p.h, C.byref(opts), C.c_void_p(x2.ctypes.data), C.c_void_p(x2.ctypes.data),
                                C.byref(st)) == 0
        assert st.iterations <= 1 and st.x0_rejected == 0
        np.testing.assert_allclose(x2, ref, rtol=0, atol=1e-8 * np.abs(ref).max())


def test_host_batch_solutions():
    from paper_1305_6653_gb300 import FDEBatch
    probs = [fi.config_small(), _variable(100, 16, "GBDF5", 1.8)]
    with FDEBatch(probs) as b:
        b.assemble().factor("fp32")
        xs, stats = b.solve(tol=1e-11)
    for prob, x, st in zip(probs, xs, stats):
        assert not x.is_cuda and st["status"] == 0
        ref = O.direct_solve(prob)
        assert np.linalg.norm(x.numpy() - ref) <= 1e-8 * np.linalg.norm(ref)


def test_error_paths():
    from paper_1305_6653_gb300 import FdeError, _lib
    prob = fi.config_small()
    from paper_1305_6653_gb300 import FDEProblem
    with FDEProblem.from_inputs(prob) as p:
        with pytest.raises(FdeError) as e:
            p.solve()
        assert e.value.code == _lib.FDE_ERR_STATE
        p.assemble().factor("fp64")
        _, st = p.solve(tol=1e-14, maxit=1, raise_on_error=False)
        assert st["status"] == _lib.FDE_ERR_NOT_CONVERGED and st["iterations"] == 1
    bad = fi.config_small()
    bad.f = bad.f.copy()
    bad.f[3, 5] = np.nan
    with pytest.raises(FdeError) as e:
        FDEProblem.from_inputs(bad)
    assert e.value.code == _lib.FDE_ERR_ARG


@pytest.mark.parametrize("precision", ["fp64", "tf32"])
def test_repeated_solve_replays_graphs(precision):
    # from its second solve on a problem replays the inner GMRES iteration as captured CUDA
    # graphs: same iterates, same iteration count, same launch count as direct launches
    from paper_1305_6653_gb300 import fde_launch_count
    prob = _variable(255, 64, "GBDF3", 1.7)
    with _gpu(prob, precision) as p:
        counts, xs, its = [], [], []
        for _ in range(3):
            l0 = fde_launch_count()
            x, st = p.solve(tol=1e-11, restart=20, maxit=400)
            torch.cuda.synchronize()
            counts.append(fde_launch_count() - l0)
            xs.append(x.cpu().numpy())
            its.append(st["iterations"])
    assert its[0] == its[1] == its[2]
    np.testing.assert_array_equal(xs[1], xs[0])
    np.testing.assert_array_equal(xs[2], xs[0])
    assert counts[0] == counts[1] == counts[2], counts
