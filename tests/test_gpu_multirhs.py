"""Many right-hand sides of one operator (fde_batch_share_operator): the Strang blocks
are factored once and every right-hand side's block solves read the same factors,
either on CUDA cores (groups of 8) or as tcgen05 products (groups of 16,
fde_batch_block_solver).  Each solution is checked against the oracle's solve of its
own system (||x - x_oracle|| / ||x_oracle|| <= 1e-8)."""
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


@pytest.mark.parametrize("precision", ["fp32", "tf32"])
def test_shared_factors_solve_every_right_hand_side(precision):
    from paper_1305_6653_gb300 import FDEBatch
    probs = fi.config_many_rhs(count=5, m=100, s=16)
    with FDEBatch(probs) as b:
        b.share_operator().assemble().factor(precision)
        xs, stats = b.solve(tol=1e-11, restart=20, maxit=400)
        xs = [x.cpu().numpy() for x in xs]
    for pr, x, st in zip(probs, xs, stats):
        ref = O.direct_solve(pr)
        assert st["status"] == 0, st
        assert np.linalg.norm(x - ref) <= 1e-8 * np.linalg.norm(ref)
    # the right-hand sides differ, so do the solutions
    assert np.linalg.norm(xs[0] - xs[4]) > 1e-3 * np.linalg.norm(xs[0])


@pytest.mark.parametrize("solver,count,m", [("cuda_cores", 10, 130), ("tensor_cores", 10, 250),
                                            ("tensor_cores", 21, 250)])
def test_shared_factors_groups_of_right_hand_sides(solver, count, m):
    """The block solves take the right-hand sides in CTA groups (8 on CUDA cores, 16 on
    tensor cores), so these run full and short groups (m = 250: m_p = 256, two 128-row
    strips of the tensor-core solves); each solution against the oracle's direct solve."""
    from paper_1305_6653_gb300 import FDEBatch
    probs = fi.config_many_rhs(count=count, m=m, s=16)
    with FDEBatch(probs) as b:
        b.share_operator().block_solver(solver).assemble().factor("tf32")
        xs, stats = b.solve(tol=1e-11, restart=20, maxit=400)
        xs = [x.cpu().numpy() for x in xs]
    for pr, x, st in zip(probs, xs, stats):
        ref = O.direct_solve(pr)
        assert st["status"] == 0, st
        assert np.abs(x - ref).max() <= 1e-8 * np.abs(ref).max(), pr.name


@pytest.mark.parametrize("solver", ["cuda_cores", "tensor_cores"])
def test_shared_factors_tensor_core_panels(solver):
    """Four right-hand sides of the benchmark operator (alpha = 1.8, d+ = 1+x, d- = 2-x,
    GBDF5) at m = 1023, s = 64: eight 128-column panels of the tensor-core LU (the
    look-ahead path with interior row-pair updates), 33 shared Strang blocks, eight
    128-row strips of the tensor-core block solves.  Each solution against the oracle's
    FP64 Strang FGMRES of its own system."""
    from paper_1305_6653_gb300 import FDEBatch
    probs = fi.config_many_rhs(count=4, m=1023, s=64)
    with FDEBatch(probs) as b:
        b.share_operator().block_solver(solver).assemble().factor("tf32")
        xs, stats = b.solve(tol=1e-11, restart=20, maxit=400)
        xs = [x.cpu().numpy() for x in xs]
    # the oracle's FGMRES with one factorisation (the operator is shared), to a true residual
    # of 1e-11: its FP64 floor at this size is 1.5e-12 (a tighter tolerance never converges)
    J = O.j_of(probs[0])
    AB = O.bvm_matrices(probs[0].family, probs[0].mu, probs[0].s)
    P = O.StrangPreconditioner(probs[0], J=J)
    for pr, x, st in zip(probs, xs, stats):
        b = O.reduced_rhs(pr, J=J)
        ref, _, ok, _ = O.gmres(lambda z: O.matvec(pr, z, J=J, AB=AB), b, precond=P.apply, side="right",
                                restart=20, tol=1e-11, maxit=200, reference="b")
        assert ok and st["status"] == 0, st
        assert np.linalg.norm(x - ref) <= 1e-8 * np.linalg.norm(ref), (pr.name, st)
        assert np.abs(x - ref).max() <= 1e-8 * np.abs(ref).max(), pr.name


def test_shared_operator_is_checked():
    from paper_1305_6653_gb300 import FDEBatch, FdeError
    a = fi.manufactured(63, 16, 1.5, "GBDF3")
    c = fi.manufactured(63, 16, 1.6, "GBDF3")  # another alpha: another operator
    with FDEBatch([a, c]) as b:
        with pytest.raises(FdeError):
            b.share_operator()
    d = fi.manufactured(63, 16, 1.5, "GBDF3", dplus_fn=lambda x: 1.0 + x)  # other coefficients
    with FDEBatch([a, d]) as b:
        with pytest.raises(FdeError):
            b.share_operator()


def test_block_solvers_agree_at_the_benchmark_size():
    """Sixteen right-hand sides of the benchmark operator at full size (m = 2047, s = 256:
    129 Strang blocks of m_p = 2048, sixteen 128-row strips, one group of 16 on the tensor
    cores).  Both block solvers run FGMRES to a true residual of 1e-10, which at this
    operator puts a solution within 1e-8 of the oracle's (the full-size parity test), so
    the two agree to 2e-8 of the solution's norm; the first tensor-core solution's true
    residual is checked with the oracle's own matvec."""
    from paper_1305_6653_gb300 import FDEBatch
    probs = fi.config_many_rhs(count=16, m=2047, s=256)
    out = {}
    for solver in ("cuda_cores", "tensor_cores"):
        with FDEBatch(probs, device_inputs=True) as b:
            b.share_operator().block_solver(solver).assemble().factor("tf32")
            xs, stats = b.solve(tol=1e-10, restart=30, maxit=300)
            out[solver] = ([x.cpu().numpy() for x in xs], [st["iterations"] for st in stats],
                           [st["status"] for st in stats])
    (xc, ic, sc), (xt, it, stt) = out["cuda_cores"], out["tensor_cores"]
    assert all(v == 0 for v in sc + stt), (sc, stt)
    for a, c in zip(xc, xt):
        assert np.linalg.norm(a - c) <= 2e-8 * np.linalg.norm(a), (ic, it)
    print("iterations: cuda cores", ic, "tensor cores", it)
    J = O.j_of(probs[0])
    AB = O.bvm_matrices(probs[0].family, probs[0].mu, probs[0].s)
    bb = O.reduced_rhs(probs[0], J=J)
    assert np.linalg.norm(bb - O.matvec(probs[0], xt[0], J=J, AB=AB)) <= 2e-10 * np.linalg.norm(bb)


def test_tensor_core_block_solves_are_checked():
    """Tensor-core block solves need TF32 factors: asking for them with FP32 factors is an error."""
    from paper_1305_6653_gb300 import FDEBatch, FdeError
    probs = fi.config_many_rhs(count=2, m=130, s=16)
    with FDEBatch(probs) as b:
        b.share_operator().block_solver("tensor_cores").assemble()
        with pytest.raises(FdeError):
            b.factor("fp32")


def test_refactoring_switches_the_block_solves():
    """Factoring the shared operator again with another precision changes the block-solve
    kernel (TF32: tensor-core solves with the saved diagonal inverses; FP32: CUDA-core
    groups), so the captured restart cycles must not outlive the factorisation.  m = 250
    (m_p = 256); every solve of the sequence TF32, FP32, TF32 against the oracle's direct
    solve."""
    from paper_1305_6653_gb300 import FDEBatch
    probs = fi.config_many_rhs(count=3, m=250, s=16)
    refs = [O.direct_solve(pr) for pr in probs]
    with FDEBatch(probs) as b:
        b.share_operator().assemble()
        for precision in ("tf32", "fp32", "tf32"):
            b.factor(precision)
            xs, stats = b.solve(tol=1e-11, restart=20, maxit=400)
            for pr, ref, x, st in zip(probs, refs, xs, stats):
                x = x.cpu().numpy()
                assert st["status"] == 0, (precision, st)
                assert np.abs(x - ref).max() <= 1e-8 * np.abs(ref).max(), (precision, pr.name)


def test_refactoring_one_problem_switches_the_factor_layout():
    """The same for one problem: the preconditioner after TF32, FP32 and TF32 factors
    (m = 500, m_p = 512).  The two TF32 applications are bit-identical, and each
    application satisfies S z = r to its precision's bound (oracle Kronecker S)."""
    from paper_1305_6653_gb300 import FDEProblem
    prob = fi.manufactured(500, 16, 1.8, "GBDF5", dplus_fn=lambda x: 1 + x, dminus_fn=lambda x: 2 - x)
    J = O.j_of(prob)
    r = np.random.default_rng(5).standard_normal(prob.n)
    out = []
    with FDEProblem.from_inputs(prob, device_inputs=True) as p:
        p.assemble()
        for precision in ("tf32", "fp32", "tf32"):
            p.factor(precision)
            out.append(p.precond_apply(torch.as_tensor(r, device="cuda")).cpu().numpy())
    assert np.array_equal(out[0], out[2])
    for z, bound in zip(out, (5e-2, 1e-3, 5e-2)):
        srel = np.linalg.norm(O.strang_matvec(prob, z, J=J) - r) / np.linalg.norm(r)
        assert srel <= bound, srel
    assert not np.array_equal(out[0], out[1])


def test_refactoring_switches_the_factor_storage():
    """The same precision with another storage of the block solves' factor copy (FP32,
    bfloat16, FP32 again; m = 500, m_p = 512): each storage is solved twice, so the second
    solve replays the iteration graphs the first captured, and a graph that still held
    the previous layout's kernel would read the copy wrongly.  The FP32 solutions agree
    bit for bit, the bfloat16 ones with each other, and all with the oracle to 1e-8."""
    from paper_1305_6653_gb300 import FDEProblem
    prob = fi.manufactured(500, 16, 1.8, "GBDF5", dplus_fn=lambda x: 1 + x, dminus_fn=lambda x: 2 - x)
    ref, _, ok, _ = O.solve_strang_gmres(prob, side="right", tol=1e-12)
    assert ok
    xs = {}
    with FDEProblem.from_inputs(prob, device_inputs=True) as p:
        p.assemble()
        for i, storage in enumerate(("fp32", "bf16", "fp32")):
            p.factor("tf32", storage=storage)
            for rep in range(2):
                x, st = p.solve(tol=1e-11, restart=20, maxit=400)
                assert st["status"] == 0, (storage, st)
                xs[(i, rep)] = x.cpu().numpy()
    for key, x in xs.items():
        assert np.linalg.norm(x - ref) <= 1e-8 * np.linalg.norm(ref), key
    assert np.array_equal(xs[(0, 0)], xs[(0, 1)]) and np.array_equal(xs[(0, 0)], xs[(2, 1)])
    assert np.array_equal(xs[(1, 0)], xs[(1, 1)]) and not np.array_equal(xs[(0, 0)], xs[(1, 0)])
