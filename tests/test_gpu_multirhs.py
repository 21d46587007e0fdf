"""Many right-hand sides of one operator (fde_batch_share_operator): the Strang blocks
are factored once and every right-hand side's block solves read the same factors.
Each solution is checked against the oracle's direct solve of its own system
(||x - x_oracle|| / ||x_oracle|| <= 1e-8)."""
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


def test_shared_factors_two_groups_of_right_hand_sides():
    """Ten right-hand sides: the block solves take them in CTA groups of eight, so this
    runs a full and a short group; each solution against the oracle's direct solve."""
    from paper_1305_6653_gb300 import FDEBatch
    probs = fi.config_many_rhs(count=10, m=130, s=16)
    with FDEBatch(probs) as b:
        b.share_operator().assemble().factor("tf32")
        xs, stats = b.solve(tol=1e-11, restart=20, maxit=400)
        xs = [x.cpu().numpy() for x in xs]
    for pr, x, st in zip(probs, xs, stats):
        ref = O.direct_solve(pr)
        assert st["status"] == 0, st
        assert np.abs(x - ref).max() <= 1e-8 * np.abs(ref).max(), pr.name


def test_shared_factors_tensor_core_panels():
    """Four right-hand sides of the benchmark operator (alpha = 1.8, d+ = 1+x, d- = 2-x,
    GBDF5) at m = 1023, s = 64: eight 128-column panels of the tensor-core LU (the
    look-ahead path with interior row-pair updates), 33 shared Strang blocks.  Each
    solution against the oracle's FP64 Strang FGMRES of its own system."""
    from paper_1305_6653_gb300 import FDEBatch
    probs = fi.config_many_rhs(count=4, m=1023, s=64)
    with FDEBatch(probs) as b:
        b.share_operator().assemble().factor("tf32")
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
