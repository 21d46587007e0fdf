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
