"""Learned warm start (fde_nop_*): the network's kernels against the CPU oracle
(oracle/nop_oracle.py), and what a network trained on method-generated solves
gains over the zero initial guess.

Tolerances: forward and gradients are FP32 kernels (the weight gradient
accumulates with float atomics over the batch) against an FP64 oracle; with
O(10^2..10^3)-term sums of O(1) values the relative error stays below 1e-4.  The
FP16 inference path (FP16 weights / activations, FP32 accumulation) agrees with
the FP32 forward to ~1e-3 relative.  Solutions started from the learned guess are
judged like every other solve: rel.err <= 1e-8 against the oracle.
"""
import numpy as np
import pytest

import fde_inputs as fi
import oracle as O
from oracle import nop_oracle as N

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def _small_net(m=37, s=8, modes=13, width=8, layers=3, K=5, seed=3):
    from paper_1305_6653_gb300 import FDENop
    net = FDENop(m, s, modes=modes, width=width, layers=layers, ksize=K, seed=seed)
    shapes = N.layer_shapes(cin=s + 6, cout=s, width=width, layers=layers, K=K)
    assert N.num_params(shapes) == net.nparam
    return net, shapes


def _sin(m, K):
    i = np.arange(1, m + 1)
    return np.sin(np.pi * np.outer(np.arange(1, K + 1), i) / (m + 1))  # K x m


def test_forward_and_gradients_match_oracle():
    net, shapes = _small_net()
    rng = np.random.default_rng(7)
    theta = (rng.standard_normal(net.nparam) * 0.3).astype(np.float32)
    net.set_params(theta)
    B, m = 3, net.modes
    x = rng.standard_normal((B, net.cin, m)).astype(np.float32)
    t = rng.standard_normal((B, net.s, m)).astype(np.float32)
    xd = torch.as_tensor(x.reshape(-1), device="cuda")
    td = torch.as_tensor(t.reshape(-1), device="cuda")
    y = net.forward(xd, B).cpu().numpy().reshape(B, net.s, m)
    y_ref = N.forward(theta.astype(np.float64), shapes, x.astype(np.float64))
    assert np.abs(y - y_ref).max() <= 1e-4 * max(1.0, np.abs(y_ref).max())
    loss, g = net.loss_grad(xd, td, B, want_grad=True)
    loss_ref, g_ref = N.loss_and_grad(theta.astype(np.float64), shapes, x.astype(np.float64), t.astype(np.float64))
    assert abs(loss - loss_ref) <= 1e-5 * abs(loss_ref)
    assert np.abs(g - g_ref).max() <= 1e-4 * np.abs(g_ref).max()


def test_adam_step_matches_oracle():
    net, shapes = _small_net()
    rng = np.random.default_rng(8)
    theta = (rng.standard_normal(net.nparam) * 0.3).astype(np.float32)
    net.set_params(theta)
    B = 2
    x = torch.as_tensor(rng.standard_normal(B * net.cin * net.modes).astype(np.float32), device="cuda")
    t = torch.as_tensor(rng.standard_normal(B * net.s * net.modes).astype(np.float32), device="cuda")
    _, g = net.loss_grad(x, t, B, want_grad=True)
    net.adam_step(1e-2)
    th_ref, _, _ = N.adam_step(theta.astype(np.float64), g.astype(np.float64), np.zeros(net.nparam),
                               np.zeros(net.nparam), t=1, lr=1e-2)
    np.testing.assert_allclose(net.get_params(), th_ref, rtol=1e-5, atol=1e-6)


def test_features_coefficients_and_fp16_inference():
    from paper_1305_6653_gb300 import FDEProblem
    prob = fi.config_learned_family(seed=11, m=63, s=16)
    K = 12
    net, shapes = _small_net(m=63, s=16, modes=K, width=16, layers=4)
    S = _sin(prob.m, K)
    an = 2.0 / (prob.m + 1)  # series coefficients c = an * v S^T, synthesis v = c S
    with FDEProblem.from_inputs(prob) as p:
        p.assemble()
        feat = torch.empty(net.cin * K, dtype=torch.float32, device="cuda")
        net.features(p.h, feat)
        f = feat.cpu().numpy().reshape(net.cin, K)
        spec = an * np.concatenate([prob.u0[None], prob.f]) @ S.T  # (s+2) x K sine-series coefficients
        ref = np.concatenate([spec, np.full((1, K), (prob.alpha - 1.5) / 0.4),
                              np.full((1, K), (prob.dplus.mean() - 1.25) / 0.75),
                              np.full((1, K), (prob.dminus.mean() - 1.25) / 0.75),
                              (np.arange(1, K + 1) / K)[None]])
        np.testing.assert_allclose(f, ref, rtol=1e-6, atol=1e-6 * np.abs(spec).max())
        # coefficients / synthesis of a space-time vector: the orthogonal projection onto the K modes
        xv = torch.as_tensor(np.random.default_rng(2).standard_normal(prob.n), device="cuda")
        coef = torch.empty(prob.s * K, dtype=torch.float32, device="cuda")
        net.coefficients(xv, coef)
        X = xv.cpu().numpy().reshape(prob.s, prob.m)
        np.testing.assert_allclose(coef.cpu().numpy().reshape(prob.s, K), an * X @ S.T, rtol=1e-5, atol=1e-5)
        back = torch.empty(prob.n, dtype=torch.float64, device="cuda")
        net.synthesize(coef, back)
        np.testing.assert_allclose(back.cpu().numpy().reshape(prob.s, prob.m), an * (X @ S.T) @ S, rtol=0, atol=1e-5)
        # FP16 inference path against the FP32 forward, both synthesised on the grid
        x0 = torch.empty(prob.n, dtype=torch.float64, device="cuda")
        net.warm_start(p.h, x0)
        y32 = net.forward(feat, 1).cpu().numpy().reshape(prob.s, K) @ S
        y16 = x0.cpu().numpy().reshape(prob.s, prob.m)
        assert np.abs(y16 - y32).max() <= 1e-2 * max(np.abs(y32).max(), 1e-3)


def _dataset(net, probs, precision="fp32"):
    """Solve the instances with the batched solver; features and solutions as FP32 device arrays."""
    from paper_1305_6653_gb300 import FDEBatch
    feats, targets = [], []
    for c0 in range(0, len(probs), 64):
        chunk = probs[c0:c0 + 64]
        with FDEBatch(chunk, device_inputs=True) as b:  # solutions stay on the device
            b.assemble().factor(precision)
            xs, st = b.solve(tol=1e-10)
            assert all(s_["status"] == 0 for s_ in st)
            for i, x in enumerate(xs):
                f = torch.empty(net.cin * net.modes, dtype=torch.float32, device="cuda")
                net.features(b.problem(i), f)
                c = torch.empty(net.s * net.modes, dtype=torch.float32, device="cuda")
                net.coefficients(x, c)
                feats.append(f)
                targets.append(c)
    return torch.stack(feats), torch.stack(targets)


def test_trained_warm_start_saves_iterations():
    """Train on method-generated solves of the learned family (m=63, s=16, GBDF3),
    then solve held-out instances from the learned guess and from zero."""
    from paper_1305_6653_gb300 import FDENop, FDEProblem
    m, s = 63, 16
    net = FDENop(m, s, modes=16, width=64, layers=6, ksize=5, seed=1305)
    train = [fi.config_learned_family(seed=i, m=m, s=s) for i in range(256)]
    X, Y = _dataset(net, train)
    B = 32
    for step in range(1500):
        i0 = (step * B) % len(train)
        loss, _ = net.loss_grad(X[i0:i0 + B].reshape(-1), Y[i0:i0 + B].reshape(-1), B)
        net.adam_step(3e-3 if step < 900 else (1e-3 if step < 1300 else 3e-4))
    zero_its, warm_its = [], []
    for seed in range(10**6, 10**6 + 12):
        prob = fi.config_learned_family(seed=seed, m=m, s=s)
        ref = O.direct_solve(prob)
        with FDEProblem.from_inputs(prob) as p:
            p.assemble().factor("fp32")
            _, st0 = p.solve(tol=1e-11)
            x0 = torch.empty(prob.n, dtype=torch.float64, device="cuda")
            net.warm_start(p.h, x0)
            x, st1 = p.solve(tol=1e-11, x0=x0)
            xs = x.cpu().numpy()
        assert st1["status"] == 0
        assert np.linalg.norm(xs - ref) / np.linalg.norm(ref) <= 1e-8
        zero_its.append(st0["iterations"])
        warm_its.append(st1["iterations"])
    # the guess must never cost iterations (worse guesses fall back to zero) and must
    # save some on average: the residual floor of a 16-mode guess is ~0.1-0.2 ||b||
    assert all(w <= z for w, z in zip(warm_its, zero_its)), (zero_its, warm_its, loss)
    assert np.mean(warm_its) < np.mean(zero_its), (zero_its, warm_its, loss)
