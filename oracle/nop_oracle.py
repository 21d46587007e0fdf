"""Plain FP64 CPU oracle of the 1-D convolutional neural operator used as a warm
start for the space-time GMRES solve.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  The paper has no learned
component; this operator is an addition whose only effect is the initial guess
x0 of GMRES -- the solution is still judged by the true FP64 residual.

Network: L layers of 1-D convolution over the spatial index x (length m, zero
padding, odd kernel size K, "same" output length); ReLU after every layer but
the last.  Parameters are stored flat, layer by layer: W_l (C_out, C_in, K) then
b_l (C_out).  Input (B, C_in, m), output (B, C_out_last, m).  Loss: mean squared
error over all outputs.

Definitions written out with explicit loops over the kernel offset (and numpy
broadcasting over batch, channels and positions).  Pinned in
tests/test_oracle_nop.py by central finite differences, by a single-channel
comparison with numpy.correlate, and by a hand-checked Adam step.
"""
from __future__ import annotations

import numpy as np

__all__ = ["layer_shapes", "num_params", "unpack", "forward", "loss_and_grad", "adam_step"]


def layer_shapes(cin: int, cout: int, width: int, layers: int, K: int):
    """[(C_in, C_out, K)] of each layer: cin -> width -> ... -> width -> cout."""
    dims = [cin] + [width] * (layers - 1) + [cout]
    return [(dims[i], dims[i + 1], K) for i in range(layers)]


def num_params(shapes) -> int:
    return sum(co * ci * k + co for ci, co, k in shapes)


def unpack(theta: np.ndarray, shapes):
    out, o = [], 0
    for ci, co, k in shapes:
        W = theta[o:o + co * ci * k].reshape(co, ci, k)
        o += co * ci * k
        b = theta[o:o + co]
        o += co
        out.append((W, b))
    return out


def _conv(x: np.ndarray, W: np.ndarray, b: np.ndarray) -> np.ndarray:
    """y[n, o, i] = b[o] + sum_c sum_k W[o, c, k] x[n, c, i + k - K//2] (zero outside 0..m-1)."""
    B, C, m = x.shape
    O, _, K = W.shape
    h = K // 2
    xp = np.zeros((B, C, m + 2 * h))
    xp[:, :, h:h + m] = x
    y = np.zeros((B, O, m)) + b[None, :, None]
    for k in range(K):
        y += np.einsum("oc,ncm->nom", W[:, :, k], xp[:, :, k:k + m])
    return y


def forward(theta, shapes, x: np.ndarray, keep: bool = False):
    params = unpack(np.asarray(theta, dtype=np.float64), shapes)
    acts = [np.asarray(x, dtype=np.float64)]
    pre = []
    a = acts[0]
    for li, (W, b) in enumerate(params):
        z = _conv(a, W, b)
        pre.append(z)
        a = np.maximum(z, 0.0) if li < len(params) - 1 else z
        acts.append(a)
    return (a, acts, pre) if keep else a


def loss_and_grad(theta, shapes, x: np.ndarray, target: np.ndarray):
    """MSE loss and its gradient with respect to the flat parameters (backpropagation)."""
    params = unpack(np.asarray(theta, dtype=np.float64), shapes)
    y, acts, pre = forward(theta, shapes, x, keep=True)
    N = y.size
    loss = float(np.sum((y - target) ** 2) / N)
    g = 2.0 * (y - target) / N  # dL/dy
    grads = []
    for li in range(len(params) - 1, -1, -1):
        W, b = params[li]
        if li < len(params) - 1:
            g = g * (pre[li] > 0)  # through the ReLU
        a = acts[li]
        B, C, m = a.shape
        O, _, K = W.shape
        h = K // 2
        ap = np.zeros((B, C, m + 2 * h))
        ap[:, :, h:h + m] = a
        dW = np.zeros_like(W)
        for k in range(K):
            dW[:, :, k] = np.einsum("nom,ncm->oc", g, ap[:, :, k:k + m])
        db = g.sum(axis=(0, 2))
        grads.append((dW, db))
        # gradient with respect to the layer input: a[n,c,j] receives W[o,c,k] g[n,o,j-k+h]
        gp = np.zeros((B, O, m + 2 * h))
        gp[:, :, h:h + m] = g
        ga = np.zeros_like(a)
        for k in range(K):
            ga += np.einsum("oc,nom->ncm", W[:, :, k], gp[:, :, 2 * h - k:2 * h - k + m])
        g = ga
    flat = []
    for dW, db in reversed(grads):
        flat.append(dW.reshape(-1))
        flat.append(db)
    return loss, np.concatenate(flat)


def adam_step(theta, grad, m1, m2, t: int, lr: float, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba): returns (theta, m1, m2) after step t (1-based)."""
    m1 = beta1 * m1 + (1 - beta1) * grad
    m2 = beta2 * m2 + (1 - beta2) * grad * grad
    mhat = m1 / (1 - beta1 ** t)
    vhat = m2 / (1 - beta2 ** t)
    return theta - lr * mhat / (np.sqrt(vhat) + eps), m1, m2
