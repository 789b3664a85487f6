"""FP64 numpy reference of the learned warm start (test infrastructure only).

Written independently of the CUDA library from the definition of the
features and of the network (9 -> 64 -> 64 -> 2, tanh, BF16 weights) so that
the GPU features, loss and gradient can be checked against it.
"""
import numpy as np

__all__ = ["IN", "NPARAMS", "bf16_round", "unpack", "features", "targets", "loss_and_grad", "forward"]

IN, H, OUT = 9, 64, 2
NPARAMS = H * IN + H + H * H + H + OUT * H + OUT


def bf16_round(w):
    """float32 -> nearest bfloat16 (ties to even), returned as float64."""
    u = np.ascontiguousarray(w, dtype=np.float32).view(np.uint32).astype(np.uint64)
    bias = 0x7FFF + ((u >> 16) & 1)
    r = ((u + bias) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32).astype(np.float64)


def unpack(w):
    w = np.asarray(w, dtype=np.float64)
    o = 0
    W1 = w[o:o + H * IN].reshape(H, IN); o += H * IN
    b1 = w[o:o + H]; o += H
    W2 = w[o:o + H * H].reshape(H, H); o += H * H
    b2 = w[o:o + H]; o += H
    W3 = w[o:o + OUT * H].reshape(OUT, H); o += OUT * H
    b3 = w[o:o + OUT]
    return W1, b1, W2, b2, W3, b3


def _scales(g, w):
    N = w.size
    sw = w.sum()
    S1 = np.sqrt(np.sum(w * g[:N] ** 2) / sw)
    S2 = np.sqrt(np.sum(w * g[N:] ** 2) / sw)
    return S1, S2, sw / N


def features(g, w, dist, curv, band_eps, eps_in, eps_out, kappa, Ax0):
    """Per-node features (N x 9) and (S1, S2, mean w).  Ax0: the operator
    applied to x0 = Lambda^-1 g (2N), so that r = g - Ax0 is the residual of
    that start."""
    N = w.size
    S1, S2, mw = _scales(g, w)
    L = S1 / S2
    kL = kappa * L
    F = np.zeros((N, IN))
    F[:, 0] = g[:N] / S1
    F[:, 1] = g[N:] / S2
    F[:, 2] = dist / band_eps if band_eps > 0 else 0.0
    F[:, 3] = np.clip(curv * L, -10.0, 10.0) / 10.0
    F[:, 4] = kL / (1.0 + kL)
    F[:, 5] = np.log(eps_out / eps_in) / 5.0
    F[:, 6] = (eps_in / eps_out) / (1.0 + kL)
    F[:, 7] = (g[:N] - Ax0[:N]) / S1
    F[:, 8] = (g[N:] - Ax0[N:]) / S2
    return F, (S1, S2, mw)


def targets(p, w, scales, eps_in, eps_out):
    """Training targets (lambda1 psi/S1, lambda2 psin/S2), Lambda the diagonal of
    the system (Sec. 3.3), and the loss weights w/mean(w)."""
    N = w.size
    S1, S2, mw = scales
    lam1 = 0.5 * (1.0 + eps_out / eps_in)
    lam2 = 0.5 * (1.0 + eps_in / eps_out)
    return np.stack([lam1 * p[:N] / S1, lam2 * p[N:] / S2], axis=1), w / mw


def forward(params_bf16, F):
    W1, b1, W2, b2, W3, b3 = unpack(params_bf16)
    h1 = np.tanh(F @ W1.T + b1)
    h2 = np.tanh(h1 @ W2.T + b2)
    return h1, h2, h2 @ W3.T + b3


def loss_and_grad(params_bf16, F, T, wt):
    """Loss sum(wt |o - t|^2)/n and its gradient w.r.t. the (BF16-valued) parameters."""
    n = F.shape[0]
    W1, b1, W2, b2, W3, b3 = unpack(params_bf16)
    h1, h2, o = forward(params_bf16, F)
    e = o - T
    loss = np.sum(wt[:, None] * e * e) / n
    dO = 2.0 * wt[:, None] * e / n
    dW3 = dO.T @ h2
    db3 = dO.sum(0)
    d2 = (dO @ W3) * (1.0 - h2 * h2)
    dW2 = d2.T @ h1
    db2 = d2.sum(0)
    d1 = (d2 @ W2) * (1.0 - h1 * h1)
    dW1 = d1.T @ F
    db1 = d1.sum(0)
    grad = np.concatenate([dW1.ravel(), db1, dW2.ravel(), db2, dW3.ravel(), db3])
    return loss, grad
