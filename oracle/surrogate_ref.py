"""FP64 reference of the learned surrogate's arithmetic (convolution stack, loss, backward, Adam).

TEST INFRASTRUCTURE ONLY (like the rest of ``oracle/``): the GPU tests compare libseb's
surrogate kernels with these functions on the same inputs.  The paper defines no learned
model (it notes learned traversability as unreliable, Sec. II-A); what is fixed here is plain
mathematics: valid dilated cross-correlation, ReLU, a 1x1 head, mean squared error, its exact
gradient, and Adam (Kingma & Ba, 2015).  Pins: ``tests/test_surrogate_pins.py`` (BF16 rounding,
the convolution against scipy.signal.correlate, the features and the network gradient against
central differences, the first Adam step against its closed form).  The network is not the
paper's, so no value printed in the paper applies to it; every function here is pinned by
the mathematics above.

Tensors are channel-last: activations [B][H][W][C], conv weights [Cout][3][3][Cin], head
weights [Cout][Cin].  Stored activations and weights are rounded to bfloat16 (round to
nearest even) exactly where the GPU stores them in bfloat16.
"""
from __future__ import annotations

import numpy as np

DILATIONS = (1, 2, 4, 8)
HIDDEN = 32
IN_FEATURES = 2


def bf16(x):
    """Round float values to the nearest bfloat16 (ties to even), returned as float64."""
    a = np.ascontiguousarray(np.asarray(x, np.float32))
    u = a.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    r = r.astype(np.uint32)
    nan = np.isnan(a)
    out = r.view(np.float32).astype(np.float64)
    out[nan] = np.nan
    return out


def features(elev, res):
    """Slope features of an elevation patch [.., H, W]: central differences / (2 res) on the
    interior [.., H-2, W-2, 2] (channel 0 along x, channel 1 along y); unknown -> 0."""
    e = np.asarray(elev, np.float64)
    fx = (e[..., 1:-1, 2:] - e[..., 1:-1, :-2]) / (2 * res)
    fy = (e[..., 2:, 1:-1] - e[..., :-2, 1:-1]) / (2 * res)
    f = np.stack([fx, fy], axis=-1)
    return np.where(np.isfinite(f), f, 0.0)


def conv_valid(x, w, b, d):
    """y[b, i, j, o] = b[o] + sum_{u, v, c} w[o, u, v, c] x[b, i + u d, j + v d, c]."""
    B, H, W, C = x.shape
    O = w.shape[0]
    Ho, Wo = H - 2 * d, W - 2 * d
    y = np.zeros((B, Ho, Wo, O)) + b
    for u in range(3):
        for v in range(3):
            patch = x[:, u * d:u * d + Ho, v * d:v * d + Wo, :]
            y += patch @ w[:, u, v, :].T
    return y


def conv_valid_backward(x, w, dy, d):
    """Gradients of conv_valid: (dx, dw, db) for upstream dy."""
    B, H, W, C = x.shape
    Ho, Wo = dy.shape[1], dy.shape[2]
    dx = np.zeros_like(x, dtype=np.float64)
    dw = np.zeros_like(w, dtype=np.float64)
    for u in range(3):
        for v in range(3):
            patch = x[:, u * d:u * d + Ho, v * d:v * d + Wo, :]
            dw[:, u, v, :] = np.einsum("bijo,bijc->oc", dy, patch)
            dx[:, u * d:u * d + Ho, v * d:v * d + Wo, :] += dy @ w[:, u, v, :]
    return dx, dw, dy.sum(axis=(0, 1, 2))


def param_shapes(n_out):
    shapes = []
    cin = IN_FEATURES
    for _ in DILATIONS:
        shapes += [(HIDDEN, 3, 3, cin), (HIDDEN,)]
        cin = HIDDEN
    shapes += [(n_out, HIDDEN), (n_out,)]
    return shapes


def unpack(theta, n_out):
    out, o = [], 0
    for s in param_shapes(n_out):
        n = int(np.prod(s))
        out.append(np.asarray(theta[o:o + n], np.float64).reshape(s))
        o += n
    return out


def forward(theta, feat, n_out, round_bf16=True):
    """feat [B][46][46][2] -> (pred [B][16][16][n_out], stored activations)."""
    r = bf16 if round_bf16 else (lambda a: np.asarray(a, np.float64))
    p = unpack(theta, n_out)
    x = r(feat)
    acts = [x]
    for li, d in enumerate(DILATIONS):
        w, b = r(p[2 * li]), p[2 * li + 1]
        x = r(np.maximum(conv_valid(x, w, b, d), 0.0))
        acts.append(x)
    wh, bh = r(p[8]), p[9]
    pred = x @ wh.T + bh
    return pred, acts


def loss_and_grad(theta, feat, labels, n_out, round_bf16=True, acts=None, pred=None):
    """Mean squared error over the finite labels and its gradient w.r.t. theta (FP64
    backward through the stored activations; the bfloat16 rounding is not differentiated).
    acts / pred, when given, are used as the stored forward values instead of recomputing."""
    r = bf16 if round_bf16 else (lambda a: np.asarray(a, np.float64))
    p = unpack(theta, n_out)
    if acts is None:
        pred, acts = forward(theta, feat, n_out, round_bf16)
    ok = np.isfinite(labels)
    cnt = max(1, int(ok.sum()))
    diff = np.where(ok, pred - np.where(ok, labels, 0.0), 0.0)
    loss = float((diff ** 2).sum() / cnt)
    dpred = 2.0 * diff / cnt
    grads = [None] * 10
    wh = r(p[8])
    grads[8] = np.einsum("bijo,bijc->oc", dpred, acts[4])
    grads[9] = dpred.sum(axis=(0, 1, 2))
    dx = dpred @ wh
    for li in reversed(range(4)):
        d = DILATIONS[li]
        dz = dx * (acts[li + 1] > 0)
        w = r(p[2 * li])
        dxi, dw, db = conv_valid_backward(acts[li], w, dz, d)
        grads[2 * li], grads[2 * li + 1] = dw, db
        dx = dxi
    return loss, np.concatenate([g.ravel() for g in grads]), pred


def adam(theta, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (t counts from 1)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v
