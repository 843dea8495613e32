"""Pins of the surrogate reference (oracle/surrogate_ref.py) against independent mathematics:
scipy's correlation for the dilated convolution, central differences for every gradient,
and the closed form of a first Adam step."""
import numpy as np
import pytest

from oracle import surrogate_ref as S

signal = pytest.importorskip("scipy.signal")


def test_bf16_rounding():
    x = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, -2.5, 0.0, 1e-30, np.nan], np.float32)
    r = S.bf16(x)
    assert r[0] == 1.0
    assert r[1] == 1.0  # halfway -> even
    assert r[2] == 1.0 + 2 ** -7  # above halfway -> up
    assert r[3] == -2.5 and r[4] == 0.0 and np.isnan(r[6])


def test_conv_matches_scipy_correlate():
    rng = np.random.default_rng(0)
    for d in (1, 2, 4):
        x = rng.normal(size=(2, 21, 19, 3))
        w = rng.normal(size=(4, 3, 3, 3))
        b = rng.normal(size=4)
        y = S.conv_valid(x, w, b, d)
        wd = np.zeros((4, 2 * d + 1, 2 * d + 1, 3))
        wd[:, ::d, ::d, :] = w  # dilated kernel
        for bi in range(2):
            for o in range(4):
                ref = b[o] + sum(signal.correlate(x[bi, :, :, c], wd[o, :, :, c], mode="valid") for c in range(3))
                assert np.allclose(y[bi, :, :, o], ref, atol=1e-12)


def test_features_central_differences():
    res = 0.05
    yy, xx = np.mgrid[0:12, 0:10] * res
    e = 0.3 * xx - 0.2 * yy + 1.0
    f = S.features(e, res)
    assert f.shape == (10, 8, 2)
    assert np.allclose(f[..., 0], 0.3) and np.allclose(f[..., 1], -0.2)


def test_network_gradient_central_differences():
    rng = np.random.default_rng(1)
    n_out = 6
    theta = np.concatenate([rng.normal(scale=0.3, size=int(np.prod(s))) for s in S.param_shapes(n_out)])
    feat = rng.normal(size=(2, 46, 46, 2))
    labels = rng.normal(size=(2, 16, 16, n_out))
    labels[0, 0, 0, 0] = np.nan  # excluded from the loss
    loss, g, _ = S.loss_and_grad(theta, feat, labels, n_out, round_bf16=False)
    idx = rng.choice(theta.size, 40, replace=False)
    h = 1e-6
    for i in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        lp = S.loss_and_grad(tp, feat, labels, n_out, round_bf16=False)[0]
        lm = S.loss_and_grad(tm, feat, labels, n_out, round_bf16=False)[0]
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[i]) <= 1e-5 * max(1.0, abs(fd)), (i, fd, g[i])


def test_adam_first_step_closed_form():
    theta = np.array([1.0, -2.0, 0.5])
    g = np.array([0.1, -3.0, 0.0])
    t1, m, v = S.adam(theta, g, np.zeros(3), np.zeros(3), 1, lr=0.01)
    # bias-corrected first step: m_hat = g, v_hat = g^2 -> step = lr * sign(g) (eps aside)
    assert np.allclose(t1[:2], theta[:2] - 0.01 * np.sign(g[:2]), atol=1e-9)
    assert t1[2] == theta[2]
