"""Pins of the CPU FP64 U-Net oracle (the learned field-solve warm start):
its operations against library routines and closed forms, and its
gradients against central finite differences."""
import numpy as np
import pytest
import scipy.signal

from oracle import unet as U
from paper_2206_14662_gb300.inputs import unet_init_flat, unet_layer_shapes


def test_conv3_single_channel_is_scipy_correlate():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((13, 21))
    k = rng.standard_normal((3, 3))
    got = U.conv3(x[None, :, :, None], k[:, :, None, None], np.zeros(1))[0, :, :, 0]
    ref = scipy.signal.correlate2d(x, k, mode="same", boundary="fill", fillvalue=0.0)
    assert np.abs(got - ref).max() <= 1e-13


def test_conv3_channel_mixing_is_a_sum_of_single_channel_correlations():
    rng = np.random.default_rng(2)
    x = rng.standard_normal((1, 8, 10, 3))
    W = rng.standard_normal((3, 3, 3, 2))
    b = rng.standard_normal(2)
    got = U.conv3(x, W, b)
    for o in range(2):
        ref = b[o] + sum(scipy.signal.correlate2d(x[0, :, :, i], W[:, :, i, o], mode="same")
                         for i in range(3))
        assert np.abs(got[0, :, :, o] - ref).max() <= 1e-12


def test_upconv_and_pool_closed_forms():
    rng = np.random.default_rng(3)
    x = rng.standard_normal((2, 4, 6, 1))
    up = U.upconv(x, np.ones((2, 2, 1, 1)), np.zeros(1))
    assert np.array_equal(up[..., 0], np.kron(x[..., 0], np.ones((1, 2, 2))))
    assert np.abs(U.pool(up) - x).max() <= 1e-15
    # a 2 x 2 kernel with one non-zero tap scatters to that sub-grid only
    Wd = np.zeros((2, 2, 1, 1))
    Wd[1, 0] = 3.0
    up = U.upconv(x, Wd, np.zeros(1))
    assert np.array_equal(up[:, 1::2, 0::2, 0], 3.0 * x[..., 0])
    assert not up[:, 0::2, :, 0].any() and not up[:, :, 1::2, 0].any()


def test_flat_layout_round_trip_and_count():
    c = 4
    v = unet_init_flat(c, seed=5)
    shapes = dict(unet_layer_shapes(c))
    assert shapes == U.layer_shapes(c)
    n = sum(int(np.prod(s)) + (1 if k == "head" else s[-1]) for k, s in shapes.items())
    assert len(v) == n
    assert np.array_equal(U.flatten(U.unflatten(v, c)), v)


@pytest.mark.parametrize("seed", [0, 1])
def test_gradients_match_central_differences(seed):
    """Directional derivatives of the loss along a random direction per
    parameter tensor (and the input) against central differences: a dropped
    term, a wrong tap, a transposed weight or a missing mask in backward
    fails this."""
    c, B, H, W = 4, 2, 16, 32
    rng = np.random.default_rng(10 + seed)
    p = U.unflatten(unet_init_flat(c, seed=seed, head_std=0.3, bias_std=0.1), c)
    x = rng.standard_normal((B, H, W, 2))
    t = rng.standard_normal((B, H, W))
    y, a = U.forward(p, x)
    g = U.backward(p, a, (y - t) / y.size)
    h = 1e-6
    for key in list(p.keys()) + ["x"]:
        base = x if key == "x" else p[key]
        d = rng.standard_normal(base.shape)
        def L(s):
            if key == "x":
                return U.loss(U.forward(p, x + s * d)[0], t)
            q = dict(p)
            q[key] = p[key] + s * d
            return U.loss(U.forward(q, x)[0], t)
        fd = (L(h) - L(-h)) / (2 * h)
        an = float(np.sum(g[key] * d))
        assert abs(fd - an) <= 1e-6 * max(abs(an), 1e-8) + 1e-12, (key, fd, an)


def test_adam_first_steps_closed_forms():
    """Adam's first steps worked out by hand: at t = 1 the bias-corrected
    moments are g and g^2, so with eps = 0 every weight moves by exactly
    lr sign(g) whatever |g|; a constant gradient keeps that step at t = 2;
    two different gradients g1, g2 give mhat = (beta1 g1 + g2)/(1 + beta1)
    and vhat = (beta2 g1^2 + g2^2)/(1 + beta2) at t = 2."""
    lr, b1, b2 = 1e-3, 0.9, 0.999
    w0 = np.array([0.5, -0.25, 2.0, 0.0, 1e-3])
    g1 = np.array([3.0, -1e-4, 2.5e5, -7.0, 0.5])
    w1, m1, v1 = U.adam_step(w0, g1, np.zeros(5), np.zeros(5), 1, lr, b1, b2, eps=0.0)
    assert np.allclose(w1, w0 - lr * np.sign(g1), rtol=0, atol=1e-15)
    assert np.allclose(m1, 0.1 * g1, rtol=1e-15) and np.allclose(v1, 0.001 * g1 ** 2, rtol=1e-12)
    w2, _, _ = U.adam_step(w1, g1, m1, v1, 2, lr, b1, b2, eps=0.0)
    assert np.allclose(w2, w0 - 2 * lr * np.sign(g1), rtol=0, atol=1e-15)
    g2 = np.array([-1.0, 2e-4, 1e5, -7.0, 0.25])
    w2, m2, v2 = U.adam_step(w1, g2, m1, v1, 2, lr, b1, b2, eps=1e-8)
    mhat = (b1 * g1 + g2) / (1 + b1)
    vhat = (b2 * g1 ** 2 + g2 ** 2) / (1 + b2)
    assert np.allclose(w2, w1 - lr * mhat / (np.sqrt(vhat) + 1e-8), rtol=0, atol=1e-15)
    # a zero gradient from zero moments leaves the weight where it is
    w, m, v = U.adam_step(np.ones(2), np.zeros(2), np.zeros(2), np.zeros(2), 1, lr)
    assert np.array_equal(w, np.ones(2)) and not m.any() and not v.any()
