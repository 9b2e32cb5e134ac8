"""Pins of the surrogate network's FP64 oracle: the convolution against a
direct per-pixel sum, and the hand-written backward pass against central
finite differences of the loss."""
import numpy as np
import pytest

from oracle import surrogate as S


def test_conv_matches_direct_sum():
    rng = np.random.default_rng(0)
    x = rng.normal(size=(2, 5, 6, 3))
    w = rng.normal(size=(9, 4, 3))
    b = rng.normal(size=4)
    out = S.conv3x3(x, w, b)
    n, y, xx, o = 1, 0, 5, 2
    ref = b[o]
    for t, (dy, dx) in enumerate(S.TAPS):
        ref += sum(x[n, (y + dy) % 5, (xx + dx) % 6, i] * w[t, o, i] for i in range(3))
    assert out[n, y, xx, o] == pytest.approx(ref, rel=1e-13)


def test_identity_when_projection_is_zero():
    p = S.init_params(channels=8, blocks=2, seed=1)
    p["proj"] = (np.zeros_like(p["proj"][0]), np.zeros_like(p["proj"][1]))
    x = np.random.default_rng(2).normal(size=(1, 6, 7, 4))
    y, _ = S.forward(p, x)
    assert np.array_equal(y, x)


def test_mass_conserving_layer_keeps_each_samples_mass():
    # the density channel's sum over each image equals the input's; the other
    # channels and the density's deviations from its mean are untouched
    rng = np.random.default_rng(5)
    p = S.init_params(channels=6, blocks=1, seed=6)
    p["proj"] = (rng.normal(0, 0.3, p["proj"][0].shape), rng.normal(0, 0.3, p["proj"][1].shape))
    x = rng.normal(size=(3, 5, 7, 4))
    y0, _ = S.forward(p, x)
    y1, _ = S.forward(p, x, conserve_mass=True)
    assert np.abs(y1[..., 0].sum(axis=(1, 2)) - x[..., 0].sum(axis=(1, 2))).max() < 1e-12
    assert np.abs(y0[..., 0].sum(axis=(1, 2)) - x[..., 0].sum(axis=(1, 2))).min() > 1e-3
    assert np.array_equal(y1[..., 1:], y0[..., 1:])
    d0 = y0[..., 0] - y0[..., 0].mean(axis=(1, 2), keepdims=True)
    d1 = y1[..., 0] - y1[..., 0].mean(axis=(1, 2), keepdims=True)
    assert np.abs(d1 - d0).max() < 1e-12


@pytest.mark.parametrize("conserve_mass", [False, True])
def test_backward_matches_finite_differences(conserve_mass):
    rng = np.random.default_rng(3)
    p = S.init_params(channels=6, blocks=2, seed=4, scale=1.0)
    # make every term matter
    p["proj"] = (rng.normal(0, 0.3, p["proj"][0].shape), rng.normal(0, 0.1, p["proj"][1].shape))
    p["blocks"] = [((rng.normal(0, 0.4, w1.shape), rng.normal(0, 0.1, b1.shape)),
                    (rng.normal(0, 0.4, w2.shape), rng.normal(0, 0.1, b2.shape)))
                   for (w1, b1), (w2, b2) in p["blocks"]]
    x = rng.normal(size=(2, 5, 6, 4))
    target = rng.normal(size=x.shape)
    y, cache = S.forward(p, x, conserve_mass)
    g = S.backward(p, cache, y, target)
    params, grads = S.flatten(p), S.flatten(g)
    for arr, garr in zip(params, grads):
        flat = arr.reshape(-1)
        for idx in rng.choice(flat.size, size=min(4, flat.size), replace=False):
            old = flat[idx]
            h = 1e-6
            flat[idx] = old + h
            lp = S.loss(S.forward(p, x, conserve_mass)[0], target)
            flat[idx] = old - h
            lm = S.loss(S.forward(p, x, conserve_mass)[0], target)
            flat[idx] = old
            fd = (lp - lm) / (2 * h)
            assert garr.reshape(-1)[idx] == pytest.approx(fd, rel=1e-5, abs=1e-10)
