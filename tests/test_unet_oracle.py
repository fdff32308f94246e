"""Pins of the numpy U-Net oracle: convolution against scipy's correlate2d,
pooling / upsampling adjoint identities, and every parameter gradient of the
whole network against central finite differences."""
import numpy as np

from oracle import unet_oracle as U
from paper_2203_01462_gb300 import inputs as I


def test_conv_matches_scipy_correlate2d():
    from scipy.signal import correlate2d
    rng = np.random.default_rng(0)
    x = rng.standard_normal((2, 3, 9, 7))
    w = rng.standard_normal((4, 3, 3, 3))
    b = rng.standard_normal(4)
    y = U.conv(x, w, b, relu=False)
    for n in range(2):
        for o in range(4):
            ref = b[o] + sum(correlate2d(x[n, c], w[o, c], mode="same") for c in range(3))
            np.testing.assert_allclose(y[n, o], ref, rtol=1e-12, atol=1e-12)


def test_pool_and_upsample_adjoints():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((2, 3, 8, 6))
    d = rng.standard_normal((2, 3, 4, 3))
    assert abs(np.sum(U.pool(x) * d) - np.sum(x * U.pool_backward(d))) < 1e-12
    z = rng.standard_normal((2, 3, 4, 3))
    e = rng.standard_normal((2, 3, 8, 6))
    assert abs(np.sum(U.up(z) * e) - np.sum(z * U.up_backward(e))) < 1e-12


def test_network_gradients_match_central_differences():
    rng = np.random.default_rng(2)
    params = I.unet_params(base=2, seed=3)
    for k in params:  # non-zero biases so that every ReLU path is exercised
        if k.endswith(".b"):
            params[k] = 0.1 * rng.standard_normal(params[k].shape)
    x = rng.standard_normal((2, 2, 16, 16))
    t = rng.standard_normal((2, 1, 16, 16))
    out, cache = U.forward(params, x)
    L0, dout = U.mse(out, t)
    grads = U.backward(params, cache, dout)
    for key in params:
        flat = params[key].reshape(-1)
        for idx in rng.choice(flat.size, min(3, flat.size), replace=False):
            h = 1e-6
            old = flat[idx]
            flat[idx] = old + h
            Lp = U.mse(U.forward(params, x)[0], t)[0]
            flat[idx] = old - h
            Lm = U.mse(U.forward(params, x)[0], t)[0]
            flat[idx] = old
            fd = (Lp - Lm) / (2 * h)
            an = grads[key].reshape(-1)[idx]
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(fd)), (key, idx, fd, an)


def test_param_count_is_about_a_million():
    assert 0.9e6 < I.unet_param_count(24) < 1.3e6


def test_bf16_rounding():
    """Round to nearest even at 8 significant bits: 1 + 2^-8 lies halfway
    between 1 and 1 + 2^-7 and goes to the even 1; 1 + 3 2^-8 goes to 1 + 2^-6;
    a value off the halfway point goes to the nearer neighbour; every result
    has at most 8 significant bits and lies within the unit roundoff 2^-8
    relative (plus the FP32 step)."""
    vals = np.array([1 + 2 ** -8, 1 + 3 * 2 ** -8, 1 + 2 ** -8 + 2 ** -12, -(1 + 2 ** -8 + 2 ** -12), 3.0, 0.0])
    r = U.bf16(vals)
    assert r.tolist() == [1.0, 1 + 2 ** -6, 1 + 2 ** -7, -(1 + 2 ** -7), 3.0, 0.0]
    x = np.random.default_rng(3).standard_normal(10000) * 10.0 ** np.random.default_rng(4).uniform(-5, 5, 10000)
    r = U.bf16(x)
    assert np.all(np.abs(r - x) <= (2 ** -8 + 2 ** -23) * np.abs(x))  # via FP32: one FP32 rounding more
    m, _ = np.frexp(r)
    assert np.all((m * 2 ** 8) == np.round(m * 2 ** 8))


def test_bf16_conv_rounds_only_the_factors():
    """With rnd = bf16 the convolution equals the exact one of the rounded
    operands (sums stay FP64)."""
    rng = np.random.default_rng(8)
    x = rng.standard_normal((2, 3, 6, 5))
    w = rng.standard_normal((4, 3, 3, 3))
    b = rng.standard_normal(4)
    np.testing.assert_allclose(U.conv(x, w, b, False, U.bf16), U.conv(U.bf16(x), U.bf16(w), b, False), rtol=1e-14)
