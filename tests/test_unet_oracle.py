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
