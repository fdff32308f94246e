"""The surrogate network on the library's kernels against the numpy oracle:
GEMM in all transpose modes on ragged sizes, the U-Net's forward output and
every parameter gradient (FP32 kernels vs FP64 oracle), and training."""
import numpy as np
import pytest

from oracle import unet_oracle as U
from paper_2203_01462_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("ta,tb", [(0, 0), (0, 1), (1, 0), (1, 1)])
def test_gemm_transposes_ragged(ta, tb):
    import torch
    from paper_2203_01462_gb300.surrogate import _nn, _p
    rng = np.random.default_rng(ta * 2 + tb)
    M, N, K = 67, 130, 45
    A = rng.standard_normal((K, M) if ta else (M, K)).astype(np.float32)
    B = rng.standard_normal((N, K) if tb else (K, N)).astype(np.float32)
    Cm = rng.standard_normal((M, N)).astype(np.float32)
    ref = 0.7 * ((A.T if ta else A).astype(np.float64) @ (B.T if tb else B).astype(np.float64)) + 0.3 * Cm
    a, b, c = (torch.tensor(v, device="cuda") for v in (A, B, Cm))
    rc = _nn().nn_gemm(ta, tb, M, N, K, 0.7, _p(a), A.shape[1], _p(b), B.shape[1], 0.3, _p(c), N, None)
    torch.cuda.synchronize()
    assert rc == 0
    np.testing.assert_allclose(c.cpu().numpy(), ref, rtol=1e-4, atol=1e-4)


def _setup(base=4, B=2, H=32, W=32, seed=5):
    rng = np.random.default_rng(seed)
    params = I.unet_params(base, seed)
    for k in params:
        if k.endswith(".b"):
            params[k] = 0.1 * rng.standard_normal(params[k].shape)
    x = rng.standard_normal((B, 2, H, W))
    t = rng.standard_normal((B, 1, H, W))
    return params, x, t


def _gpu(a):
    import torch
    return torch.tensor(np.ascontiguousarray(a.transpose(1, 0, 2, 3)), dtype=torch.float32, device="cuda")


def test_unet_forward_and_gradients_match_oracle():
    from paper_2203_01462_gb300.surrogate import UNet
    params, x, t = _setup()
    out_ref, cache = U.forward(params, x)
    L_ref, dout_ref = U.mse(out_ref, t)
    g_ref = U.backward(params, cache, dout_ref)
    net = UNet(base=4, batch=2, H=32, W=32, params=params)
    out = net.forward(_gpu(x)).cpu().numpy().transpose(1, 0, 2, 3)
    assert np.linalg.norm(out - out_ref) <= 1e-5 * np.linalg.norm(out_ref)
    net.backward(_gpu(dout_ref))
    g = net.grads()
    for key in g_ref:
        err = np.linalg.norm(g[key] - g_ref[key]) / max(np.linalg.norm(g_ref[key]), 1e-30)
        assert err <= 1e-4, (key, err)


def test_unet_training_reduces_the_loss():
    import torch
    from paper_2203_01462_gb300.surrogate import UNet
    params, x, t = _setup(base=8, B=4, H=32, W=32, seed=6)
    # a learnable target: a smooth function of the input
    t = np.tanh(x[:, :1] + 0.5 * x[:, 1:2])
    net = UNet(base=8, batch=4, H=32, W=32, params=params)
    xg, tg = _gpu(x), _gpu(t)
    first = float(net.train_step(xg, tg, lr=3e-3).item())
    for _ in range(150):
        last = float(net.train_step(xg, tg, lr=3e-3).item())
    assert last < 0.1 * first
