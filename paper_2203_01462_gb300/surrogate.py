"""Learned sensitivity surrogate: a 4-level convolutional U-Net trained on
(rho, damping level) -> normalised dW~/drho pairs that the adjoint runs
produce, used to take cheap design steps between adjoint runs.

The network runs on the library's own kernels (``include/surrogate.h``):
im2col + GEMM convolutions, bias + ReLU, average pooling, nearest
upsampling, MSE and Adam.  The GEMMs run either in FP32 on the library's
tiled kernel (precision "f32") or with BF16 operands on the tensor cores
(the library's mma.sync kernel) and FP32 accumulation (precision "bf16";
FP32 master weights and Adam state).  This module only allocates buffers
(PyTorch) and sequences kernel calls.  Activations are [C][B][H][W]; a decoder level's
input is one buffer [upsampled deeper features | skip], and the encoder
writes its skip straight into the second half.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import inputs as I
from .binding import load

_FNS = {
    "nn_gemm": [C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_float, C.c_void_p, C.c_int, C.c_void_p, C.c_int,
                C.c_float, C.c_void_p, C.c_int, C.c_void_p, C.c_longlong, C.c_void_p],
    "nn_im2col3": [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p],
    "nn_col2im3_add": [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p],
    "nn_bias_act": [C.c_void_p, C.c_void_p, C.c_int, C.c_longlong, C.c_int, C.c_void_p],
    "nn_act_bwd_bias": [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_longlong, C.c_int, C.c_void_p],
    "nn_pool2": [C.c_void_p, C.c_longlong, C.c_int, C.c_int, C.c_void_p, C.c_void_p],
    "nn_pool2_bwd_add": [C.c_void_p, C.c_longlong, C.c_int, C.c_int, C.c_void_p, C.c_void_p],
    "nn_up2": [C.c_void_p, C.c_longlong, C.c_int, C.c_int, C.c_void_p, C.c_void_p],
    "nn_up2_bwd_add": [C.c_void_p, C.c_longlong, C.c_int, C.c_int, C.c_void_p, C.c_void_p],
    "nn_mse": [C.c_void_p, C.c_void_p, C.c_longlong, C.c_void_p, C.c_void_p, C.c_void_p],
    "nn_adam": [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_longlong, C.c_float, C.c_float, C.c_float,
                C.c_float, C.c_int, C.c_void_p],
    "nn_zero": [C.c_void_p, C.c_longlong, C.c_void_p],
    "nn_gemm_bf16": [C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_float, C.c_void_p, C.c_int, C.c_void_p,
                     C.c_int, C.c_float, C.c_void_p, C.c_int, C.c_void_p, C.c_longlong, C.c_void_p],
}
EXPORTS = sorted(_FNS)
_lib = None


def _nn():
    global _lib
    if _lib is None:
        L = load()
        for name, args in _FNS.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = C.c_int
        _lib = L
    return _lib


def _p(t: torch.Tensor) -> C.c_void_p:
    return C.c_void_p(t.data_ptr())


def _ck(rc: int, what: str) -> None:
    if rc != 0:
        raise RuntimeError("%s failed (%d)" % (what, rc))


class UNet:
    """The surrogate network for batches of B inputs of H x W (H, W multiples of 8)."""

    def __init__(self, base: int = 24, batch: int = 4, H: int = 256, W: int = 256, seed: int = 0,
                 device="cuda", stream=None, params: dict | None = None, precision: str = "f32"):
        assert H % 8 == 0 and W % 8 == 0
        if precision not in ("f32", "bf16"):
            raise ValueError("precision must be 'f32' or 'bf16'")
        self.base, self.B, self.H, self.W = base, batch, H, W
        self.precision = precision
        self.dev = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.dev)
        self.layers = I.unet_layers(base)
        p = params if params is not None else I.unet_params(base, seed)
        f32 = dict(dtype=torch.float32, device=self.dev)
        self.w = {n: torch.tensor(p[n + ".w"].reshape(co, ci * k * k), **f32) for n, ci, co, k in self.layers}
        self.b = {n: torch.tensor(p[n + ".b"], **f32) for n, ci, co, k in self.layers}
        self.gw = {n: torch.zeros_like(t) for n, t in self.w.items()}
        self.gb = {n: torch.zeros_like(t) for n, t in self.b.items()}
        self.m = {k: torch.zeros_like(t) for k, t in self._params()}
        self.v = {k: torch.zeros_like(t) for k, t in self._params()}
        self.step = 0
        b, B = base, batch
        sz = [(H >> l, W >> l) for l in range(4)]

        def buf(c, l):
            return torch.zeros((c, B, sz[l][0], sz[l][1]), **f32)

        # activations (a) and their gradients (g); cat_l = [up | skip_l]
        self.a = {"x": buf(2, 0), "enc1a": buf(b, 0), "cat1": buf(3 * b, 0),
                  "p1": buf(b, 1), "enc2a": buf(2 * b, 1), "cat2": buf(6 * b, 1),
                  "p2": buf(2 * b, 2), "enc3a": buf(4 * b, 2), "cat3": buf(12 * b, 2),
                  "p3": buf(4 * b, 3), "bota": buf(8 * b, 3), "botb": buf(8 * b, 3),
                  "dec3a": buf(4 * b, 2), "dec3b": buf(4 * b, 2),
                  "dec2a": buf(2 * b, 1), "dec2b": buf(2 * b, 1),
                  "dec1a": buf(b, 0), "dec1b": buf(b, 0), "head": buf(1, 0)}
        self.g = {k: torch.zeros_like(v) for k, v in self.a.items()}
        self.skip = {"enc1b": ("cat1", 2 * b, b), "enc2b": ("cat2", 4 * b, 2 * b), "enc3b": ("cat3", 8 * b, 4 * b)}
        col_elems = max(ci * k * k * B * sz[self._level(n)][0] * sz[self._level(n)][1]
                        for n, ci, co, k in self.layers)
        self.col = torch.zeros(col_elems, **f32)
        self.dcol = torch.zeros(col_elems, **f32)
        # split-K scratch of the GEMMs (partial products summed in a fixed
        # order): room for 16 slices of the largest weight matrix
        self.gemm_work = torch.zeros(max(1 << 20, 16 * max(co * ci * k * k for n, ci, co, k in self.layers)), **f32)
        self.loss = torch.zeros(1, dtype=torch.float64, device=self.dev)

    def sibling(self, batch: int) -> "UNet":
        """A network for another batch size that shares this one's parameter
        tensors (its gradients and Adam state are its own)."""
        twin = UNet(self.base, batch, self.H, self.W, device=self.dev, stream=self.stream,
                    params=self.numpy_params(), precision=self.precision)
        twin.w, twin.b = self.w, self.b
        return twin

    def numpy_params(self) -> dict:
        out = {}
        for n, ci, co, k in self.layers:
            out[n + ".w"] = self.w[n].double().cpu().numpy().reshape(co, ci, k, k)
            out[n + ".b"] = self.b[n].double().cpu().numpy()
        return out

    # ------------------------------------------------------------ helpers
    def _params(self):
        for n in self.w:
            yield n + ".w", self.w[n]
            yield n + ".b", self.b[n]

    @staticmethod
    def _level(name: str) -> int:
        return {"enc1a": 0, "enc1b": 0, "enc2a": 1, "enc2b": 1, "enc3a": 2, "enc3b": 2, "bota": 3, "botb": 3,
                "dec3a": 2, "dec3b": 2, "dec2a": 1, "dec2b": 1, "dec1a": 0, "dec1b": 0, "head": 0}[name]

    def _view(self, store: dict, name: str) -> torch.Tensor:
        """Output tensor of layer `name` (skips live inside the concat buffers)."""
        if name in self.skip:
            cat, lo, n = self.skip[name]
            return store[cat][lo:lo + n]
        return store[name]

    def _st(self):
        return C.c_void_p(self.stream.cuda_stream)

    def _gemm(self, ta, tb, M, N, K, A, lda, B, ldb, beta, Cm, ldc, what):
        L, st = _nn(), self._st()
        wk, nw = _p(self.gemm_work), self.gemm_work.numel()
        if self.precision == "bf16":
            rc = L.nn_gemm_bf16(ta, tb, M, N, K, 1.0, _p(A), lda, _p(B), ldb, beta, _p(Cm), ldc, wk, nw, st)
        else:
            rc = L.nn_gemm(ta, tb, M, N, K, 1.0, _p(A), lda, _p(B), ldb, beta, _p(Cm), ldc, wk, nw, st)
        _ck(rc, what)

    def _conv_fwd(self, name, ci, co, k, x, y, relu):
        L, st = _nn(), self._st()
        Bhw = x[0].numel()
        if k == 3:
            _ck(L.nn_im2col3(_p(x), ci, self.B, x.shape[2], x.shape[3], _p(self.col), st), "im2col")
            src = self.col
        else:
            src = x
        self._gemm(0, 0, co, Bhw, ci * k * k, self.w[name], ci * k * k, src, Bhw, 0.0, y, Bhw, "gemm fwd")
        _ck(L.nn_bias_act(_p(y), _p(self.b[name]), co, Bhw, int(relu), st), "bias_act")

    def _conv_bwd(self, name, ci, co, k, x, y, dy, dx, relu):
        """dy: gradient of the layer output (masked in place); dx += input gradient."""
        L, st = _nn(), self._st()
        Bhw = x[0].numel()
        _ck(L.nn_act_bwd_bias(_p(y), _p(dy), _p(self.gb[name]), co, Bhw, int(relu), st), "act_bwd")
        if k == 3:
            _ck(L.nn_im2col3(_p(x), ci, self.B, x.shape[2], x.shape[3], _p(self.col), st), "im2col")
            src = self.col
        else:
            src = x
        K = ci * k * k
        self._gemm(0, 1, co, K, Bhw, dy, Bhw, src, Bhw, 0.0, self.gw[name], K, "gemm wgrad")
        if dx is None:
            return
        if k == 3:
            self._gemm(1, 0, K, Bhw, co, self.w[name], K, dy, Bhw, 0.0, self.dcol, Bhw, "gemm dgrad")
            _ck(L.nn_col2im3_add(_p(self.dcol), ci, self.B, x.shape[2], x.shape[3], _p(dx), st), "col2im")
        else:
            self._gemm(1, 0, K, Bhw, co, self.w[name], K, dy, Bhw, 1.0, dx, Bhw, "gemm dgrad")

    # ------------------------------------------------------------ network
    def _in_of(self, name: str, store: dict) -> torch.Tensor:
        return {"enc1a": store["x"], "enc1b": store["enc1a"], "enc2a": store["p1"], "enc2b": store["enc2a"],
                "enc3a": store["p2"], "enc3b": store["enc3a"], "bota": store["p3"], "botb": store["bota"],
                "dec3a": store["cat3"], "dec3b": store["dec3a"], "dec2a": store["cat2"], "dec2b": store["dec2a"],
                "dec1a": store["cat1"], "dec1b": store["dec1a"], "head": store["dec1b"]}[name]

    def forward(self, x: torch.Tensor) -> torch.Tensor:
        """x: [2][B][H][W] (rho, damping-level map).  Returns [1][B][H][W]."""
        L, st, a, b = _nn(), self._st(), self.a, self.base
        a["x"].copy_(x)
        pools = {"enc1b": "p1", "enc2b": "p2", "enc3b": "p3"}
        ups = {"botb": ("cat3", 8 * b), "dec3b": ("cat2", 4 * b), "dec2b": ("cat1", 2 * b)}
        for name, ci, co, k in self.layers:
            y = self._view(a, name)
            self._conv_fwd(name, ci, co, k, self._in_of(name, a), y, name != "head")
            if name in pools:
                _ck(L.nn_pool2(_p(y), co * self.B, y.shape[2], y.shape[3], _p(a[pools[name]]), st), "pool")
            if name in ups:
                cat, n = ups[name]
                _ck(L.nn_up2(_p(y), n * self.B, y.shape[2], y.shape[3], _p(a[cat][:n]), st), "up")
        return a["head"]

    def backward(self, dout: torch.Tensor) -> None:
        """dout: dL/d(output) [1][B][H][W]; fills the parameter gradients."""
        L, st, a, g, b = _nn(), self._st(), self.a, self.g, self.base
        for t in g.values():
            _ck(L.nn_zero(_p(t), t.numel(), st), "zero")
        g["head"].copy_(dout)
        pools = {"enc1b": "p1", "enc2b": "p2", "enc3b": "p3"}
        ups = {"botb": ("cat3", 8 * b), "dec3b": ("cat2", 4 * b), "dec2b": ("cat1", 2 * b)}
        for name, ci, co, k in reversed(self.layers):
            y, dy = self._view(a, name), self._view(g, name)
            if name in ups:  # the upsampled copy of y feeds the next decoder level
                cat, n = ups[name]
                _ck(L.nn_up2_bwd_add(_p(g[cat][:n]), n * self.B, y.shape[2], y.shape[3], _p(dy), st), "up_bwd")
            if name in pools:
                _ck(L.nn_pool2_bwd_add(_p(g[pools[name]]), co * self.B, y.shape[2], y.shape[3], _p(dy), st),
                    "pool_bwd")
            x = self._in_of(name, a)
            dx = None if name == "enc1a" else self._in_of(name, g)
            self._conv_bwd(name, ci, co, k, x, y, dy, dx, name != "head")

    def train_step(self, x: torch.Tensor, target: torch.Tensor, lr: float = 1e-3) -> torch.Tensor:
        """One Adam step on the MSE between the network output and target ([1][B][H][W])."""
        L, st = _nn(), self._st()
        out = self.forward(x)
        dout = self.g["head"]
        _ck(L.nn_mse(_p(out), _p(target), out.numel(), _p(dout), _p(self.loss), st), "mse")
        d = dout.clone()
        self.backward(d)
        self.step += 1
        for key, t in self._params():
            grad = self.gw[key[:-2]] if key.endswith(".w") else self.gb[key[:-2]]
            _ck(L.nn_adam(_p(t), _p(grad), _p(self.m[key]), _p(self.v[key]), t.numel(), lr, 0.9, 0.999, 1e-8,
                          self.step, st), "adam")
        return self.loss

    def grads(self) -> dict:
        """Parameter gradients in the oracle's shapes (numpy, FP64)."""
        out = {}
        for n, ci, co, k in self.layers:
            out[n + ".w"] = self.gw[n].double().cpu().numpy().reshape(co, ci, k, k)
            out[n + ".b"] = self.gb[n].double().cpu().numpy()
        return out
