"""ctypes binding of ``libfdtd_gb300.so`` (C ABI in ``include/fdtd.h``).

Argument marshalling only: every step of the path runs in the library's CUDA
kernels.  PyTorch provides the device memory (the workspace, rho, the
gradient) and the CUDA stream.  There is no fallback: if the library has not
been built, loading it raises.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libfdtd_gb300.so")

STATUS = {0: "FDTD_OK", 1: "FDTD_EINVAL", 2: "FDTD_ENOMEM", 3: "FDTD_ECUDA", 4: "FDTD_ESTATE",
          5: "FDTD_EUNSTABLE", 6: "FDTD_ETIMEOUT", 7: "FDTD_ERANGE"}
SNAP = {"f32": 0, "bf16": 1, "f16": 2}
ACC = {"f64": 0, "comp_f32": 1}

# Every symbol the header declares (checked by the CPU test-suite).
EXPORTS = ["fdtd_workspace_bytes", "fdtd_create", "fdtd_set_design", "fdtd_set_damping",
           "fdtd_forward", "fdtd_adjoint", "fdtd_gradient", "fdtd_gap_history", "fdtd_sync",
           "fdtd_run_host", "fdtd_get_info", "fdtd_status_string", "fdtd_destroy",
           "fdtd_gradient_static", "fdtd_gap_spectrum", "fdtd_ascent_step", "fdtd_mma_asymptotes", "fdtd_mma_solve",
           "fdtd_mirror_average", "fdtd_fix_design", "fdtd_grayness", "fdtd_threshold", "fdtd_set_graphs",
           "fdtd_set_l2_residency", "fdtd_set_sensitivity_terms", "fdtd_set_stability_guard",
           "fdtd_set_steps_per_launch", "fdtd_selftest_bounded_wait", "fdtd_set_filter_width",
           "fdtd_set_wavefront"]


TERM_PSI, TERM_EPS, TERM_SIGMA, TERM_ALL = 1, 2, 4, 7


class FdtdError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__("%s: %s (%s)" % (where, STATUS.get(status, status), _status_string(status)))


class FdtdConfig(C.Structure):
    _fields_ = [
        ("ndim", C.c_int), ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
        ("dx", C.c_double), ("courant", C.c_double),
        ("npml", C.c_int), ("pml_m", C.c_double), ("pml_sigma_factor", C.c_double),
        ("pml_kappa_max", C.c_double), ("pml_alpha_max", C.c_double),
        ("eps_inf", C.c_double), ("omega_p", C.c_double), ("gamma_p", C.c_double),
        ("eps_s", C.c_double), ("psi_s_ratio", C.c_double), ("eps_g", C.c_double),
        ("design_lo", C.c_int * 3), ("design_hi", C.c_int * 3),
        ("gap_lo", C.c_int * 3), ("gap_hi", C.c_int * 3),
        ("src_lo", C.c_int * 3), ("src_hi", C.c_int * 3),
        ("nbands", C.c_int), ("f0", C.c_double * 2), ("tau", C.c_double), ("t0", C.c_double),
        ("src_amp", C.c_double), ("nsteps", C.c_int),
        ("filter_radius", C.c_int), ("filter_sigma", C.c_double),
        ("sigma_form", C.c_int), ("sub_eps", C.c_double), ("sub_hi", C.c_int),
        ("real_bytes", C.c_int), ("snapshot_every", C.c_int), ("snapshot_dtype", C.c_int),
        ("accum_kind", C.c_int), ("src_comp", C.c_int),
        ("waveform", C.c_int), ("bandwidth", C.c_double), ("lobes", C.c_int), ("pol", C.c_int),
        ("tfsf", C.c_int), ("tf_lo", C.c_int * 3), ("tf_hi", C.c_int * 3),
    ]


class FdtdInfo(C.Structure):
    _fields_ = [("dt", C.c_double), ("n_cells", C.c_longlong), ("n_design", C.c_longlong),
                ("n_gap", C.c_longlong), ("launches", C.c_longlong), ("cell_updates", C.c_longlong),
                ("workspace_bytes", C.c_size_t), ("step_blocks", C.c_longlong),
                ("vector_blocks", C.c_longlong)]


_lock = threading.Lock()
_lib = None


def load():
    """Open the library (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libfdtd_gb300.so is not built (%s); run __graft_entry__.build()" % LIB_PATH)
        L = C.CDLL(LIB_PATH)
        P = C.c_void_p
        cfgp = C.POINTER(FdtdConfig)
        sig = {
            "fdtd_workspace_bytes": [cfgp, C.POINTER(C.c_size_t)],
            "fdtd_create": [cfgp, P, C.c_size_t, P, C.POINTER(P)],
            "fdtd_set_design": [P, P, C.c_size_t],
            "fdtd_set_damping": [P, C.c_double, C.c_double],
            "fdtd_forward": [P, P],
            "fdtd_adjoint": [P],
            "fdtd_gradient": [P, P, C.c_size_t],
            "fdtd_gradient_static": [P, P, C.c_size_t],
            "fdtd_ascent_step": [P, P, P, C.c_size_t, C.c_double],
            "fdtd_gap_spectrum": [P, P, C.c_int, P],
            "fdtd_mma_asymptotes": [P, P, P, P, C.c_size_t, C.c_int, P],
            "fdtd_mma_solve": [P, P, P, C.c_size_t, C.c_double, C.c_double, C.c_double, P, P],
            "fdtd_mirror_average": [P, P, C.c_size_t, C.c_int, C.c_int],
            "fdtd_fix_design": [P, P, P, P, C.c_size_t, C.c_double],
            "fdtd_grayness": [P, P],
            "fdtd_set_graphs": [P, C.c_int],
            "fdtd_set_l2_residency": [P, C.c_double],
            "fdtd_set_sensitivity_terms": [P, C.c_int],
            "fdtd_set_stability_guard": [P, C.c_int, C.c_double],
            "fdtd_set_steps_per_launch": [P, C.c_int],
            "fdtd_set_wavefront": [P, C.c_int],
            "fdtd_set_filter_width": [P, C.c_double],
            "fdtd_selftest_bounded_wait": [P, C.c_longlong, P],
            "fdtd_threshold": [P, P, C.c_size_t, C.c_double],
            "fdtd_gap_history": [P, P, C.c_size_t],
            "fdtd_sync": [P],
            "fdtd_run_host": [P, P, C.c_size_t, P, P],
            "fdtd_get_info": [P, C.POINTER(FdtdInfo)],
        }
        for name, args in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = C.c_int
        L.fdtd_status_string.argtypes = [C.c_int]
        L.fdtd_status_string.restype = C.c_char_p
        L.fdtd_destroy.argtypes = [P]
        L.fdtd_destroy.restype = None
        _lib = L
        return L


def _status_string(s: int) -> str:
    try:
        return load().fdtd_status_string(int(s)).decode()
    except Exception:  # library missing while formatting an error
        return "?"


def _check(rc: int, where: str) -> None:
    if rc != 0:
        raise FdtdError(rc, where)


def config(w: dict) -> FdtdConfig:
    """Fill the C struct from a workload dict (see ``inputs``)."""
    c = FdtdConfig()
    for name, ctype in FdtdConfig._fields_:
        if name == "real_bytes":
            c.real_bytes = 8 if w.get("real", "f64") == "f64" else 4
            continue
        if name == "snapshot_dtype":
            c.snapshot_dtype = SNAP[w.get("snapshot_dtype", "f32")]
            continue
        if name == "accum_kind":
            c.accum_kind = ACC[w.get("accum", "f64")]
            continue
        v = w[name] if name in w else {"snapshot_every": 0, "src_comp": 2, "waveform": 0, "bandwidth": 0.0,
                                       "lobes": 0, "pol": 0, "tfsf": 0, "tf_lo": (0, 0, 0),
                                       "tf_hi": (0, 0, 0)}.get(name)
        if name == "f0":
            c.f0[0], c.f0[1] = float(v[0]), float(v[1])
        elif isinstance(getattr(c, name), C.Array):
            arr = getattr(c, name)
            for a in range(3):
                arr[a] = int(v[a])
        elif ctype is C.c_int:
            setattr(c, name, int(v))
        else:
            setattr(c, name, float(v))
    return c


def workspace_bytes(w: dict) -> int:
    n = C.c_size_t(0)
    cfg = config(w)
    _check(load().fdtd_workspace_bytes(C.byref(cfg), C.byref(n)), "fdtd_workspace_bytes")
    return int(n.value)


class Solver:
    """One context: a caller-owned workspace on one device and one stream."""

    def __init__(self, w: dict, device=None, stream=None):
        import torch
        self.torch = torch
        self.w = dict(w)
        self.lib = load()
        self.cfg = config(w)
        self.device = torch.device(device if device is not None else "cuda")
        self.real = torch.float64 if self.cfg.real_bytes == 8 else torch.float32
        nbytes = workspace_bytes(w)
        self.ws = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        ctx = C.c_void_p()
        _check(self.lib.fdtd_create(C.byref(self.cfg), C.c_void_p(self.ws.data_ptr()), nbytes,
                                    C.c_void_p(self.stream.cuda_stream), C.byref(ctx)), "fdtd_create")
        self.ctx = ctx
        inf = self.info()
        self.n_design = int(inf.n_design)
        self.n_gap = int(inf.n_gap)
        self.dt = float(inf.dt)
        self._W = torch.zeros(1, dtype=torch.float64, device=self.device)
        # Counts calls that change the solver's state (set_design,
        # set_damping, forward); the autograd wrapper compares it to find out
        # whether the solver still holds the forward run it needs.
        self.generation = 0

    def close(self) -> None:
        if getattr(self, "ctx", None):
            self.lib.fdtd_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self) -> FdtdInfo:
        i = FdtdInfo()
        _check(self.lib.fdtd_get_info(self.ctx, C.byref(i)), "fdtd_get_info")
        return i

    def set_design(self, rho) -> None:
        t = self.torch
        r = rho if isinstance(rho, t.Tensor) else t.as_tensor(np.asarray(rho))
        r = r.to(device=self.device, dtype=self.real).contiguous().reshape(-1)
        if r.numel() != self.n_design:
            raise ValueError("rho has %d entries, design box has %d" % (r.numel(), self.n_design))
        self._rho = r
        self.generation += 1
        _check(self.lib.fdtd_set_design(self.ctx, C.c_void_p(r.data_ptr()), r.numel()), "fdtd_set_design")

    def set_damping(self, sigma_max: float = 0.0, gamma_scale: float = 1.0) -> None:
        self.generation += 1
        _check(self.lib.fdtd_set_damping(self.ctx, float(sigma_max), float(gamma_scale)), "fdtd_set_damping")

    def forward(self, out=None):
        out = self._W if out is None else out
        self.generation += 1
        _check(self.lib.fdtd_forward(self.ctx, C.c_void_p(out.data_ptr())), "fdtd_forward")
        return out

    def adjoint(self) -> None:
        _check(self.lib.fdtd_adjoint(self.ctx), "fdtd_adjoint")

    def gradient(self, out=None):
        t = self.torch
        if out is None:
            out = t.empty(self.n_design, dtype=t.float64, device=self.device)
        _check(self.lib.fdtd_gradient(self.ctx, C.c_void_p(out.data_ptr()), out.numel()), "fdtd_gradient")
        return out

    def gradient_static(self, out=None):
        """fdtd_gradient_static: the gradient with the library's fixed device
        scratch instead of the workspace (no allocation at call time)."""
        t = self.torch
        if out is None:
            out = t.empty(self.n_design, dtype=t.float64, device=self.device)
        _check(self.lib.fdtd_gradient_static(self.ctx, C.c_void_p(out.data_ptr()), out.numel()),
               "fdtd_gradient_static")
        return out

    def ascent_step(self, rho, grad, move: float) -> None:
        """rho <- clip(rho + move * grad / max|grad|, 0, 1) in place (device tensors)."""
        _check(self.lib.fdtd_ascent_step(self.ctx, C.c_void_p(rho.data_ptr()), C.c_void_p(grad.data_ptr()),
                                         rho.numel(), float(move)), "fdtd_ascent_step")

    def gap_spectrum(self, freqs):
        """Spectrum of the gap field of the last forward run at ``freqs`` (Hz):
        complex128 tensor (nf, M_g) in 2D, (nf, 3, M_g) in 3D."""
        t = self.torch
        f = t.as_tensor(freqs, dtype=t.float64).to(self.device).contiguous().reshape(-1)
        nc = 3 if self.cfg.ndim == 3 else 1
        out = t.empty(f.numel() * nc * self.n_gap * 2, dtype=t.float64, device=self.device)
        _check(self.lib.fdtd_gap_spectrum(self.ctx, C.c_void_p(f.data_ptr()), f.numel(),
                                          C.c_void_p(out.data_ptr())), "fdtd_gap_spectrum")
        z = t.view_as_complex(out.reshape(-1, 2))
        return z.reshape((f.numel(), 3, self.n_gap) if nc == 3 else (f.numel(), self.n_gap))

    def set_l2_residency(self, fraction: float) -> None:
        """Keep ``fraction`` of the ping-pong state persisting in L2 (2D E_z mode; 0: off)."""
        _check(self.lib.fdtd_set_l2_residency(self.ctx, float(fraction)), "fdtd_set_l2_residency")

    def set_sensitivity_terms(self, terms: int) -> None:
        """Eq. (25) terms the adjoint accumulates: an OR of TERM_PSI, TERM_EPS,
        TERM_SIGMA (default TERM_ALL, the gradient of W~)."""
        _check(self.lib.fdtd_set_sensitivity_terms(self.ctx, int(terms)), "fdtd_set_sensitivity_terms")

    def set_stability_guard(self, every: int = 256, max_abs: float = 0.0) -> None:
        """Check the forward state every ``every`` steps (0: off) for words that
        are not finite or exceed ``max_abs`` (0: the automatic bound)."""
        _check(self.lib.fdtd_set_stability_guard(self.ctx, int(every), float(max_abs)), "fdtd_set_stability_guard")

    def set_filter_width(self, sigma: float) -> None:
        """New width (cells) of the Gaussian design filter; the design has to be set again."""
        self.generation += 1
        _check(self.lib.fdtd_set_filter_width(self.ctx, float(sigma)), "fdtd_set_filter_width")
        self.w["filter_sigma"] = float(sigma)

    def set_steps_per_launch(self, steps: int) -> None:
        """Time steps per launch (1: one launch per step): in-plane 2D mode, a
        cooperative launch with grid barriers; 2D E_z, temporal blocking on
        square tiles (16 to 32 nodes a side) with a halo in shared memory (up
        to 8 steps, 4 in FP64)."""
        _check(self.lib.fdtd_set_steps_per_launch(self.ctx, int(steps)), "fdtd_set_steps_per_launch")

    def set_wavefront(self, steps: int) -> None:
        """3D: time steps per wavefront launch (0: two launches per step, the H
        then the E half step over the whole grid); results are bit-identical."""
        _check(self.lib.fdtd_set_wavefront(self.ctx, int(steps)), "fdtd_set_wavefront")

    def set_graphs(self, mode: int) -> None:
        """0: plain launches, 1: replay CUDA graphs of whole passes, 2: automatic by grid size."""
        _check(self.lib.fdtd_set_graphs(self.ctx, int(mode)), "fdtd_set_graphs")

    def mirror_average(self, vec, axis: int) -> None:
        """Make ``vec`` (rho in the field precision, or an FP64 gradient)
        mirror-symmetric across the design box's mid-plane normal to ``axis``."""
        _check(self.lib.fdtd_mirror_average(self.ctx, C.c_void_p(vec.data_ptr()), vec.numel(),
                                            vec.element_size(), int(axis)), "fdtd_mirror_average")

    def fix_design(self, mask, rho=None, grad=None, value: float = 1.0) -> None:
        """rho = value and grad = 0 where the uint8 device ``mask`` is set."""
        _check(self.lib.fdtd_fix_design(self.ctx, C.c_void_p(rho.data_ptr() if rho is not None else None),
                                        C.c_void_p(grad.data_ptr() if grad is not None else None),
                                        C.c_void_p(mask.data_ptr()), mask.numel(), float(value)),
               "fdtd_fix_design")

    def mma_state(self):
        """Device state of the moving-asymptote update (4 M_d doubles)."""
        t = self.torch
        return t.zeros(4 * self.n_design, dtype=t.float64, device=self.device)

    def mma_asymptotes(self, rho, grad, state, k: int):
        """Outer MMA iteration k: asymptotes from rho = x^k and the history in
        ``state``.  Returns a device tensor (sum |g|, squared optimality residual)."""
        t = self.torch
        sums = t.empty(2, dtype=t.float64, device=self.device)
        _check(self.lib.fdtd_mma_asymptotes(self.ctx, C.c_void_p(rho.data_ptr()), C.c_void_p(grad.data_ptr()),
                                            C.c_void_p(state.data_ptr()), rho.numel(), int(k),
                                            C.c_void_p(sums.data_ptr())), "fdtd_mma_asymptotes")
        return sums

    def mma_solve(self, state, grad, scale: float, raa0: float, move: float, out):
        """Subproblem minimiser into ``out`` (field precision).  Returns a device
        tensor (approximation change f~(y) - f(x), GCMMA term d(y))."""
        t = self.torch
        sums = t.empty(2, dtype=t.float64, device=self.device)
        _check(self.lib.fdtd_mma_solve(self.ctx, C.c_void_p(state.data_ptr()), C.c_void_p(grad.data_ptr()),
                                       out.numel(), float(scale), float(raa0), float(move),
                                       C.c_void_p(out.data_ptr()), C.c_void_p(sums.data_ptr())), "fdtd_mma_solve")
        return sums

    def grayness(self):
        """zeta = 4 rho~^T (1 - rho~) / M of the current filtered design (device FP64 scalar)."""
        t = self.torch
        out = t.zeros(1, dtype=t.float64, device=self.device)
        _check(self.lib.fdtd_grayness(self.ctx, C.c_void_p(out.data_ptr())), "fdtd_grayness")
        return out

    def threshold(self, rho, level: float = 0.5) -> None:
        _check(self.lib.fdtd_threshold(self.ctx, C.c_void_p(rho.data_ptr()), rho.numel(), float(level)),
               "fdtd_threshold")

    def gap_history(self):
        """(N+1, M_g) in 2D; (N+1, 3, M_g) in 3D."""
        t = self.torch
        nc = 3 if self.cfg.ndim == 3 else 1
        n = (int(self.cfg.nsteps) + 1) * nc * self.n_gap
        out = t.empty(n, dtype=t.float64, device=self.device)
        _check(self.lib.fdtd_gap_history(self.ctx, C.c_void_p(out.data_ptr()), n), "fdtd_gap_history")
        shape = (int(self.cfg.nsteps) + 1, 3, self.n_gap) if nc == 3 else (int(self.cfg.nsteps) + 1, self.n_gap)
        return out.reshape(shape)

    def sync(self) -> None:
        _check(self.lib.fdtd_sync(self.ctx), "fdtd_sync")

    def run_host(self, rho: np.ndarray):
        """One evaluation from host memory (copies inside the call)."""
        dt = np.float64 if self.cfg.real_bytes == 8 else np.float32
        r = np.ascontiguousarray(np.asarray(rho, dtype=dt).reshape(-1))
        g = np.empty(self.n_design, dtype=np.float64)
        Wv = C.c_double(0.0)
        _check(self.lib.fdtd_run_host(self.ctx, C.c_void_p(r.ctypes.data), r.size, C.byref(Wv),
                                      C.c_void_p(g.ctypes.data)), "fdtd_run_host")
        return Wv.value, g

    def evaluate(self, rho, sigma_max: float = 0.0, gamma_scale: float = 1.0):
        """W~ and dW~/drho on the device (both FP64 tensors)."""
        self.set_design(rho)
        self.set_damping(sigma_max, gamma_scale)
        W = self.forward().clone()
        self.adjoint()
        g = self.gradient()
        return W, g


def selftest_bounded_wait(limit_cycles: int, stream=None) -> int:
    """Run the library's bounded-wait self-test (a wait on a flag nothing
    sets, limited to ``limit_cycles`` clock cycles); returns the status."""
    import torch
    words = torch.zeros(4, dtype=torch.int32, device="cuda")
    st = stream if stream is not None else torch.cuda.current_stream()
    return int(load().fdtd_selftest_bounded_wait(C.c_void_p(words.data_ptr()), int(limit_cycles),
                                                 C.c_void_p(st.cuda_stream)))
