"""ctypes front end of the FP64 CPU oracle (``fdtd_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg use it to check and time the CUDA path.  It
imports nothing from the CUDA package; it takes the plain workload dicts of
``paper_2203_01462_gb300.inputs`` and fills its own C struct.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

C0 = 299792458.0  # speed of light in vacuum, m/s
_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fdtd_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None


class OrConfig(C.Structure):
    _fields_ = [
        ("ndim", C.c_int), ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
        ("dx", C.c_double), ("courant", C.c_double),
        ("npml", C.c_int), ("pml_m", C.c_double), ("pml_sigma_factor", C.c_double),
        ("pml_kappa_max", C.c_double), ("pml_alpha_max", C.c_double),
        ("periodic_x", C.c_int),
        ("eps_inf", C.c_double), ("omega_p", C.c_double), ("gamma_p", C.c_double),
        ("eps_s", C.c_double), ("psi_s_ratio", C.c_double), ("eps_g", C.c_double),
        ("design_lo", C.c_int * 3), ("design_hi", C.c_int * 3),
        ("gap_lo", C.c_int * 3), ("gap_hi", C.c_int * 3),
        ("src_lo", C.c_int * 3), ("src_hi", C.c_int * 3),
        ("nbands", C.c_int), ("f0", C.c_double * 2), ("tau", C.c_double), ("t0", C.c_double),
        ("src_amp", C.c_double), ("nsteps", C.c_int),
        ("filter_radius", C.c_int), ("filter_sigma", C.c_double),
        ("sigma_form", C.c_int), ("sub_eps", C.c_double), ("sub_hi", C.c_int),
        ("src_comp", C.c_int), ("waveform", C.c_int), ("bandwidth", C.c_double), ("lobes", C.c_int),
        ("pol", C.c_int), ("tfsf", C.c_int), ("tf_lo", C.c_int * 3), ("tf_hi", C.c_int * 3),
    ]

_DEFAULTS = {"src_comp": 2, "waveform": 0, "bandwidth": 0.0, "lobes": 0, "pol": 0, "tfsf": 0,
             "tf_lo": (0, 0, 0), "tf_hi": (0, 0, 0)}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP64, -O2, OpenMP)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-std=c11",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            dp = C.POINTER(C.c_double)
            L.or_forward.argtypes = [C.POINTER(OrConfig), dp, C.c_double, C.c_double, dp, dp, dp,
                                     C.POINTER(C.c_int), C.c_int, dp, dp]
            L.or_gradient.argtypes = [C.POINTER(OrConfig), dp, C.c_double, C.c_double, dp, dp,
                                      dp, dp, dp]
            L.or_filter.argtypes = [C.POINTER(OrConfig), dp, dp]
            L.or_filter_T.argtypes = [C.POINTER(OrConfig), dp, dp]
            L.or_material.argtypes = [C.POINTER(OrConfig), C.c_double, C.c_double, dp, dp, dp]
            L.or_signal_samples.argtypes = [C.POINTER(OrConfig), dp, C.c_int, dp]
            L.or_sizes.argtypes = [C.POINTER(OrConfig), C.POINTER(C.c_long), C.POINTER(C.c_long)]
            L.or_free_design.argtypes = [C.POINTER(OrConfig)]
            L.or_free_design.restype = C.c_long
            L.or_tfsf_incident.argtypes = [C.POINTER(OrConfig), C.c_double, C.POINTER(C.c_int), C.c_int, dp, dp]
            L.or_set_threads.argtypes = [C.c_int]
            L.or_get_threads.restype = C.c_int
            _lib = L
    return _lib


def set_threads(n: int) -> None:
    lib().or_set_threads(int(n))


def threads() -> int:
    return lib().or_get_threads()


def config(w: dict) -> OrConfig:
    c = OrConfig()
    for name, ctype in OrConfig._fields_:
        v = w.get(name, _DEFAULTS.get(name))
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


def _dptr(a: np.ndarray | None):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _sizes(w: dict) -> tuple[int, int]:
    M, G = C.c_long(0), C.c_long(0)
    cfg = config(w)
    lib().or_sizes(C.byref(cfg), C.byref(M), C.byref(G))
    return int(M.value), int(G.value)


def free_design(w: dict) -> int:
    """Design variables outside the gap (per Yee edge in the in-plane 2D mode)."""
    cfg = config(w)
    return int(lib().or_free_design(C.byref(cfg)))


def forward(w: dict, rho: np.ndarray, sigma_max: float = 0.0, gamma_scale: float = 1.0,
            record_gap: bool = False, record_design: bool = False, probes=None,
            energy: bool = False) -> dict:
    """Forward solve; returns W and whatever histories were asked for.

    2D: gap_hist (N+1, M_g), design_hist (N+1, M_d), probes (i, j) of Ez
    (E in plane: of the E_x edge (i+1/2, j); gap and design values per edge).
    3D: gap_hist (N+1, 3, M_g), design_hist (N+1, 3, M_d) with components
    x, y, z, probes (i, j, k, component)."""
    M, G = _sizes(w)
    N = int(w["nsteps"])
    nc = 3 if w["ndim"] == 3 else 1
    rho = np.ascontiguousarray(rho, dtype=np.float64).reshape(-1)
    assert rho.size == M
    cfg = config(w)
    Wout = C.c_double(0.0)
    gshape = (N + 1, 3, G) if nc == 3 else (N + 1, G)
    dshape = (N + 1, 3, M) if nc == 3 else (N + 1, M)
    gh = np.zeros(gshape) if record_gap else None
    dh = np.zeros(dshape) if record_design else None
    if probes is not None:
        pr = np.ascontiguousarray(np.asarray(probes, dtype=np.int32).reshape(-1, 4 if nc == 3 else 2))
        ph = np.zeros((N + 1, pr.shape[0]))
        pptr, npr = pr.ctypes.data_as(C.POINTER(C.c_int)), pr.shape[0]
    else:
        ph, pptr, npr = None, None, 0
    en = np.zeros(N) if energy else None
    rc = lib().or_forward(C.byref(cfg), _dptr(rho), float(sigma_max), float(gamma_scale),
                          C.byref(Wout), _dptr(gh), _dptr(dh), pptr, npr, _dptr(ph), _dptr(en))
    if rc != 0:
        raise RuntimeError("oracle forward failed (%d)" % rc)
    return dict(W=Wout.value, gap_hist=gh, design_hist=dh, probe_hist=ph, energy=en)


def objective(w: dict, rho: np.ndarray, sigma_max: float = 0.0, gamma_scale: float = 1.0) -> float:
    return forward(w, rho, sigma_max, gamma_scale)["W"]


def gradient(w: dict, rho: np.ndarray, sigma_max: float = 0.0, gamma_scale: float = 1.0,
             parts: bool = False) -> dict:
    """W~ and dW~/drho via the adjoint run and Eq. (25)/(27)."""
    M, _ = _sizes(w)
    rho = np.ascontiguousarray(rho, dtype=np.float64).reshape(-1)
    assert rho.size == M
    cfg = config(w)
    Wout = C.c_double(0.0)
    g = np.zeros(M)
    gp = np.zeros(M) if parts else None
    ge = np.zeros(M) if parts else None
    gs = np.zeros(M) if parts else None
    rc = lib().or_gradient(C.byref(cfg), _dptr(rho), float(sigma_max), float(gamma_scale),
                           C.byref(Wout), _dptr(g), _dptr(gp), _dptr(ge), _dptr(gs))
    if rc != 0:
        raise RuntimeError("oracle gradient failed (%d)" % rc)
    out = dict(W=Wout.value, grad=g)
    if parts:
        out.update(g_psi=gp, g_eps=ge, g_sig=gs)
    return out


def filt(w: dict, x: np.ndarray, transpose: bool = False) -> np.ndarray:
    M, _ = _sizes(w)
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1)
    assert x.size == M
    out = np.zeros(M)
    cfg = config(w)
    (lib().or_filter_T if transpose else lib().or_filter)(C.byref(cfg), _dptr(x), _dptr(out))
    return out


def signal(w: dict, t: np.ndarray) -> np.ndarray:
    """The excitation g(t) of the workload at times t (s)."""
    c = config(w)
    t = np.ascontiguousarray(t, dtype=np.float64)
    out = np.empty_like(t)
    lib().or_signal_samples(C.byref(c), _dptr(t), t.size, _dptr(out))
    return out


def gap_spectrum(w: dict, gap_hist: np.ndarray, freqs) -> np.ndarray:
    """E(f) = dt sum_n E^n exp(-j 2 pi f n dt) of each recorded gap value
    (the e^{j w t} convention of Sec. 2), from the history of ``forward``:
    (nf, M_g) in 2D, (nf, 3, M_g) in 3D."""
    dt = w["courant"] * w["dx"] / C0
    h = np.asarray(gap_hist, dtype=np.float64)
    n = np.arange(h.shape[0])
    out = []
    for f in np.atleast_1d(np.asarray(freqs, dtype=np.float64)):
        ph = np.exp(-2j * np.pi * f * n * dt)
        out.append(dt * np.tensordot(ph, h, axes=(0, 0)))
    return np.array(out)


def material(w: dict, rho: float, sigma_max: float = 0.0) -> tuple[float, float, float]:
    cfg = config(w)
    e, p, s = C.c_double(), C.c_double(), C.c_double()
    lib().or_material(C.byref(cfg), float(rho), float(sigma_max), C.byref(e), C.byref(p), C.byref(s))
    return e.value, p.value, s.value


def grayness(w: dict, rho: np.ndarray) -> float:
    """zeta = 4 rho~^T (1 - rho~) / M over the design nodes outside the gap
    (Sec. 3.2), rho~ = F(rho)."""
    rt = filt(w, rho).reshape(-1)
    lo, hi, dlo = w["gap_lo"], w["gap_hi"], w["design_lo"]
    shape = tuple(w["design_hi"][a] - w["design_lo"][a] for a in reversed(range(w["ndim"])))
    mask = np.ones(shape, dtype=bool)
    sl = tuple(slice(lo[a] - dlo[a], hi[a] - dlo[a]) for a in reversed(range(w["ndim"])))
    mask[sl] = False
    v = rt[mask.reshape(-1)]
    return float(4.0 * np.sum(v * (1.0 - v)) / v.size)


def tfsf_incident(w: dict, ks, gamma_scale: float = 1.0) -> tuple[np.ndarray, np.ndarray]:
    """The incident plane wave of a 3D workload with ``tfsf``: E_x at the
    node indices ks along z for t = 0..N, shape (N+1, len(ks)), and H_y at
    the same indices for t + 1/2, t = 0..N-1, shape (N, len(ks))."""
    ks = np.ascontiguousarray(np.asarray(ks, dtype=np.int32).reshape(-1))
    N = int(w["nsteps"])
    E = np.zeros((N + 1, ks.size))
    H = np.zeros((max(N, 1), ks.size))
    cfg = config(w)
    rc = lib().or_tfsf_incident(C.byref(cfg), float(gamma_scale), ks.ctypes.data_as(C.POINTER(C.c_int)),
                                int(ks.size), _dptr(E), _dptr(H))
    if rc != 0:
        raise RuntimeError("oracle tfsf_incident failed (%d)" % rc)
    return E, H[:N]
