"""Exact discrete reverse mode of the 2D E_z-out-of-plane scheme, by automatic
differentiation of a plain FP64 PyTorch forward on the CPU -- TEST
INFRASTRUCTURE ONLY.

This is a third, independent statement of the forward scheme (the C oracle
is the first, the CUDA path the second): the Yee leapfrog with CPML, the
trapezoidal Drude update of every E_z node solved by Cramer's rule, the
soft line source and the objective W~ of Eq. (24).  Autograd keeps every
intermediate state on its tape and differentiates W~ through all N steps,
which gives the exact gradient of the discrete objective.  The paper's
adjoint (Eq. 20, 25, 27) computed by the C oracle must agree with it to
round-off; that is what the discretisation chosen for the Drude term is
meant to guarantee.  For tiny grids only (the tape holds every step).

Only tests use this module.
"""
from __future__ import annotations

import math

import numpy as np
import torch

C0 = 299792458.0
MU0 = 1.25663706212e-6
EPS0 = 1.0 / (MU0 * C0 * C0)


def _pml(w: dict, n: int, p: float):
    """(b, c, kappa) of the CPML at position p (cell units) of an axis of n nodes."""
    L = w["npml"]
    d = 0.0
    if L > 0:
        if p < L:
            d = L - p
        elif p > (n - 1) - L:
            d = p - ((n - 1) - L)
    if d <= 0.0:
        return 0.0, 0.0, 1.0
    x = d / L
    xm = x ** w["pml_m"]
    sig = w["pml_sigma_factor"] * (w["pml_m"] + 1.0) / (MU0 * C0 * w["dx"]) * xm
    kap = 1.0 + (w["pml_kappa_max"] - 1.0) * xm
    alp = w["pml_alpha_max"] * (1.0 - x)
    dt = w["courant"] * w["dx"] / C0
    b = math.exp(-(sig / kap + alp) * dt / EPS0)
    c = sig / (sig * kap + kap * kap * alp) * (b - 1.0) if sig > 0 else 0.0
    return b, c, kap


def _signal(w: dict, t: float) -> float:
    """Gaussian-envelope carrier(s) (the workloads' excitation)."""
    u = t - w["t0"]
    s = sum(math.sin(2.0 * math.pi * w["f0"][b] * u) for b in range(w["nbands"]))
    return math.exp(-(u / w["tau"]) ** 2) * s


def objective_tm(w: dict, rho: torch.Tensor, sigma_max: float = 0.0, gamma_scale: float = 1.0) -> torch.Tensor:
    """W~ of a 2D TM_z workload (no filter, Gaussian excitation) as a
    differentiable function of the design rho (FP64 tensor, design box,
    x fastest)."""
    assert w["ndim"] == 2 and w.get("pol", 0) == 0 and w.get("filter_radius", 0) == 0
    assert w.get("waveform", 0) == 0 and not w.get("periodic_x", 0)
    nx, ny, N, dx = w["nx"], w["ny"], w["nsteps"], w["dx"]
    dt = w["courant"] * dx / C0
    f64 = dict(dtype=torch.float64)
    # material per node: background, design (Eq. 5 from rho), gap (eps_g, no Drude)
    psi_m = w["omega_p"] ** 2
    psi_s = w["psi_s_ratio"] * psi_m
    dl, dh, gl, gh = w["design_lo"], w["design_hi"], w["gap_lo"], w["gap_hi"]
    r = rho.reshape(dh[1] - dl[1], dh[0] - dl[0])
    eps = torch.full((ny, nx), w["eps_s"], **f64)
    psi = torch.zeros((ny, nx), **f64)
    sig = torch.zeros((ny, nx), **f64)
    sform = 4.0 if w.get("sigma_form", 0) else 1.0
    eps_d = w["eps_s"] + r * (w["eps_inf"] - w["eps_s"])
    psi_d = psi_s + r * (psi_m - psi_s)
    sig_d = r * (1.0 - r) * sigma_max * sform
    mask = torch.zeros((ny, nx), dtype=torch.bool)
    mask[dl[1]:dh[1], dl[0]:dh[0]] = True
    gmask = torch.zeros((ny, nx), dtype=torch.bool)
    gmask[gl[1]:gh[1], gl[0]:gh[0]] = True
    pad = lambda t: torch.nn.functional.pad(t, (dl[0], nx - dh[0], dl[1], ny - dh[1]))
    dmask = mask & ~gmask
    eps = torch.where(dmask, pad(eps_d), eps)
    psi = torch.where(dmask, pad(psi_d), psi)
    sig = torch.where(dmask, pad(sig_d), sig)
    eps = torch.where(gmask, torch.full_like(eps, w["eps_g"]), eps)
    gam = w["gamma_p"] * gamma_scale
    # CPML tables: E at nodes, H at half positions
    ex = torch.tensor([_pml(w, nx, i) for i in range(nx)], **f64)
    hx = torch.tensor([_pml(w, nx, i + 0.5) for i in range(nx)], **f64)
    ey = torch.tensor([_pml(w, ny, j) for j in range(ny)], **f64)
    hy = torch.tensor([_pml(w, ny, j + 0.5) for j in range(ny)], **f64)
    # trapezoidal node system (Cramer): a11 E' + a12 J' = b1, a21 E' + a22 J' = b2
    a11 = EPS0 * eps / dt + 0.5 * sig
    a12 = 0.5
    a21 = -0.5 * EPS0 * psi
    a22 = 1.0 / dt + 0.5 * gam
    det = a11 * a22 - a12 * a21
    src = torch.zeros((ny, nx), dtype=torch.bool)
    sl, sh = w["src_lo"], w["src_hi"]
    src[sl[1]:sh[1], sl[0]:sh[0]] = True
    J0 = w["src_amp"] * EPS0 * C0 / dx
    interior = torch.zeros((ny, nx), dtype=torch.bool)
    interior[1:ny - 1, 1:nx - 1] = True
    Ez = torch.zeros((ny, nx), **f64)
    Jz = torch.zeros((ny, nx), **f64)
    Hx = torch.zeros((ny, nx), **f64)
    Hy = torch.zeros((ny, nx), **f64)
    pexy = torch.zeros((ny, nx), **f64)  # psi of dHx/dy in the E update
    pexx = torch.zeros((ny, nx), **f64)  # psi of dHy/dx
    phxy = torch.zeros((ny, nx), **f64)  # psi of dEz/dy in the Hx update
    phyx = torch.zeros((ny, nx), **f64)  # psi of dEz/dx in the Hy update
    ch = dt / MU0
    W = torch.zeros((), **f64)
    coefW = 0.5 * w["eps_g"] * dt * dx * dx
    for t in range(N + 1):
        W = W + coefW * torch.sum(Ez[gmask] ** 2)
        if t == N:
            break
        # H: mu0 dH/dt = -curl E (forward differences); Hx on rows j < ny-1, Hy on columns i < nx-1
        dEy = torch.zeros_like(Ez)
        dEy[:-1] = (Ez[1:] - Ez[:-1]) / dx
        dEx = torch.zeros_like(Ez)
        dEx[:, :-1] = (Ez[:, 1:] - Ez[:, :-1]) / dx
        phxy = hy[:, 0:1] * phxy + hy[:, 1:2] * dEy
        phyx = hx[None, :, 0] * phyx + hx[None, :, 1] * dEx
        rowm = torch.zeros((ny, 1), **f64)
        rowm[:-1] = 1.0
        colm = torch.zeros((1, nx), **f64)
        colm[0, :-1] = 1.0
        phxy = phxy * rowm
        phyx = phyx * colm
        Hx = Hx - rowm * ch * (dEy / hy[:, 2:3] + phxy)
        Hy = Hy + colm * ch * (dEx / hx[None, :, 2] + phyx)
        # E, J: trapezoidal Drude at interior nodes (backward differences)
        dHy = torch.zeros_like(Ez)
        dHy[:, 1:] = (Hy[:, 1:] - Hy[:, :-1]) / dx
        dHx = torch.zeros_like(Ez)
        dHx[1:] = (Hx[1:] - Hx[:-1]) / dx
        pexx = torch.where(interior, ex[None, :, 0] * pexx + ex[None, :, 1] * dHy, pexx)
        pexy = torch.where(interior, ey[:, 0:1] * pexy + ey[:, 1:2] * dHx, pexy)
        curl = dHy / ex[None, :, 2] + pexx - dHx / ey[:, 2:3] - pexy
        js = torch.where(src, torch.full_like(Ez, J0 * _signal(w, (t + 0.5) * dt)), torch.zeros_like(Ez))
        b1 = (EPS0 * eps / dt - 0.5 * sig) * Ez - 0.5 * Jz + curl - js
        b2 = (1.0 / dt - 0.5 * gam) * Jz + 0.5 * EPS0 * psi * Ez
        En = (b1 * a22 - a12 * b2) / det
        Jn = (a11 * b2 - a21 * b1) / det
        Ez = torch.where(interior, En, Ez)
        Jz = torch.where(interior, Jn, Jz)
    return W


def gradient_tm(w: dict, rho, sigma_max: float = 0.0, gamma_scale: float = 1.0):
    """(W~, dW~/drho) by reverse-mode differentiation through the whole run."""
    r = torch.tensor(np.asarray(rho, dtype=np.float64).reshape(-1), requires_grad=True)
    W = objective_tm(w, r, sigma_max, gamma_scale)
    W.backward()
    g = r.grad.numpy().copy()
    gap = np.zeros((w["design_hi"][1] - w["design_lo"][1], w["design_hi"][0] - w["design_lo"][0]), dtype=bool)
    gap[w["gap_lo"][1] - w["design_lo"][1]:w["gap_hi"][1] - w["design_lo"][1],
        w["gap_lo"][0] - w["design_lo"][0]:w["gap_hi"][0] - w["design_lo"][0]] = True
    assert np.all(g.reshape(gap.shape)[gap] == 0.0)
    return float(W.item()), g
