"""Seeded synthetic workloads shared by the CUDA path, the oracle and the tests.

This module only describes inputs: grid sizes, boxes, material constants,
excitation parameters and seeded design densities.  It holds none of the
method's arithmetic (no update coefficients, no CPML profiles, no source
waveform samples); each implementation derives those itself.

Workload shapes follow the nanoantenna problems of Sec. 4 of the paper (a
square design box with a small observation gap at its centre, a soft current
source on the incident side, absorbing layers around everything) at the
sizes of the benchmark configurations:

* ``cfg_2d_160``: 160 x 160 nodes, dx = 5 nm, S = 0.5, 10-cell CPML, 2000
  steps, FP64; 60 x 60 centred design box, 3 x 3 gap.
* ``cfg_2d_2048``: 2048 x 2048 nodes, dx = 2 nm, 20000 steps, FP32;
  1024 x 1024 design box smoothed by a 5-cell Gaussian filter, snapshots
  every 64 steps.

Material: Drude gold, eps_inf = 1, omega_p = 1.37e16 rad/s, gamma = 1e14 1/s.
Excitation: Gaussian-modulated carrier at 800 nm whose spectral amplitude
falls to one half 100 THz either side of the carrier (600-1000 nm band).
"""
from __future__ import annotations

import copy
import math

import numpy as np

C0 = 299792458.0

GOLD = dict(eps_inf=1.0, omega_p=1.37e16, gamma_p=1.0e14)
SILVER = dict(eps_inf=4.469, omega_p=1.426e16, gamma_p=4.571e13)  # Sec. 2 fit
# Artificial-damping conductivity sigma_max of Eq. (5c) that the paper's sweep
# settles on (Sec. 2.1), S/m.
SIGMA_MAX_PAPER = 5e5


def pulse(center_m: float = 800e-9, half_width_hz: float = 100e12, nbands: int = 1,
          centers_m=None) -> dict:
    """Gaussian envelope exp(-((t-t0)/tau)^2) on carrier(s) at c/center.

    The envelope's spectrum exp(-(pi f tau)^2) drops to one half at
    ``half_width_hz`` from the carrier; t0 = 4 tau starts the pulse from ~0.
    """
    tau = math.sqrt(math.log(2.0)) / (math.pi * half_width_hz)
    cs = list(centers_m) if centers_m is not None else [center_m]
    f0 = [C0 / c for c in cs] + [0.0] * (2 - len(cs))
    return dict(nbands=len(cs), f0=f0, tau=tau, t0=4.0 * tau)


def sinc_hanning(center_m: float = 500e-9, rel_bandwidth: float = 0.2, lobes: int = 4) -> dict:
    """The paper's excitation (Sec. 2, Fig. 1c-d): a sinc truncated after
    ``lobes`` lobes per side, Hanning-smoothed, on a carrier at c/center.
    Its spectrum is a rectangle of width B = rel_bandwidth * f0 with rounded
    edges, i.e. ``rel_bandwidth`` of f0 at half maximum; t0 = lobes / B."""
    f0 = C0 / center_m
    B = rel_bandwidth * f0
    t0 = lobes / B
    return dict(waveform=1, bandwidth=B, lobes=int(lobes), nbands=1, f0=[f0, 0.0], tau=t0, t0=t0)


def _centered_box(n: int, w: int) -> tuple[int, int]:
    lo = (n - w) // 2
    return lo, lo + w


def workload_2d(nx: int, ny: int, *, dx: float, nsteps: int, npml: int = 10,
                design: tuple[int, int] = (60, 60), gap: tuple[int, int] = (3, 3),
                courant: float = 0.5, real: str = "f64", material: dict | None = None,
                filter_radius: int = 0, filter_fwhm: float = 5.0,
                snapshot_every: int = 0, snapshot_dtype: str = "f32",
                accum: str = "f64", src_offset: int = 5, **over) -> dict:
    """A 2D TM_z nanoantenna-shaped workload (E_z out of plane).

    Design and gap boxes are centred; the line source is one row of E_z
    ``src_offset`` nodes inside the lower CPML, spanning the non-CPML x range.
    """
    mat = dict(GOLD if material is None else material)
    dlo_x, dhi_x = _centered_box(nx, design[0])
    dlo_y, dhi_y = _centered_box(ny, design[1])
    glo_x, ghi_x = _centered_box(nx, gap[0])
    glo_y, ghi_y = _centered_box(ny, gap[1])
    w = dict(
        ndim=2, nx=nx, ny=ny, nz=1, dx=dx, courant=courant, npml=npml,
        pml_m=3.0, pml_sigma_factor=0.8, pml_kappa_max=1.0, pml_alpha_max=0.0,
        periodic_x=0,
        eps_s=1.0, psi_s_ratio=0.01, eps_g=1.0,
        design_lo=[dlo_x, dlo_y, 0], design_hi=[dhi_x, dhi_y, 1],
        gap_lo=[glo_x, glo_y, 0], gap_hi=[ghi_x, ghi_y, 1],
        src_lo=[npml, npml + src_offset, 0], src_hi=[nx - npml, npml + src_offset + 1, 1],
        src_amp=1.0, nsteps=nsteps,
        filter_radius=filter_radius,
        filter_sigma=(filter_fwhm / (2.0 * math.sqrt(2.0 * math.log(2.0)))) if filter_radius else 1.0,
        sigma_form=0, sub_eps=1.0, sub_hi=0, src_comp=2,
        real=real, snapshot_every=snapshot_every, snapshot_dtype=snapshot_dtype, accum=accum,
    )
    w.update(mat)
    w.update(pulse())
    w.update(over)
    return w


def workload_2d_inplane(nx: int, ny: int, *, dx: float, nsteps: int, npml: int = 10,
                        design: tuple[int, int] = (60, 60), gap: tuple[int, int] = (4, 4),
                        courant: float = 0.5, real: str = "f64", material: dict | None = None,
                        snapshot_every: int = 0, snapshot_dtype: str = "f32", accum: str = "f64",
                        src_offset: int = 5, **over) -> dict:
    """A 2D workload with E in plane (Ex, Ey, Hz; the paper's 2D "TM" case,
    in which surface plasmons exist).  Design and gap boxes are centred cell
    ranges whose Yee edges carry the design variables; the source is one row
    of E_x edges ``src_offset`` rows inside the lower CPML across the non-CPML
    x range, so it launches an E_x-polarised wave along +y and -y."""
    w = workload_2d(nx, ny, dx=dx, nsteps=nsteps, npml=npml, design=design, gap=gap, courant=courant, real=real,
                    material=material, snapshot_every=snapshot_every, snapshot_dtype=snapshot_dtype, accum=accum,
                    src_offset=src_offset)
    dlo_x, dhi_x = _centered_box(nx - 1, design[0])
    dlo_y, dhi_y = _centered_box(ny - 1, design[1])
    glo_x, ghi_x = _centered_box(nx - 1, gap[0])
    glo_y, ghi_y = _centered_box(ny - 1, gap[1])
    w.update(pol=1, design_lo=[dlo_x, dlo_y, 0], design_hi=[dhi_x, dhi_y, 1],
             gap_lo=[glo_x, glo_y, 0], gap_hi=[ghi_x, ghi_y, 1],
             src_lo=[npml, npml + src_offset, 0], src_hi=[nx - 1 - npml, npml + src_offset + 1, 1])
    w.update(over)
    return w


def cfg_2d_inplane_paper(design_nm: float = 100.0, nsteps: int = 78000, real: str = "f32",
                         snapshot_every: int = 64) -> dict:
    """The geometry of the paper's 2D nanoantennas with E in plane (Sec. 3.2):
    dx = 0.5 nm, a square design box of ``design_nm`` (100 or 200 nm), a
    centred 10 nm gap, 15 absorbing cells placed 30 cells beyond the design
    box, the truncated-sinc excitation of 20 % bandwidth around 413 nm
    (t0 = 27.5 fs; 78 000 steps of 0.83 as cover the pulse and its ring-down)."""
    dx = 0.5e-9
    d = int(round(design_nm * 1e-9 / dx))
    g = int(round(10e-9 / dx))
    n = d + 2 * 30 + 2 * 15 + 1
    w = workload_2d_inplane(n, n, dx=dx, nsteps=nsteps, npml=15, design=(d, d), gap=(g, g), real=real,
                            material=SILVER, src_offset=5, snapshot_every=snapshot_every)
    w.update(sinc_hanning(center_m=413e-9, rel_bandwidth=0.2, lobes=4))
    return w


def cfg_2d_160() -> dict:
    """160^2 FP64 parity workload: full forward + adjoint + gradient."""
    return workload_2d(160, 160, dx=5e-9, nsteps=2000, npml=10, design=(60, 60), gap=(3, 3),
                       real="f64")


def cfg_2d_2048(nsteps: int = 20000) -> dict:
    """2048^2 FP32 workload with a 1024^2 filtered design box, snapshots every 64."""
    return workload_2d(2048, 2048, dx=2e-9, nsteps=nsteps, npml=10, design=(1024, 1024),
                       gap=(3, 3), real="f32", filter_radius=5, filter_fwhm=5.0,
                       snapshot_every=64, snapshot_dtype="f32", accum="f64")


def cfg_2d_316(nsteps: int = 4000) -> dict:
    """Surrogate-loop workload: 256 x 256 design box on a 316^2 grid, dx = 5 nm,
    10-cell CPML, 4000 steps, FP32, full design-box history (1 GB)."""
    return workload_2d(316, 316, dx=5e-9, nsteps=nsteps, npml=10, design=(256, 256), gap=(3, 3), real="f32",
                       snapshot_every=0)


def small_2d(nx: int = 40, ny: int = 36, nsteps: int = 300, real: str = "f64", **kw) -> dict:
    """A small 2D case that spans several GPU tiles with ragged edges."""
    d = kw.pop("design", (16, 14))
    g = kw.pop("gap", (3, 3))
    npml = kw.pop("npml", 6)
    return workload_2d(nx, ny, dx=kw.pop("dx", 5e-9), nsteps=nsteps, npml=npml, design=d, gap=g,
                       real=real, src_offset=kw.pop("src_offset", 2), **kw)


def workload_3d(nx: int, ny: int, nz: int, *, dx: float, nsteps: int, npml: int = 12,
                design: tuple[int, int, int] = (32, 32, 16), gap: tuple[int, int, int] = (4, 4, 4),
                courant: float = 0.5, real: str = "f32", material: dict | None = None,
                source: str = "sheet", src_offset: int = 5, substrate: bool = False,
                snapshot_every: int = 0, snapshot_dtype: str = "f32", accum: str = "f64",
                pulse_kw: dict | None = None, tf_margin: int = 2, **over) -> dict:
    """A 3D nanoantenna-shaped workload: centred design slab and gap.

    source="sheet": a soft E_x current sheet on the plane z = npml + src_offset
    over the non-CPML x-y range (a plane wave along +z, x-polarised).
    source="tfsf": the same x-polarised plane wave along +z, injected by
    total-field / scattered-field: the current of the plane z = npml +
    src_offset drives a 1D column, and the total-field box spans x and y from
    npml + tf_margin to n - 1 - npml - tf_margin and z from two nodes above
    the source plane to nz - 1 - npml - tf_margin.
    source="dipole": a soft E_z current at the centre node of the gap.
    substrate=True: background eps 2.25 below the design slab.
    """
    mat = dict(GOLD if material is None else material)
    d_lo = [(n - w_) // 2 for n, w_ in zip((nx, ny, nz), design)]
    g_lo = [(n - w_) // 2 for n, w_ in zip((nx, ny, nz), gap)]
    w = dict(
        ndim=3, nx=nx, ny=ny, nz=nz, dx=dx, courant=courant, npml=npml,
        pml_m=3.0, pml_sigma_factor=0.8, pml_kappa_max=1.0, pml_alpha_max=0.0,
        periodic_x=0, eps_s=1.0, psi_s_ratio=0.01, eps_g=1.0,
        design_lo=d_lo, design_hi=[l + w_ for l, w_ in zip(d_lo, design)],
        gap_lo=g_lo, gap_hi=[l + w_ for l, w_ in zip(g_lo, gap)],
        src_amp=1.0, nsteps=nsteps, filter_radius=0, filter_sigma=1.0, sigma_form=0,
        sub_eps=2.25 if substrate else 1.0, sub_hi=d_lo[2] if substrate else 0,
        real=real, snapshot_every=snapshot_every, snapshot_dtype=snapshot_dtype, accum=accum,
    )
    if source in ("sheet", "tfsf"):
        zs = npml + src_offset
        w.update(src_lo=[npml, npml, zs], src_hi=[nx - npml, ny - npml, zs + 1], src_comp=0)
        if source == "tfsf":
            m = tf_margin
            w.update(tfsf=1, tf_lo=[npml + m, npml + m, zs + 2],
                     tf_hi=[nx - 1 - npml - m, ny - 1 - npml - m, nz - 1 - npml - m])
    elif source == "dipole":
        c = [(l + h) // 2 for l, h in zip(w["gap_lo"], w["gap_hi"])]
        w.update(src_lo=c, src_hi=[x + 1 for x in c], src_comp=2)
    else:
        raise ValueError("unknown source " + source)
    w.update(mat)
    w.update(pulse(**(pulse_kw or {})))
    w.update(over)
    return w


def cfg_3d_256(nsteps: int = 10000) -> dict:
    """256^3 FP32: 128 x 128 x 64 design slab on an eps 2.25 substrate, 4^3 gap,
    x-polarised plane wave along +z injected by total-field / scattered-field
    (box 4 nodes in from the CPML), BF16 snapshots every 32."""
    return workload_3d(256, 256, 256, dx=5e-9, nsteps=nsteps, npml=12, design=(128, 128, 64), gap=(4, 4, 4),
                       source="tfsf", tf_margin=4, substrate=True, snapshot_every=32, snapshot_dtype="bf16")


def cfg_3d_512(nsteps: int = 16000) -> dict:
    """512 x 512 x 384 FP32: 256 x 256 x 96 design region, z-dipole in the gap,
    two bands (650-750 nm and 850-950 nm), FP16 snapshots."""
    return workload_3d(512, 512, 384, dx=5e-9, nsteps=nsteps, npml=12, design=(256, 256, 96), gap=(4, 4, 4),
                       source="dipole", snapshot_every=500, snapshot_dtype="f16",
                       pulse_kw=dict(centers_m=[700e-9, 900e-9], half_width_hz=C0 / 650e-9 - C0 / 700e-9))


def n_cells(w: dict) -> int:
    n = w["nx"] * w["ny"]
    return n * w["nz"] if w["ndim"] == 3 else n


def grid_shape(w: dict) -> list[int]:
    return [w["nx"], w["ny"], w["nz"]] if w["ndim"] == 3 else [w["nx"], w["ny"]]


def describe(w: dict) -> str:
    """One-line description of a workload."""
    dims = "x".join(str(v) for v in grid_shape(w))
    des = "x".join(str(v) for v in reversed(design_shape(w)))
    kind = ("2D in-plane E" if inplane(w) else "2D TM_z") if w["ndim"] == 2 else "3D Yee"
    snap = ("snapshots every %d (%s)" % (w["snapshot_every"], w.get("snapshot_dtype", "f32"))
            if w.get("snapshot_every") else "full history")
    filt = ", %d-cell Gaussian filter" % w["filter_radius"] if w.get("filter_radius") else ""
    if w.get("tfsf"):
        filt += ", TFSF plane wave"
    return "%s %s %s, %d steps, %s design%s, %s" % (kind, dims, w["real"].upper(), w["nsteps"], des, filt, snap)


def inplane(w: dict) -> bool:
    return w["ndim"] == 2 and w.get("pol", 0) == 1


def edge_shapes(lo, hi) -> tuple[tuple[int, int], tuple[int, int]]:
    """Shapes (rows, columns) of the E_x and E_y edge sets of a cell box."""
    wd, h = hi[0] - lo[0], hi[1] - lo[1]
    return (h + 1, wd), (h, wd + 1)


def n_design(w: dict) -> int:
    if inplane(w):
        (a, b), (c, d) = edge_shapes(w["design_lo"], w["design_hi"])
        return a * b + c * d
    n = 1
    for a in range(w["ndim"]):
        n *= w["design_hi"][a] - w["design_lo"][a]
    return n


def design_shape(w: dict) -> tuple[int, ...]:
    """Design-array shape, slowest axis first (x fastest); the in-plane 2D
    mode keeps its E_x edges then its E_y edges in one flat vector."""
    if inplane(w):
        return (n_design(w),)
    s = [w["design_hi"][a] - w["design_lo"][a] for a in range(w["ndim"])]
    return tuple(reversed(s))


def split_edges(w: dict, v: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """(E_x-edge array, E_y-edge array) views of an in-plane design vector."""
    (a, b), (c, d) = edge_shapes(w["design_lo"], w["design_hi"])
    v = np.asarray(v).reshape(-1)
    return v[:a * b].reshape(a, b), v[a * b:].reshape(c, d)


def gap_edge_mask(w: dict) -> np.ndarray:
    """True on the design edges that belong to the gap (in-plane 2D mode)."""
    m = np.zeros(n_design(w), dtype=bool)
    mx, my = split_edges(w, m)
    dl, gl, gh = w["design_lo"], w["gap_lo"], w["gap_hi"]
    mx[gl[1] - dl[1]:gh[1] - dl[1] + 1, gl[0] - dl[0]:gh[0] - dl[0]] = True
    my[gl[1] - dl[1]:gh[1] - dl[1], gl[0] - dl[0]:gh[0] - dl[0] + 1] = True
    return m


def rho_uniform(w: dict, seed: int) -> np.ndarray:
    """rho ~ U[0,1] on the design box (PCG64(seed)), gap entries set to 0."""
    rng = np.random.Generator(np.random.PCG64(seed))
    r = rng.random(design_shape(w))
    return zero_gap(w, r)


def zero_gap(w: dict, r: np.ndarray) -> np.ndarray:
    r = np.array(r, dtype=np.float64, copy=True)
    if inplane(w):
        r = r.reshape(-1)
        r[gap_edge_mask(w)] = 0.0
        return r
    sl = tuple(slice(w["gap_lo"][a] - w["design_lo"][a], w["gap_hi"][a] - w["design_lo"][a])
               for a in reversed(range(w["ndim"])))
    r[sl] = 0.0
    return r


def fixed_blocks_mask(w: dict, axis: int = 0) -> np.ndarray:
    """Design variables of two blocks beside the gap along ``axis``, each the
    gap's size: the paper fixes such regions to metal (Sec. 3.2, AntTM3/4).
    Along x (the E_x polarisation of the in-plane workloads) they make the
    two arms of a dipole gap.  Gap entries are not included."""
    lo, hi = list(w["gap_lo"]), list(w["gap_hi"])
    size = hi[axis] - lo[axis]
    boxes = []
    for sgn in (-1, 1):
        blo, bhi = list(lo), list(hi)
        if sgn < 0:
            blo[axis], bhi[axis] = lo[axis] - size, lo[axis]
        else:
            blo[axis], bhi[axis] = hi[axis], hi[axis] + size
        boxes.append((blo, bhi))
    dl = w["design_lo"]
    if inplane(w):
        m = np.zeros(n_design(w), dtype=bool)
        mx, my = split_edges(w, m)
        for blo, bhi in boxes:
            mx[blo[1] - dl[1]:bhi[1] - dl[1] + 1, blo[0] - dl[0]:bhi[0] - dl[0]] = True
            my[blo[1] - dl[1]:bhi[1] - dl[1], blo[0] - dl[0]:bhi[0] - dl[0] + 1] = True
        m[gap_edge_mask(w)] = False
        return m
    m = np.zeros(design_shape(w), dtype=bool)
    for blo, bhi in boxes:
        sl = tuple(slice(blo[a] - dl[a], bhi[a] - dl[a]) for a in reversed(range(w["ndim"])))
        m[sl] = True
    return m.reshape(-1)


def _bowtie_at(x, y, cx, cy, gx):
    ax = np.abs(y - cy)
    return (np.abs(x - cx) >= gx) & (ax <= 0.6 * (np.abs(x - cx) - gx) + 1.0)


def rho_bowtie(w: dict) -> np.ndarray:
    """Binary bowtie: two triangles whose tips face each other across the gap."""
    if inplane(w):
        # the same shape sampled at the edge midpoints (cell units from the box corner)
        dl, gl, gh = w["design_lo"], w["gap_lo"], w["gap_hi"]
        cx = (gl[0] + gh[0]) / 2.0 - dl[0]
        cy = (gl[1] + gh[1]) / 2.0 - dl[1]
        gx = (gh[0] - gl[0]) / 2.0 + 0.5
        (a, b), (c, d) = edge_shapes(w["design_lo"], w["design_hi"])
        yx, xx = np.mgrid[0:a, 0:b]
        yy, xy = np.mgrid[0:c, 0:d]
        r = np.concatenate([_bowtie_at(xx + 0.5, yx, cx, cy, gx).reshape(-1),
                            _bowtie_at(xy, yy + 0.5, cx, cy, gx).reshape(-1)]).astype(np.float64)
        return zero_gap(w, r)
    shape = design_shape(w)
    h, wd = shape[-2], shape[-1]
    y, x = np.mgrid[0:h, 0:wd]
    cx = (w["gap_lo"][0] + w["gap_hi"][0]) / 2.0 - w["design_lo"][0] - 0.5
    cy = (w["gap_lo"][1] + w["gap_hi"][1]) / 2.0 - w["design_lo"][1] - 0.5
    gx = (w["gap_hi"][0] - w["gap_lo"][0]) / 2.0 + 0.5
    r = _bowtie_at(x, y, cx, cy, gx).astype(np.float64)
    if len(shape) == 3:
        r = np.broadcast_to(r, shape).copy()
    return zero_gap(w, r)


def with_(w: dict, **kw) -> dict:
    v = copy.deepcopy(w)
    v.update(kw)
    return v


# ---------------------------------------------------------------- surrogate

def unet_layers(base: int = 24, in_ch: int = 2) -> list[tuple[str, int, int, int]]:
    """Layers (name, c_in, c_out, kernel) of the 4-level U-Net surrogate, in
    forward order.  Encoder levels double the width (base, 2b, 4b), the
    bottleneck has 8b channels; each decoder level takes [upsampled deeper
    features, skip] concatenated; a 1 x 1 head gives one channel."""
    b = base
    return [("enc1a", in_ch, b, 3), ("enc1b", b, b, 3),
            ("enc2a", b, 2 * b, 3), ("enc2b", 2 * b, 2 * b, 3),
            ("enc3a", 2 * b, 4 * b, 3), ("enc3b", 4 * b, 4 * b, 3),
            ("bota", 4 * b, 8 * b, 3), ("botb", 8 * b, 8 * b, 3),
            ("dec3a", 12 * b, 4 * b, 3), ("dec3b", 4 * b, 4 * b, 3),
            ("dec2a", 6 * b, 2 * b, 3), ("dec2b", 2 * b, 2 * b, 3),
            ("dec1a", 3 * b, b, 3), ("dec1b", b, b, 3),
            ("head", b, 1, 1)]


def unet_params(base: int = 24, seed: int = 0, in_ch: int = 2) -> dict:
    """He-normal weights (W[c_out][c_in][k][k]) and zero biases, PCG64(seed)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    p = {}
    for name, ci, co, k in unet_layers(base, in_ch):
        p[name + ".w"] = rng.standard_normal((co, ci, k, k)) * math.sqrt(2.0 / (ci * k * k))
        p[name + ".b"] = np.zeros(co)
    return p


def unet_param_count(base: int = 24, in_ch: int = 2) -> int:
    return sum(co * ci * k * k + co for _, ci, co, k in unet_layers(base, in_ch))
