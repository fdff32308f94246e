"""CPU-only checks of the C ABI library: it loads, exports every symbol that
include/fdtd.h declares, sizes workspaces and rejects bad configurations
(no compute calls: there is no GPU here)."""
import ctypes as C
import os
import re

import pytest

from paper_2203_01462_gb300 import binding as B
from paper_2203_01462_gb300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_symbols():
    src = open(os.path.join(ROOT, "include", "fdtd.h")).read()
    return sorted(set(re.findall(r"\b(fdtd_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_every_header_symbol():
    L = B.load()
    syms = header_symbols()
    assert syms, "no declarations found"
    for name in syms:
        assert hasattr(L, name), name
    assert sorted(B.EXPORTS) == syms


def test_status_strings():
    L = B.load()
    for s in range(8):
        assert L.fdtd_status_string(s)


def test_workspace_sizes():
    small = B.workspace_bytes(I.small_2d())
    assert small > 0 and small % 256 == 0
    big = B.workspace_bytes(I.cfg_2d_2048())
    # 313 FP32 snapshots of ~54 MB dominate the 2048^2 workload.
    assert 15e9 < big < 25e9
    full = B.workspace_bytes(dict(I.cfg_2d_2048(), snapshot_every=0))
    assert full > 80e9  # full FP32 design-box history: 20000 x 1024^2 x 4 B


@pytest.mark.parametrize("bad", [
    dict(courant=0.75),                    # above the 2D Courant limit
    dict(real="f16"),
    dict(design_lo=[0, 0, 0]),             # design box wider than the grid? (lo 0 still valid)
    dict(gap_lo=[1, 1, 0], gap_hi=[4, 4, 1]),  # gap outside the design box
    dict(npml=30),                         # CPML slabs overlap
    dict(nsteps=0),
    dict(omega_p=0.0),
    dict(psi_s_ratio=0.0),                 # Eq. (25a) divides by psi_i
    dict(waveform=2),                      # no such excitation
    dict(waveform=1, bandwidth=0.0, lobes=4),
    dict(waveform=1, bandwidth=1e14, lobes=0),
])
def test_bad_configurations_rejected(bad):
    w = I.small_2d()
    if "real" in bad and bad["real"] == "f16":
        cfg = B.config(w)
        cfg.real_bytes = 2
        n = C.c_size_t()
        assert B.load().fdtd_workspace_bytes(C.byref(cfg), C.byref(n)) == 1
        return
    w.update(bad)
    if bad.get("design_lo") == [0, 0, 0]:
        return  # valid: design box may start at the corner
    with pytest.raises(B.FdtdError) as e:
        B.workspace_bytes(w)
    assert e.value.status == 1


@pytest.mark.parametrize("medium,ok", [
    (dict(eps_s=0.4), False),    # background: S sqrt(2) = 0.71 > sqrt(0.4) = 0.63
    (dict(eps_g=0.45), False),   # gap medium
    (dict(eps_inf=0.3), False),  # the metal's high-frequency limit
    (dict(eps_s=0.55), True),    # sqrt(0.55) = 0.74: still inside the limit
    (dict(eps_inf=4.469), True),
])
def test_courant_limit_checked_in_every_medium(medium, ok):
    """Light is 1/sqrt(eps) slower in a medium of permittivity eps, so the
    Courant limit S sqrt(d) < 1 of vacuum becomes S sqrt(d) < sqrt(eps): a
    configuration that breaks it in any of its media is refused."""
    w = dict(I.small_2d(), **medium)
    if ok:
        assert B.workspace_bytes(w) > 0
    else:
        with pytest.raises(B.FdtdError) as e:
            B.workspace_bytes(w)
        assert e.value.status == 1
    w3 = I.workload_3d(21, 19, 31, dx=20e-9, nsteps=10, npml=4, design=(9, 7, 6), gap=(2, 2, 2), substrate=True,
                       courant=0.5)
    assert B.workspace_bytes(w3) > 0
    with pytest.raises(B.FdtdError):
        B.workspace_bytes(dict(w3, sub_eps=0.7))  # 0.5 sqrt(3) = 0.87 > sqrt(0.7) = 0.84


def test_grid_beyond_32_bit_indexing_rejected():
    """The 2D step kernel indexes one array with 32-bit integers: a grid of
    2^31 or more padded nodes is refused before anything is allocated."""
    w = I.small_2d()
    w.update(nx=65536, ny=40000, npml=10, design_lo=[100, 100, 0], design_hi=[200, 200, 1],
             gap_lo=[140, 140, 0], gap_hi=[143, 143, 1], src_lo=[10, 15, 0], src_hi=[65526, 16, 1])
    with pytest.raises(B.FdtdError) as e:
        B.workspace_bytes(w)
    assert e.value.status == 1
    w.update(ny=30000)  # 1.97e9 nodes: accepted
    assert B.workspace_bytes(w) > 0


def _tfsf_case(**kw):
    w = I.workload_3d(21, 19, 31, dx=20e-9, nsteps=50, npml=4, design=(9, 7, 6), gap=(2, 2, 2),
                      source="tfsf", substrate=True, real="f32", tf_margin=1)
    w.update(kw)
    return w


def test_plane_wave_configuration_sized_and_checked():
    """A valid total-field box adds one incident row per step to the
    workspace; boxes that cut the design box, reach the CPML or sit below
    the source plane, and non-x sources, are refused."""
    w = _tfsf_case()
    plain = dict(w, tfsf=0)
    row = 2 * (w["tf_hi"][2] - w["tf_lo"][2] + 1) + 1
    extra = B.workspace_bytes(w) - B.workspace_bytes(plain)
    assert row * w["nsteps"] * 4 <= extra <= row * w["nsteps"] * 4 + 4 * w["nz"] * 4 + 1024
    lo, hi, d_lo, d_hi = w["tf_lo"], w["tf_hi"], w["design_lo"], w["design_hi"]
    bad = [
        dict(tf_lo=[d_lo[0], lo[1], lo[2]]),                     # face on the design box
        dict(tf_hi=[d_hi[0] - 1, hi[1], hi[2]]),                 # box inside the design box
        dict(tf_lo=[w["npml"], lo[1], lo[2]]),                   # face in the CPML
        dict(tf_hi=[hi[0], w["ny"] - w["npml"] - 1, hi[2]]),     # far face in the CPML
        dict(tf_lo=[lo[0], lo[1], w["src_lo"][2]]),              # source plane inside the box
        dict(src_comp=1),                                         # only the x-polarised wave
        dict(src_hi=[w["src_hi"][0], w["src_hi"][1], w["src_lo"][2] + 2]),  # two source planes
        dict(tfsf=2),
    ]
    for kw in bad:
        with pytest.raises(B.FdtdError) as e:
            B.workspace_bytes(dict(w, **kw))
        assert e.value.status == 1, kw
    two_d = I.small_2d()
    with pytest.raises(B.FdtdError):
        B.workspace_bytes(dict(two_d, tfsf=1, tf_lo=[2, 2, 0], tf_hi=[10, 10, 0]))


def _c_layout(tmp_path, include: str, struct: str, fields, extra_flags=()):
    """sizeof and offsetof of each field of a C struct, from gcc."""
    import subprocess
    src = tmp_path / ("layout_%s.c" % struct.replace(" ", "_"))
    lines = ["#include <stddef.h>", "#include <stdio.h>", include, "int main(void) {",
             '  printf("%%zu\\n", sizeof(%s));' % struct]
    lines += ['  printf("%%zu\\n", offsetof(%s, %s));' % (struct, f) for f in fields]
    lines += ["  return 0;", "}"]
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / ("layout_%s" % struct.replace(" ", "_"))
    subprocess.run(["gcc", "-std=c11", "-Wall", "-Werror", *extra_flags, "-o", str(exe), str(src), "-lm"],
                   check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()
    return int(out[0]), [int(v) for v in out[1:]]


@pytest.mark.parametrize("struct,cls", [("fdtd_config", "FdtdConfig"), ("fdtd_info", "FdtdInfo")])
def test_binding_structs_match_the_c_header(tmp_path, struct, cls):
    """The ctypes mirrors of the ABI structs have the header's size and
    field offsets (compiled as C11, so the header is valid C)."""
    ct = getattr(B, cls)
    names = [f[0] for f in ct._fields_]
    size, offs = _c_layout(tmp_path, '#include "%s"' % os.path.join(ROOT, "include", "fdtd.h"), struct, names)
    assert size == C.sizeof(ct)
    assert offs == [getattr(ct, n).offset for n in names]


def test_surrogate_header_is_valid_c(tmp_path):
    import subprocess
    src = tmp_path / "sur.c"
    src.write_text('#include "%s"\nint main(void) { return 0; }\n' % os.path.join(ROOT, "include", "surrogate.h"))
    subprocess.run(["gcc", "-std=c11", "-Wall", "-Werror", "-c", "-o", str(tmp_path / "sur.o"), str(src)],
                   check=True, capture_output=True)


def test_oracle_config_mirror_matches_its_c_struct(tmp_path):
    from oracle import oracle as O
    names = [f[0] for f in O.OrConfig._fields_]
    size, offs = _c_layout(tmp_path, '#include "%s"' % os.path.join(ROOT, "oracle", "fdtd_oracle.c"), "or_config",
                           names, extra_flags=("-Wno-unused-function", "-fopenmp"))
    assert size == C.sizeof(O.OrConfig)
    assert offs == [getattr(O.OrConfig, n).offset for n in names]


def test_library_exports_every_surrogate_header_symbol():
    src = open(os.path.join(ROOT, "include", "surrogate.h")).read()
    syms = sorted(set(re.findall(r"\b(nn_[a-z0-9_]+)\s*\(", src)))
    assert syms, "no declarations found"
    L = B.load()
    for name in syms:
        assert hasattr(L, name), name
    from paper_2203_01462_gb300 import surrogate as S
    assert sorted(S._FNS) == syms
