#!/usr/bin/env python3
"""Throughput of the FDTD + Drude adjoint hot path on one GB300 (or N replicas).

One bench step = one design evaluation of the 3D 256^3 FP32 workload:
set_design -> forward (10000 steps of the Yee + Drude + CPML leapfrog, an
x-polarised plane wave injected through a total-field / scattered-field
box, BF16 checkpoints every 32 steps) -> adjoint (segment recompute +
adjoint + fused sensitivities) -> gradient.  It is the largest workload
whose 20 + 5 evaluations fit a few minutes; the 512 x 512 x 384 one (about
a minute per evaluation) and the 2D ones run with --workload.  The metric
counts forward + adjoint cell-updates (2 x cells x steps per evaluation);
recompute sweeps are work the method pays but are not counted there (the
"raw" key counts them).

Timing: CUDA events on the solver's stream around each step, L2 flushed
(a 256 MB write) between steps outside the events, max over ranks.  Under
torchrun each rank runs an independent replica (the path needs no
collective), so value = ranks x work / slowest rank ("weak" scaling).

``--impl reference`` times the FP64 CPU oracle on the host cores on a
bounded sample of the same workload (fewer time steps per evaluation).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2203_01462_gb300 import inputs as I  # noqa: E402

METRIC = "Gcell-updates/s fwd+adjoint"
UNIT = "Gcell-updates/s"
# Bounded oracle samples, in grid-node time steps of the forward run: about
# 1.3e9 node steps (75 steps of a 256^3 grid, about 15 s of forward +
# adjoint on 16 host cores) for the cpu_baseline key, and 5e8 (30 steps at
# 256^3) per reference-arm evaluation.
CPU_CELL_STEPS = 256 ** 3 * 75
REF_CELL_STEPS = 256 ** 3 * 30


WORKLOADS = {
    "cfg_2d_2048": I.cfg_2d_2048,
    "cfg_2d_160": I.cfg_2d_160,
    "cfg_3d_256": I.cfg_3d_256,
    "cfg_3d_512": I.cfg_3d_512,
    "cfg_2d_inplane_200": lambda: I.cfg_2d_inplane_paper(200.0, nsteps=78000, snapshot_every=64),
}


def workload(name: str, nsteps: int | None):
    if name not in WORKLOADS:
        raise SystemExit("unknown workload " + name)
    w = WORKLOADS[name]()
    if nsteps:
        w["nsteps"] = int(nsteps)
    return w


# DRAM bytes (read + write) of the forward step kernels of one time step,
# measured by ncu on each workload's own grid (k_step2d<float,0>; k_h3d +
# k_e3d<float,0>); entries are removed whenever a kernel changes.
NCU_TRAFFIC_PER_STEP = {"cfg_2d_2048": 74.2e6, "cfg_3d_256": 1298.4e6}


def damping(k: int) -> float:
    """Artificial-damping schedule: gamma x10 decaying geometrically to x1 over 50 iterations."""
    return 10.0 ** (1.0 - min(k, 50) / 50.0)


def algorithmic_bytes(w: dict) -> dict:
    """Algorithmic HBM bytes per time step: one read + one write of each
    state word touched, no temporal-blocking credit.  2D: Ez, Hx, Hy per
    node; 3D: six components per node.  Design nodes add J (read + write per
    E component) and rho~ (read); CPML slab nodes add their psi terms (2 in
    2D, 4 per slab crossed in 3D, read + write); the forward pays the
    amortised checkpoint copy, the recompute the design record, the adjoint
    the forward-field read and the FP64 accumulator."""
    rb = 8 if w["real"] == "f64" else 4
    npml = w["npml"]
    md = I.n_design(w)
    if w["ndim"] == 2:
        nx, ny = w["nx"], w["ny"]
        nc = nx * ny
        ncomp, psi_per_slab = 3, 2
        slab_nodes = 2 * npml * (nx + ny)
    else:
        nx, ny, nz = w["nx"], w["ny"], w["nz"]
        nc = nx * ny * nz
        ncomp, psi_per_slab = 6, 4
        slab_nodes = 2 * npml * (nx * ny + ny * nz + nx * nz)
    ne = ncomp // 3 if w["ndim"] == 2 else 3   # E components carrying J
    grid = 2 * ncomp * rb * nc
    design = (2 * ne + 1) * rb * md
    pml = 2 * psi_per_slab * rb * slab_nodes
    K = w.get("snapshot_every", 0)
    snap_rb = {"f32": rb, "bf16": 2, "f16": 2}[w.get("snapshot_dtype", "f32")]
    state_words = ncomp * nc + ne * md + 2 * psi_per_slab * slab_nodes
    fwd = grid + design + pml + (2 * (rb + snap_rb) * state_words / 2 / K if K else ne * rb * md)
    rec = grid + design + pml + ne * rb * md
    adj = grid + design + pml + ne * rb * md + 16 * md
    return dict(forward=fwd, recompute=rec, adjoint=adj, cells=nc)


def sample_clocks(path: str):
    q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    try:
        f = open(path, "w")
        return subprocess.Popen(["nvidia-smi", "--query-gpu=" + q, "--format=csv,noheader,nounits", "-lms", "200"],
                                stdout=f, stderr=subprocess.DEVNULL), f
    except Exception:
        return None, None


def parse_clocks(path: str, gpu_index: int):
    out = dict(sm_mhz=None, sm_max_mhz=None, reasons=[])
    try:
        rows = [r.split(",") for r in open(path).read().strip().splitlines() if r.strip()]
    except Exception:
        return out
    rows = [[x.strip() for x in r] for r in rows if len(r) >= 9 and r[0].strip() == str(gpu_index)]
    if not rows:
        return out
    sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
    mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
    out.update(sm_mhz=statistics.median(sm) if sm else None, sm_max_mhz=max(mx) if mx else None,
               reasons=reasons)
    return out


def sample_nsteps(w: dict, requested: int, cell_steps: float) -> int:
    """Time steps of the oracle's bounded sample: ``requested`` if given, else
    as many as fit ``cell_steps`` grid-node steps (forward), between 10 and
    1000 and at most the workload's own count."""
    if requested > 0:
        return min(requested, w["nsteps"])
    return max(1, min(w["nsteps"], 1000, max(10, int(cell_steps / I.n_cells(w)))))


def cpu_baseline(w: dict, nsteps: int) -> dict:
    """The oracle, as it stands, on the host cores: one forward + adjoint +
    gradient of the same workload cut to ``nsteps`` time steps, on all cores
    (the reported value), then on one thread over a proportionally shorter
    cut (value_1_thread)."""
    from oracle import oracle as O
    cores = os.cpu_count() or 1

    def run(threads, ns):
        O.set_threads(threads)
        ws = dict(w, nsteps=ns)
        rho = I.rho_uniform(ws, 0)
        t = time.perf_counter()
        O.gradient(ws, rho, 0.0, damping(0))
        return 2.0 * I.n_cells(ws) * ns / (time.perf_counter() - t) / 1e9, time.perf_counter() - t

    v_all, dt = run(cores, nsteps)
    ns1 = max(5, nsteps // cores)
    v_one, dt1 = run(1, ns1)
    O.set_threads(cores)
    return dict(value=v_all, unit=UNIT, cores=O.threads(), kind="oracle",
                sample="%s with %d of %d time steps, one forward+adjoint+gradient, %.1f s"
                       % (w.get("name", "workload"), nsteps, w["nsteps"], dt),
                value_1_thread=v_one,
                sample_1_thread="%d of %d time steps on one thread, %.1f s" % (ns1, w["nsteps"], dt1))


def run_reference(args, w) -> None:
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import oracle as O
    cores = os.cpu_count() or 1
    O.set_threads(cores)
    ns = sample_nsteps(w, args.ref_nsteps, REF_CELL_STEPS)
    ws = dict(w, nsteps=ns)
    rho = I.rho_uniform(ws, 0)
    for k in range(args.warmup):
        O.gradient(ws, rho, 0.0, damping(k))
    times = []
    for k in range(args.steps):
        t = time.perf_counter()
        O.gradient(ws, rho, 0.0, damping(args.warmup + k))
        times.append(time.perf_counter() - t)
    cu = 2.0 * I.n_cells(w) * ns
    value = cu * len(times) / sum(times) / 1e9
    # the oracle runs on the host cores; n_gpus repeats the launch's N so the
    # line matches the accelerated arm it is compared with
    line = dict(impl="reference", metric=METRIC, value=value, unit=UNIT, n_gpus=args.gpus, steps=args.steps,
                warmup=args.warmup, ms_per_step=1e3 * sum(times) / len(times), higher_is_better=True,
                scaling="weak", vs_baseline=None, dtype="f64", data="synthetic",
                config=dict(workload=I.describe(w), grid=I.grid_shape(w), nsteps=w["nsteps"],
                            sample_nsteps=ns),
                cpu_baseline=dict(value=value, unit=UNIT, cores=O.threads(), kind="oracle",
                                  sample="%d of %d time steps per evaluation" % (ns, w["nsteps"])),
                e2e=dict(value=value, unit=UNIT, h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(line), flush=True)


def run_surrogate(args) -> None:
    """Print the surrogate comparison (surrogate_measure) as one JSON line."""
    print(json.dumps(surrogate_measure(args)), flush=True)


def surrogate_measure(args) -> dict:
    """Design iterations/s at a matched objective: the plain adjoint loop
    (one forward + adjoint solve per design step) against the
    surrogate-assisted loop (one solve + four U-Net steps per round), on the
    256^2-design workload, both under the same damping continuation (gamma
    x10 decaying to x1 over the first half of the plain run).  The network
    is pretrained on (rho, damping level) -> gradient pairs from plain
    trajectories that follow the same continuation from random starts; the
    compared runs start from a half-metal bowtie, a design outside that
    distribution.  The surrogate loop stops once the W~ of one of its full
    solves is within 1 % of the plain loop's final W~.  Wall time is
    reported for the loop alone, with the pretraining (pair collection +
    training) included, and with the pretraining shared by a stated number
    of designs optimised with one network, and the number of designs from
    which the surrogate pays for its pretraining."""
    import torch
    from paper_2203_01462_gb300.binding import Solver
    from paper_2203_01462_gb300.optimize import optimize
    from paper_2203_01462_gb300.surrogate_loop import Trainer, collect_pairs_concurrent, surrogate_optimize
    w = I.cfg_2d_316()
    s = Solver(w)
    U, D, g0 = args.sur_updates, args.sur_damping_iters, args.sur_damping
    t = time.perf_counter()
    rho0s = [I.zero_gap(w, 0.02 * I.rho_uniform(w, 300 + k)) for k in range(args.sur_trajectories)]
    # the training trajectories are independent: they run side by side
    pairs = collect_pairs_concurrent(w, rho0s, iters=args.sur_pairs_per_trajectory, move=0.05, damping_start=g0,
                                     damping_iters=D, width=args.sur_trajectories, steps_per_launch=1)
    torch.cuda.synchronize()
    collect_s = time.perf_counter() - t
    tr = Trainer(256, 256, base=24, batch=8, seed=0, lr=1e-3)
    t = time.perf_counter()
    loss = tr.fit(pairs, args.sur_train_steps)
    # a two-update surrogate run on its own pair list: the first use of the
    # loop's operations in a process costs about 0.8 s of one-time setup,
    # counted here with the pretraining rather than in a design's loop
    surrogate_optimize(s, tr, I.zero_gap(w, 0.5 * I.rho_bowtie(w)), updates=2, inner=1, move=0.05,
                       damping_start=g0, damping_iters=D, pairs=None, fit_steps=0)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t
    rho_start = I.zero_gap(w, 0.5 * I.rho_bowtie(w))
    t = time.perf_counter()
    _, hp = optimize(s, rho_start, iters=U, move=0.05, zeta_stop=0.0, damping_start=g0, damping_iters=D,
                     move_decay=1.0)
    torch.cuda.synchronize()
    plain_s = time.perf_counter() - t
    target = hp.W[-1]
    t = time.perf_counter()
    _, hs, st = surrogate_optimize(s, tr, rho_start, updates=3 * U, inner=4, move=0.05, damping_start=g0,
                                   damping_iters=D, pairs=pairs, fit_steps=0, target_W=0.99 * target)
    torch.cuda.synchronize()
    sur_s = time.perf_counter() - t
    Ws = [x for x in hs.W if x == x]
    pre = collect_s + train_s
    R = args.sur_designs
    levels = sorted({round(float(x[1, 0, 0, 0].item()), 6) for x in pairs.x})
    line = dict(metric="design iters/s at matched objective", value=len(hs.W) / sur_s, unit="design updates/s",
                higher_is_better=True, n_gpus=1, data="synthetic",
                config=dict(workload=I.describe(w), network="U-Net base 24 (%d parameters), BF16 GEMM operands on the "
                            "tensor cores (mma.sync), FP32 accumulation and master weights" % I.unet_param_count(24),
                            solver="temporally blocked, 8 steps per launch (the library's default on this grid)",
                            inner_steps=4, matched="within 1 % of the plain loop's final W",
                            damping="gamma x%g decaying to x1 over %d updates" % (g0, D),
                            start="half-metal bowtie (0.5 x binary bowtie)"),
                plain=dict(updates=U, seconds=plain_s, updates_per_s=U / plain_s, final_W=target),
                surrogate=dict(updates=len(hs.W), seconds=sur_s, final_W=Ws[-1], reached=Ws[-1] >= 0.99 * target,
                               **st),
                wall_time_ratio=sur_s / plain_s,
                wall_time_ratio_with_pretraining=(sur_s + pre) / plain_s,
                wall_time_ratio_amortised=dict(designs=R, ratio=(sur_s + pre / R) / plain_s),
                break_even_designs=(pre / (plain_s - sur_s)) if plain_s > sur_s else None,
                pretraining=dict(pairs=len(pairs), damping_levels_in_pairs=len(levels), collect_s=collect_s,
                                 collect="%d trajectories side by side, one solver and CUDA stream each, "
                                 "one launch per step" % args.sur_trajectories,
                                 train_steps=args.sur_train_steps, train_s=train_s, final_loss=loss))
    return line


def max_over_ranks(x: float, dist, device) -> float:
    """The slowest rank's time (all ranks call this after their timed region)."""
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.barrier()
    return float(t.item())


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="cfg_3d_256")
    ap.add_argument("--nsteps", type=int, default=0, help="override the time-step count (quick runs)")
    ap.add_argument("--cpu-nsteps", type=int, default=0,
                    help="time steps of the oracle sample (0: sized to 256^3 x 75 node steps)")
    ap.add_argument("--ref-nsteps", type=int, default=0,
                    help="time steps per reference-arm evaluation (0: sized to 256^3 x 30 node steps)")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--surrogate", action="store_true",
                    help="measure the surrogate-assisted optimization loop against the plain adjoint loop")
    ap.add_argument("--sur-trajectories", type=int, default=16)
    ap.add_argument("--sur-pairs-per-trajectory", type=int, default=40)
    ap.add_argument("--sur-updates", type=int, default=80)
    ap.add_argument("--sur-damping", type=float, default=10.0, help="initial damping factor of the continuation")
    ap.add_argument("--sur-damping-iters", type=int, default=40, help="updates over which the damping decays to x1")
    ap.add_argument("--sur-train-steps", type=int, default=300)
    ap.add_argument("--sur-designs", type=int, default=10,
                    help="designs sharing one pretrained network, for the amortised wall-time ratio")
    ap.add_argument("--no-surrogate", action="store_true",
                    help="leave the surrogate comparison (design_iters) out of the default line")
    args = ap.parse_args()
    if args.surrogate:
        run_surrogate(args)
        return
    w = workload(args.workload, args.nsteps)
    w["name"] = args.workload
    if args.impl == "reference":
        run_reference(args, w)
        return

    import torch
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    # The oracle's host-core sample runs before any GPU work, on rank 0 of a
    # one-GPU run only.
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(w, sample_nsteps(w, args.cpu_nsteps, CPU_CELL_STEPS))

    from paper_2203_01462_gb300.binding import Solver
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(dev)
    s = Solver(w, device=dev, stream=stream)
    # 2D E_z workloads: keep 30 % of the ping-pong state persisting in L2
    # (the share that measured fastest; results are bit-identical)
    l2_share = 0.3 if (w["ndim"] == 2 and not I.inplane(w)) else 0.0
    if l2_share:
        s.set_l2_residency(l2_share)
    rho = torch.tensor(I.rho_uniform(w, rank), dtype=torch.float32 if w["real"] == "f32" else torch.float64,
                       device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    Wout = torch.zeros(1, dtype=torch.float64, device=dev)
    gout = torch.empty(s.n_design, dtype=torch.float64, device=dev)

    def one_step(k, ev=None):
        with torch.cuda.stream(stream):
            if ev: ev[0].record(stream)
            s.set_design(rho)
            s.set_damping(0.0, damping(k))
            if ev: ev[1].record(stream)
            s.forward(Wout)
            if ev: ev[2].record(stream)
            s.adjoint()
            if ev: ev[3].record(stream)
            s.gradient(gout)
            if ev: ev[4].record(stream)

    for k in range(args.warmup):
        one_step(k)
    s.sync()

    clk_path = os.path.join(os.environ.get("FDTD_RESULTS_DIR") or os.path.join(ROOT, "results"),
                            "clocks_bench_rank%d.csv" % rank)
    os.makedirs(os.path.dirname(clk_path), exist_ok=True)
    proc, fh = sample_clocks(clk_path)
    launches0 = s.info().launches
    if dist:
        dist.barrier()
    torch.cuda.synchronize(dev)
    step_ms, fwd_ms, adj_ms = [], [], []
    for k in range(args.steps):
        with torch.cuda.stream(stream):
            flush.fill_(k & 0xff)
        stream.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
        one_step(args.warmup + k, ev)
        ev[4].synchronize()
        step_ms.append(ev[0].elapsed_time(ev[4]))
        fwd_ms.append(ev[1].elapsed_time(ev[2]))
        adj_ms.append(ev[2].elapsed_time(ev[3]))
    s.sync()
    torch.cuda.synchronize(dev)
    launches = s.info().launches - launches0 - 0
    if proc:
        proc.terminate()
        proc.wait()
        fh.close()
    total_ms = sum(step_ms)
    if dist:
        total_ms = max_over_ranks(total_ms, dist, dev)

    nc, N = I.n_cells(w), w["nsteps"]
    cu_step = 2.0 * nc * N
    value = world * cu_step * args.steps / (total_ms / 1e3) / 1e9

    # e2e through the C ABI with host buffers (copies inside the call).
    rho_h = rho.cpu().numpy()
    e2e_t = []
    for k in range(args.e2e_steps):
        t0 = time.perf_counter()
        s.run_host(rho_h)
        e2e_t.append(time.perf_counter() - t0)
    e2e_val = cu_step * len(e2e_t) / sum(e2e_t) / 1e9 if e2e_t else None
    n_design = s.n_design

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return

    # The metric's second half, design iterations/s at a matched objective
    # (the surrogate loop against the plain adjoint loop on the 256^2-design
    # workload), measured after the timed region on a one-GPU run.
    design_iters = None
    if world == 1 and not args.no_surrogate and not args.nsteps:
        del s
        torch.cuda.empty_cache()
        design_iters = surrogate_measure(args)

    import json as _j
    peaks = {}
    try:
        peaks = _j.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm = peaks.get("hbm_gbs")
    peak_src = "measured" if hbm else "fallback"
    hbm = hbm or 6800.0
    ab = algorithmic_bytes(w)
    fwd_s = statistics.median(fwd_ms) / 1e3
    achieved = ab["forward"] * N / fwd_s / 1e9
    clocks = parse_clocks(clk_path, local)
    rb = 8 if w["real"] == "f64" else 4
    line = dict(
        metric=METRIC, value=value, unit=UNIT, n_gpus=world, steps=args.steps, warmup=args.warmup,
        ms_per_step=total_ms / args.steps, higher_is_better=True, scaling="weak", vs_baseline=None,
        dtype=w["real"], data="synthetic",
        config=dict(workload=I.describe(w), grid=I.grid_shape(w), nsteps=N, design=list(I.design_shape(w))[::-1],
                    snapshot_every=w["snapshot_every"], snapshot_dtype=w.get("snapshot_dtype", "f32"),
                    parallelism="replicas" if world > 1 else "1 GPU",
                    l2="flushed (256 MB write) between timed steps",
                    l2_residency=l2_share),
        roofline=dict(bound="hbm", achieved=achieved, peak=hbm, unit="GB/s", frac=achieved / hbm,
                      traffic=NCU_TRAFFIC_PER_STEP.get(w["name"]), traffic_unit="bytes per forward step",
                      algorithmic_bytes_per_step=ab["forward"],
                      kernel=("k_hp + k_ep<float,0> (forward H and E half steps, E in plane)" if I.inplane(w)
                              else "k_step2d<float,0> (fused forward leapfrog step)") if w["ndim"] == 2
                      else "k_h3d + k_e3d<float,0> (forward H and E half steps; a plane wave's face corrections "
                      "inside them)",
                      peak_source=peak_src),
        phases_ms=dict(forward=statistics.median(fwd_ms), adjoint_with_recompute=statistics.median(adj_ms)),
        # every sweep the method runs: with checkpoints the adjoint phase also
        # recomputes the forward once
        raw=dict(value=world * (2.0 + (1.0 if w.get("snapshot_every") else 0.0)) * nc * N * args.steps
                 / (total_ms / 1e3) / 1e9, unit=UNIT, counts="forward + recompute + adjoint sweeps"),
        cpu_baseline=cpu,
        e2e=dict(value=e2e_val, unit=UNIT, h2d_bytes_per_step=n_design * rb,
                 d2h_bytes_per_step=8 + 8 * n_design),
        clocks=clocks,
        gpu_launches=int(launches),
        design_iters=design_iters,
    )
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
