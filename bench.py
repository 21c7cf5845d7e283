#!/usr/bin/env python3
"""Benchmark: FP64 WENO5/WENO7 + SSP-RK3 cell-updates/s on one GB300.

Workload (headline): 3+1D ellipsoidal flow on a 256^3 grid, WENO7, FP64,
synthetic seeded data shaped like the paper's Sec. 3 test (Gaussian ellipsoid
e0 = 20, a, b, c = 2, 3, 4, linear axis-scaled velocity, n ~ e, p = e/3).
A "step" is one full RK3 step (per stage an x-, a y- and a z-face pass and a
per-cell combination kernel, plus two 1-thread bookkeeping kernels).  A cell-update is one interior cell advanced by one RK3
step.  The state (3.6 GB of FP64 fields) is far larger than L2 (129 MB), so
no flush is needed between steps.

Prints ONE JSON line (rank 0).  Multi-GPU (torchrun): every rank runs an
independent replica of the grid (the single-grid path does not shard); value =
all ranks' cell-updates / max-over-ranks time.
"""
import argparse
import ctypes
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# Algorithmic FP64 work of one interior cell and one RK3 stage, every face
# reconstructed from its own stencil as the scheme defines it (FMA = 2 flops,
# add/mul/reciprocal/sqrt = 1): 15 face-field reconstruction pairs
# (2 x 61 / 2 x 136 flops + 6 to combine), flux differences 40, RK combine 20
# (mean of 10/25/25), split fluxes 75, primitive recovery 22, speeds 34.  The
# pencil-sweep kernels carry stencil differences between neighbouring faces
# and take the products with constants on the integer pipe, so they execute
# fewer FP64 instructions than this count implies; the flop rate by this count
# is reported as an equivalent work rate, not as a utilisation.
FLOPS_PER_CELL_STAGE = {5: 15 * (2 * 61 + 6) + 40 + 20 + 75 + 22 + 34,
                        7: 15 * (2 * 136 + 6) + 40 + 20 + 75 + 22 + 34}
# Executed FP64 instructions (thread-level DFMA + DADD + DMUL, each one issue
# slot of the FP64 pipe) per interior cell and RK3 stage, z pass + stage kernel,
# and the DRAM bytes (read + write) per cell and stage, from ncu captures of the
# 128^3 ellipsoidal workload (mean of stages 1-3, every launch of a stage:
# the face passes and the stage or combination kernel), keyed by (scheme,
# launch variant, tile x, tile y).  roofline.frac = this count x cells / stage time /
# the FP64 FMA issue rate measured in the same run: the FP64 pipe's
# utilisation.  A launch without a capture reports null.
NCU_FP64_INST_PER_CELL_STAGE = {(7, 16, 16, 16): 1237.0, (7, 15, 16, 16): 1297.5, (5, 12, 16, 16): 746.5}
NCU_DRAM_BYTES_PER_CELL_STAGE = {(7, 16, 16, 16): 686.1, (7, 15, 16, 16): 683.2, (5, 12, 16, 16): 509.1}
# FP64 pipe busy, time-weighted over the launches of one stage
NCU_FP64_PIPE_BUSY = {(7, 16, 16, 16): 0.750, (7, 15, 16, 16): 0.802, (5, 12, 16, 16): 0.845}
# Algorithmic HBM traffic per cell-update: stage 1 reads u^n, writes u1 (80 B);
# stages 2, 3 read u^n and u^(k), write u^(k+1) (120 B each).
HBM_BYTES_PER_CELL_UPDATE = 320
SMS = 152


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {"hbm_gbs": 6800.0, "source": "fallback"}


class ClockSampler:
    """nvidia-smi clocks/throttle sampling during the timed region."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.idx = device_index
        self.p = None
        self.lines = []

    def __enter__(self):
        ids = []
        try:
            import torch
            u = getattr(torch.cuda.get_device_properties(self.idx), "uuid", None)
            if u is not None:
                s = str(u)
                ids.append(s if s.startswith("GPU-") else "GPU-" + s)
        except Exception:
            pass
        ids.append(str(self.idx))
        for i in ids:
            try:
                chk = subprocess.run(["nvidia-smi", "-i", i, "--query-gpu=clocks.sm", "--format=csv,noheader"],
                                     capture_output=True, text=True, timeout=20)
                if chk.returncode == 0:
                    self.p = subprocess.Popen(["nvidia-smi", "-i", i, "--query-gpu=" + self.Q,
                                               "--format=csv,noheader,nounits", "-lms", "200"],
                                              stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
                    break
            except Exception:
                continue
        return self

    def __exit__(self, *exc):
        if self.p is not None:
            self.p.terminate()
            try:
                out, _ = self.p.communicate(timeout=10)
            except Exception:
                self.p.kill()
                out, _ = self.p.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            parts = [x.strip() for x in l.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def workload(scheme, N=256):
    import workloads as W
    return W.ellipsoidal(N=N, scheme=scheme)


def cpu_sample(scheme, N=256, sub=128):
    """Central sub^3 block of the N^3 workload (same dx), outflow edges."""
    g, w = workload(scheme, N)
    lo = (N - sub) // 2
    ws = np.ascontiguousarray(w[:, lo:lo + sub, lo:lo + sub, lo:lo + sub])
    import workloads as W
    gs = W.Grid(n=(sub, sub, sub), dx=g.dx, origin=tuple(o + lo * d for o, d in zip(g.origin, g.dx)),
                bc=(0, 0, 0), scheme=scheme, cfl=g.cfl, name="ellipsoidal-subblock")
    return gs, ws


def time_oracle(scheme, steps, sub, N=256):
    import oracle
    oracle.build()
    gs, ws = cpu_sample(scheme, N=N, sub=sub)
    c = oracle.make_cfg(gs.n, gs.dx, scheme=scheme, cfl=gs.cfl)
    u0 = oracle.prim2con(ws)
    t0 = time.perf_counter()
    oracle.run(c, u0, steps)
    dt = time.perf_counter() - t0
    return gs.cells * steps / dt, dt, oracle.max_threads()


def headline_metric(scheme, grid):
    return "FP64 WENO%d cell-updates/s at %d^3 (ellipsoidal flow); %%HBM peak" % (scheme, grid)


def reference_arm(args):
    """The oracle (plain FP64 C, OpenMP over the host cores) on a bounded
    sample of the same workload: each step = one RK3 step of the central
    48^3 block of the 256^3 grid."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    sub = 48
    import oracle
    oracle.build()
    gs, ws = cpu_sample(args.scheme, N=args.grid, sub=min(sub, args.grid))
    c = oracle.make_cfg(gs.n, gs.dx, scheme=args.scheme, cfl=gs.cfl)
    u = oracle.prim2con(ws)
    for _ in range(args.warmup):
        u = oracle.run(c, u, 1)[0]
    t0 = time.perf_counter()
    for _ in range(args.steps):
        u = oracle.run(c, u, 1)[0]
    dt = time.perf_counter() - t0
    v = gs.cells * args.steps / dt
    line = {"impl": "reference", "metric": headline_metric(args.scheme, args.grid),
            "value": v, "unit": "cell-updates/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "ellipsoidal-%d^3-WENO%d" % (args.grid, args.scheme), "grid": [args.grid] * 3,
                       "steps_per_timing": args.steps, "parallelism": "single"},
            "cpu_baseline": {"value": v, "unit": "cell-updates/s", "cores": oracle.max_threads(), "kind": "oracle",
                             "sample": "central %d^3 block of the %d^3 workload, %d RK3 steps"
                                       % (min(sub, args.grid), args.grid, args.steps)},
            "e2e": {"value": v, "unit": "cell-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def lumpy_on_device(g, seed, dev, width=0.5):
    """The seeded lumpy event (workloads.lumpy_params) evaluated on the GPU
    with torch as separable Gaussians: e = 0.1 + sum A gx(x) gy(y) gz(z), v = 0, n = e."""
    import torch
    import workloads as W
    centres, amps = W.lumpy_params(seed)
    ax = [torch.tensor(g.origin[d] + (np.arange(g.n[d]) + 0.5) * g.dx[d], device=dev) for d in range(3)]
    e = torch.full((g.n[2], g.n[1], g.n[0]), 0.1, dtype=torch.float64, device=dev)
    for c, A in zip(centres, amps):
        gx = torch.exp(-(ax[0] - c[0]) ** 2 / (2 * width * width))
        gy = torch.exp(-(ax[1] - c[1]) ** 2 / (2 * width * width))
        gz = torch.exp(-(ax[2] - c[2]) ** 2 / (2 * width * width))
        e += float(A) * gz[:, None, None] * gy[None, :, None] * gx[None, None, :]
    z = torch.zeros_like(e)
    return torch.stack([e, z, z, z, e]).contiguous()


def batched_vs_looped(dev, stream, barrier, steps, warmup, events=256):
    """The event-by-event configuration: 256 seeded lumpy events, per-axis
    sizes U{48..160}, WENO5, 100 RK3 steps each.  Times `steps` steps of (a)
    the batched path (per stage a z pass over all events and one persistent
    launch over the tile work-list, each step one graph replay) and (b) a loop
    of the single-grid path (also graph-replayed) over the same events;
    events/s counts events finishing all 100 steps at the measured rate."""
    import torch
    import workloads as W
    from paper_1604_03360_gb300 import Hydro, HydroBatch
    sizes = W.batch_sizes(events)
    grids = [W.batch_grid(i, sizes) for i in range(events)]
    cells = sum(g.cells for g in grids)
    out = {"workload": "%d lumpy events, per-axis sizes U{48..160}, WENO5, 100 RK3 steps" % events,
           "events": events, "cells": cells, "steps_timed": steps}
    b = HydroBatch(grids, stream=stream)
    for i, g in enumerate(grids):
        b.set_primitive(i, lumpy_on_device(g, 1604 + i, dev))
    tune_ms = b.autotune()
    b.step(warmup)
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    b.step(steps)                 # the production path: one graph replay per step
    e1.record(stream)
    barrier()
    b.sync()
    tb = e0.elapsed_time(e1) / 1e3 / steps
    kms = b.profile_step(1)       # per-kernel breakdown of one more step (direct launches)
    out["batched"] = {"ms_per_step": 1e3 * tb, "events_per_s": events / (100 * tb), "cell_updates_per_s": cells / tb,
                      "launch": list(b.launch()), "autotune_stage1_ms": tune_ms,
                      "stage_ms_profiled": float(kms[1:4].sum()) / 3,
                      "gpu_launches_per_step": b.kernels_per_step()}
    b.close()
    del b
    torch.cuda.empty_cache()
    hs = []
    for i, g in enumerate(grids):
        h = Hydro.from_grid(g, stream=stream)
        h.set_primitive(lumpy_on_device(g, 1604 + i, dev))
        hs.append(h)
    loop_launches = sum(h.kernels_per_step() for h in hs)
    for _ in range(warmup):
        for h in hs:
            h.step(1)
    barrier()
    e0.record(stream)
    for _ in range(steps):
        for h in hs:
            h.step(1)
    e1.record(stream)
    barrier()
    for h in hs:
        h.sync()
    tl = e0.elapsed_time(e1) / 1e3 / steps
    out["looped"] = {"ms_per_step": 1e3 * tl, "events_per_s": events / (100 * tl), "cell_updates_per_s": cells / tl,
                     "gpu_launches_per_step": loop_launches}
    out["batched_over_looped"] = tl / tb
    for h in hs:
        h.close()
    torch.cuda.empty_cache()
    return out


def musta_force_256(dev, stream, barrier, grid, with_cpu):
    """The paper's second scheme (Sec. 1.1): MUSCL (minmod) + 2-stage
    MUSTA-FORCE on the same ellipsoidal workload; and, for the paper's only
    published comparison (the GPU program ~200x faster than a single-threaded
    CPU program for MUSTA-FORCE, Sec. 2), the oracle's MUSTA-FORCE on ONE host
    thread over a bounded 48^3 central block."""
    import torch
    from paper_1604_03360_gb300 import Hydro
    g, w = workload(5, grid)
    g.scheme, g.limiter, g.musta_stages = 2, 0, 2
    h = Hydro.from_grid(g, stream=stream)
    h.set_primitive(torch.from_numpy(w).to(dev))
    h.autotune()
    h.step(3)
    barrier()
    a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a0.record(stream)
    km = h.profile_step(3)
    a1.record(stream)
    barrier()
    h.sync()
    el = a0.elapsed_time(a1) / 1e3
    out = {"value": g.cells * 3 / el, "unit": "cell-updates/s", "steps": 3, "limiter": "minmod",
           "musta_stages": 2, "ms_per_step": 1e3 * el / 3, "launch": h.launch(),
           "stage_ms": float(km[1:4].sum()) / 9}
    h.close()
    if with_cpu:
        import oracle
        oracle.build()
        gs, ws = cpu_sample(5, grid, 48)
        c = oracle.make_cfg(gs.n, gs.dx, scheme=2, cfl=gs.cfl, limiter=0, musta_k=2)
        oracle.set_threads(1)
        t0 = time.perf_counter()
        oracle.run(c, oracle.prim2con(ws), 1)
        dt1 = time.perf_counter() - t0
        oracle.set_threads(0)
        v1 = gs.cells / dt1
        out["single_thread_oracle"] = {"value": v1, "unit": "cell-updates/s", "cores": 1, "kind": "oracle",
                                       "sample": "1 RK3 step of the central 48^3 block (%.1f s)" % dt1}
        out["gpu_over_single_thread_cpu"] = out["value"] / v1
    return out


def slabs_256(dev, stream, barrier, scheme, grid, variant, nslabs=4, steps=3, warmup=2):
    """The benchmark grid cut into z-slabs on this one GPU (halo handles,
    ghost planes exchanged device to device and speeds max-reduced between
    RK stages): throughput against the whole grid, and whether the final
    state is bit-identical to the whole grid's after the same steps."""
    import torch
    from paper_1604_03360_gb300 import Hydro
    from paper_1604_03360_gb300.domain import LocalExchange, SlabDomain, split_grid
    g, w = workload(scheme, grid)
    wd = torch.from_numpy(w).to(dev)
    slabs, bounds = split_grid(g, nslabs, stream=stream)
    for s, (z0, z1) in zip(slabs, bounds):
        s.set_launch(variant)
        s.set_primitive(wd[:, z0:z1].contiguous())
    dom = SlabDomain(LocalExchange(slabs, g.bc[2], device=dev))
    dom.loaded()
    dom.step(warmup)
    barrier()
    a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a0.record(stream)
    dom.step(steps)
    a1.record(stream)
    barrier()
    el = a0.elapsed_time(a1) / 1e3
    got = torch.cat([s.get_state(torch.empty((5, z1 - z0) + w.shape[2:], dtype=torch.float64, device=dev))
                     for s, (z0, z1) in zip(slabs, bounds)], dim=1)
    for s in slabs:
        s.close()
    h = Hydro.from_grid(g, stream=stream)
    h.set_launch(variant)
    h.set_primitive(wd)
    h.step(warmup + steps)
    ref = h.get_state(torch.empty_like(wd))
    h.close()
    barrier()
    G = {5: 3, 7: 4}[scheme]
    return {"value": g.cells * steps / el, "unit": "cell-updates/s", "slabs": nslabs, "steps": steps,
            "ms_per_step": 1e3 * el / steps, "bounds": bounds,
            "ghost_block_bytes": 9 * G * grid * grid * 8, "ghost_copies_per_stage": 4 * nslabs - 2,
            "bit_identical_to_whole_grid": bool(torch.equal(got, ref))}


def adjoint_96(dev, stream, barrier):
    """Adjoint configuration: 96^3 lumpy event (seed 1604), WENO5, 50 RK3 steps
    with a checkpoint every 10; gradient of eps_2 with respect to the initial
    state.  Times the recorded forward and the reverse sweep."""
    import torch
    import workloads as W
    from paper_1604_03360_gb300 import Hydro
    g, w = W.lumpy(n=(96, 96, 96), seed=1604)
    h = Hydro.from_grid(g, stream=stream)
    wd = torch.from_numpy(w).to(dev)
    h.set_primitive(wd)
    h.autotune()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    lam = torch.empty_like(wd)
    grad = torch.empty_like(wd)
    uN = torch.empty_like(wd)
    out = {}
    for rep in range(2):                       # first pass warms up
        h.set_primitive(wd)
        barrier()
        ev[0].record(stream)
        h.forward_record(50, 10)
        ev[1].record(stream)
        h.get_state(uN)
        eps = h.eps2(uN, lam)
        barrier()
        ev[1].synchronize()
        t_fwd = ev[0].elapsed_time(ev[1])
        ev[0].record(stream)
        h.adjoint(lam, grad)
        ev[2].record(stream)
        barrier()
        t_adj = ev[0].elapsed_time(ev[2])
        out = {"workload": "96^3 lumpy (seed 1604), WENO5, 50 RK3 steps, checkpoint every 10, d eps_2 / d u_0",
               "eps2": eps, "forward_record_ms": t_fwd, "adjoint_ms": t_adj,
               "adjoint_over_forward": t_adj / t_fwd,
               "cell_updates_per_s_forward": g.cells * 50 / (t_fwd * 1e-3),
               "gradient_norm": float(grad[0].norm())}
    # context, not the configuration: one segment of 50 steps (every stage
    # input kept by the recorded forward, about 9.6 GB), so the reverse sweep
    # recomputes nothing and times the stage adjoints alone
    from paper_1604_03360_gb300 import HydroError
    grad1 = torch.empty_like(wd)
    try:
        h.set_primitive(wd)
        h.forward_record(50, 50)              # untimed: sizes the workspace for one segment
        h.set_primitive(wd)
        barrier()
        ev[0].record(stream)
        h.forward_record(50, 50)
        ev[1].record(stream)
        h.get_state(uN)
        h.eps2(uN, lam)
        barrier()
        t_fwd1 = ev[0].elapsed_time(ev[1])
        ev[0].record(stream)
        h.adjoint(lam, grad1)
        ev[2].record(stream)
        barrier()
        t_adj1 = ev[0].elapsed_time(ev[2])
        out["one_segment"] = {"checkpoint_every": 50, "forward_record_ms": t_fwd1, "adjoint_ms": t_adj1,
                              "adjoint_over_forward": t_adj1 / t_fwd1,
                              "gradient_bitwise_equal": bool(torch.equal(grad1, grad))}
    except HydroError as e:                   # e.g. no room for the 9.6 GB workspace
        out["one_segment"] = {"checkpoint_every": 50, "error": str(e)}
    h.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--scheme", type=int, default=7, choices=[5, 7])
    ap.add_argument("--grid", type=int, default=256, help="cells per axis (256: the benchmark workload)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the WENO5 and e2e extras")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-vs-looped ensemble")
    ap.add_argument("--batch-events", type=int, default=256)
    ap.add_argument("--charwise", action="store_true",
                    help="headline run with characteristic-wise WENO (profiling; the metric stays component-wise)")
    ap.add_argument("--split", type=int, default=0, choices=[0, 1],
                    help="headline run with local Lax-Friedrichs splitting (profiling; the metric stays global LF)")
    ap.add_argument("--nq", type=int, default=1, choices=[1, 2, 3],
                    help="headline run with this many charges (profiling; the metric stays one charge)")
    ap.add_argument("--launch", type=int, default=None,
                    help="force this stage-kernel launch variant instead of autotuning (profiling)")
    ap.add_argument("--only", choices=["adjoint", "batch"], default=None,
                    help="run one extra measurement alone and print it (for profiling)")
    args = ap.parse_args()
    if args.impl == "reference":
        return reference_arm(args)
    if args.only == "adjoint":
        import torch
        from paper_1604_03360_gb300 import build as B
        B.build()
        torch.cuda.set_device(0)
        stream = torch.cuda.current_stream()
        print(json.dumps({"adjoint_96": adjoint_96(torch.device("cuda", 0), stream, torch.cuda.synchronize)}),
              flush=True)
        return
    if args.only == "batch":
        import torch
        from paper_1604_03360_gb300 import build as B
        B.build()
        torch.cuda.set_device(0)
        stream = torch.cuda.current_stream()
        print(json.dumps({"batched_vs_looped": batched_vs_looped(torch.device("cuda", 0), stream, torch.cuda.synchronize,
                                                                 10, 3, args.batch_events)}), flush=True)
        return

    import torch
    from paper_1604_03360_gb300 import Hydro
    from paper_1604_03360_gb300 import build as B
    B.build()
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
        pg = dist

    def barrier():
        if pg is not None:
            pg.barrier()
        torch.cuda.synchronize()

    stream = torch.cuda.current_stream()
    g, w = workload(args.scheme, args.grid)
    g.charwise = 1 if args.charwise else 0
    g.split = args.split
    if args.nq > 1:
        import workloads as W
        g.nq = args.nq
        w = W.with_charges(g, w, args.nq)
    cells = g.cells
    h = Hydro.from_grid(g, stream=stream)
    w_dev = torch.from_numpy(w).to(dev)
    h.set_primitive(w_dev)
    if args.launch is None:
        tuned_ms = h.autotune()
    else:
        h.set_launch(args.launch)
        tuned_ms = None
    launch = h.launch()
    h.step(args.warmup)
    torch.cuda.synchronize()
    h.sync()

    # ---- timed region: K steps, per-kernel CUDA events on the launching stream
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        e0.record(stream)
        kms = h.profile_step(args.steps)
        e1.record(stream)
        barrier()
    el = e0.elapsed_time(e1) / 1e3
    h.sync()
    step_launches = h.kernels_per_step()
    t_all = torch.tensor([el], device=dev)
    if pg is not None:
        pg.all_reduce(t_all, op=pg.ReduceOp.MAX)
    tmax = float(t_all.item())
    value = world * cells * args.steps / tmax
    stage_ms = float(kms[1:4].sum()) / (3 * args.steps)
    flops = FLOPS_PER_CELL_STAGE[args.scheme] * cells
    achieved = flops / (stage_ms * 1e-3) / 1e12
    peaks = load_peaks()
    from paper_1604_03360_gb300 import measure_fp64_peak
    fp64_inst_peak = measure_fp64_peak(stream) / 1e12    # FP64 FMA (= FP64 pipe issue slots) per second, T/s
    fp64_peak = 2.0 * fp64_inst_peak                     # TFLOP/s, FMA = 2 flops
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    hbm_achieved = HBM_BYTES_PER_CELL_UPDATE * (cells * args.steps / el) / 1e9

    # ---- end to end through the C ABI with pinned host buffers: every step
    # copies its input state in from host memory and its result out to host
    # memory (hydro_run_many: each step one item, copies double-buffered
    # against the steps); the serial form (set_state, step, get_state per
    # step, nothing overlapped) is reported beside it
    e2e = None
    if not args.no_extra:
        u_host = torch.empty((4 + args.nq,) + w.shape[1:], dtype=torch.float64).pin_memory()
        h.get_state(u_host)
        outs = [torch.empty_like(u_host).pin_memory() for _ in range(2)]
        h.run_many([u_host] * 2, outs, nsteps=1)          # first call: staging buffers
        barrier()
        t0 = time.perf_counter()
        h.run_many([u_host] * args.steps, [outs[i % 2] for i in range(args.steps)], nsteps=1)
        barrier()
        te = time.perf_counter() - t0
        t0 = time.perf_counter()
        for _ in range(args.steps):
            h.set_state(u_host)
            h.step(1)
            h.get_state(outs[0])
        barrier()
        ts = time.perf_counter() - t0
        t_e = torch.tensor([te, ts], device=dev)
        if pg is not None:
            pg.all_reduce(t_e, op=pg.ReduceOp.MAX)
        nbytes = (4 + args.nq) * cells * 8
        e2e = {"value": world * cells * args.steps / float(t_e[0].item()), "unit": "cell-updates/s",
               "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes,
               "api": "hydro_run_many (one item per step, pinned host buffers)",
               "serial_value": world * cells * args.steps / float(t_e[1].item()),
               "serial_api": "hydro_set_state + hydro_step + hydro_get_state per step"}

    extra = {}
    if not args.no_extra and args.scheme == 7:
        g5, w5 = workload(5, args.grid)
        h5 = Hydro.from_grid(g5, stream=stream)
        h5.set_primitive(torch.from_numpy(w5).to(dev))
        h5.autotune()
        h5.step(3)
        barrier()
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        k5 = h5.profile_step(args.steps)
        a1.record(stream)
        barrier()
        el5 = a0.elapsed_time(a1) / 1e3
        st5 = float(k5[1:4].sum()) / (3 * args.steps)
        inst5 = NCU_FP64_INST_PER_CELL_STAGE.get((5,) + tuple(h5.launch()[:3]))
        extra["weno5_256"] = {"value": cells * args.steps / el5, "unit": "cell-updates/s", "launch": h5.launch(),
                              "ms_per_step": 1e3 * el5 / args.steps, "stage_ms": st5,
                              "fp64_inst_per_cell_stage": inst5,
                              "fp64_pipe_frac": None if inst5 is None
                              else inst5 * cells / (st5 * 1e-3) / 1e12 / fp64_inst_peak,
                              "equivalent_tflops": FLOPS_PER_CELL_STAGE[5] * cells / (st5 * 1e-3) / 1e12,
                              "hbm_frac": HBM_BYTES_PER_CELL_UPDATE * cells * args.steps / el5 / 1e9 / hbm_peak}
        h5.close()
    h.close()
    if not args.no_extra:
        # local Lax-Friedrichs splitting, same workload and scheme
        gl, wl = workload(args.scheme, args.grid)
        gl.split = 1
        hl = Hydro.from_grid(gl, stream=stream)
        hl.set_primitive(torch.from_numpy(wl).to(dev))
        hl.autotune()
        hl.step(3)
        barrier()
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        kl = hl.profile_step(3)
        a1.record(stream)
        barrier()
        hl.sync()
        ell = a0.elapsed_time(a1) / 1e3
        extra["local_lf_256"] = {"value": cells * 3 / ell, "unit": "cell-updates/s", "steps": 3,
                                 "ms_per_step": 1e3 * ell / 3, "launch": hl.launch(),
                                 "stage_ms": float(kl[1:4].sum()) / 9,
                                 "over_componentwise": (float(kl[1:4].sum()) / 9) / stage_ms}
        hl.close()
    if not args.no_extra:
        # characteristic-wise WENO (global LF), same workload and scheme
        gc, wc = workload(args.scheme, args.grid)
        gc.charwise = 1
        hc = Hydro.from_grid(gc, stream=stream)
        hc.set_primitive(torch.from_numpy(wc).to(dev))
        hc.autotune()
        hc.step(3)
        barrier()
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        kc = hc.profile_step(3)
        a1.record(stream)
        barrier()
        hc.sync()
        elc = a0.elapsed_time(a1) / 1e3
        extra["charwise_%d" % args.grid] = {"value": cells * 3 / elc, "unit": "cell-updates/s", "steps": 3,
                                            "ms_per_step": 1e3 * elc / 3, "launch": hc.launch(),
                                            "stage_ms": float(kc[1:4].sum()) / 9,
                                            "over_componentwise": (float(kc[1:4].sum()) / 9) / stage_ms}
        hc.close()
    if not args.no_extra:
        # general EOS p = cs2 (e - m n_1) with m = 1 (iterative primitive recovery), same workload
        gg, wg = workload(args.scheme, args.grid)
        gg.mass = 1.0
        hg = Hydro.from_grid(gg, stream=stream)
        hg.set_primitive(torch.from_numpy(wg).to(dev))
        hg.autotune()
        hg.step(3)
        barrier()
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        kg = hg.profile_step(3)
        a1.record(stream)
        barrier()
        hg.sync()
        elg = a0.elapsed_time(a1) / 1e3
        extra["gas_eos_%d" % args.grid] = {"value": cells * 3 / elg, "unit": "cell-updates/s", "steps": 3,
                                           "eos": "p = cs2 (e - m n), cs2 = 1/3, m = 1",
                                           "ms_per_step": 1e3 * elg / 3, "launch": hg.launch(),
                                           "stage_ms": float(kg[1:4].sum()) / 9,
                                           "over_default_eos": (float(kg[1:4].sum()) / 9) / stage_ms}
        hg.close()
    if not args.no_extra:
        # three conserved charges (state of 7 fields), same workload and scheme
        import workloads as W
        gq, wq = workload(args.scheme, args.grid)
        gq.nq = 3
        hq = Hydro.from_grid(gq, stream=stream)
        hq.set_primitive(torch.from_numpy(W.with_charges(gq, wq, 3)).to(dev))
        hq.autotune()
        hq.step(3)
        barrier()
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        kq = hq.profile_step(3)
        a1.record(stream)
        barrier()
        hq.sync()
        elq = a0.elapsed_time(a1) / 1e3
        extra["charges3_256"] = {"value": cells * 3 / elq, "unit": "cell-updates/s", "steps": 3, "fields": 7,
                                 "ms_per_step": 1e3 * elq / 3, "launch": hq.launch(),
                                 "stage_ms": float(kq[1:4].sum()) / 9}
        hq.close()
    if not args.no_extra:
        extra["musta_force_256"] = musta_force_256(dev, stream, barrier, args.grid, rank == 0 and not args.no_cpu_baseline)
    if not args.no_extra and not args.no_batch:
        extra["batched_vs_looped"] = batched_vs_looped(dev, stream, barrier, 10, 3, args.batch_events)
    if not args.no_extra:
        extra["adjoint_96"] = adjoint_96(dev, stream, barrier)
    if not args.no_extra:
        extra["slabs4_%d" % args.grid] = slabs_256(dev, stream, barrier, args.scheme, args.grid, launch[0])

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        # about 10 s of oracle work on the host cores
        sub = min(args.grid, 256 if args.scheme == 5 else 208)
        v, secs, cores = time_oracle(args.scheme, 1, sub, args.grid)
        cpu = {"value": v, "unit": "cell-updates/s", "cores": cores, "kind": "oracle",
               "sample": "1 RK3 step of the central %d^3 block of the %d^3 workload (%.1f s)"
               % (sub, args.grid, secs)}

    # the ncu figures hold for the launch they were captured on
    key = (args.scheme,) + tuple(launch[:3])
    other = args.charwise or args.split or args.nq > 1
    inst = None if other else NCU_FP64_INST_PER_CELL_STAGE.get(key)
    traffic = None if other or key not in NCU_DRAM_BYTES_PER_CELL_STAGE else \
        NCU_DRAM_BYTES_PER_CELL_STAGE[key] * cells
    inst_rate = None if inst is None else inst * cells / (stage_ms * 1e-3) / 1e12
    if rank == 0:
        line = {
            "metric": headline_metric(args.scheme, args.grid),
            "value": value, "unit": "cell-updates/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * tmax / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "ellipsoidal-%d^3-WENO%d%s%s" % (args.grid, args.scheme,
                                                                    "-characteristic" if args.charwise else "",
                                                                    "-localLF" if args.split else "")
                       + ("-%dcharges" % args.nq if args.nq > 1 else ""),
                       "grid": [args.grid] * 3,
                       "steps_per_timing": args.steps, "parallelism": "replicas" if world > 1 else "single",
                       "l2": "state %.2f GB > 129 MB L2: no flush needed" % (27 * 8 * cells / 1e9),
                       "launch": {"variant": launch[0], "tile": [launch[1], launch[2]], "z_chunk": launch[3],
                                  "autotune_stage_ms": tuned_ms}},
            "roofline": {"bound": "alu", "achieved": inst_rate, "peak": fp64_inst_peak,
                         "unit": "FP64 Tinst/s", "frac": None if inst_rate is None else inst_rate / fp64_inst_peak,
                         "traffic": traffic,
                         "traffic_source": "ncu dram__bytes_read+write of the 128^3 stage launches of the same "
                                           "variant (all launches of a stage, mean of stages 1-3), scaled by cells",
                         "fp64_inst_per_cell_stage": inst,
                         "achieved_source": "executed FP64 instructions per cell and stage (ncu, thread-level DFMA + "
                                            "DADD + DMUL of all launches of a stage on the 128^3 case of this launch) "
                                            "x cells / stage time (CUDA events); peak = FP64 FMA issue rate measured "
                                            "in this run (hydro_measure_fp64_peak)",
                         "ncu_fp64_pipe_busy": None if other else NCU_FP64_PIPE_BUSY.get(key),
                         "equivalent_tflops": achieved, "equivalent_tflops_of_fp64_peak": achieved / fp64_peak,
                         "equivalent_count": "%d flops per cell-stage, every face reconstructed from its own stencil "
                                             "(FMA = 2); the kernels share differences between faces and run some "
                                             "products on the integer pipe, so this rate can exceed the FP64 peak"
                                             % FLOPS_PER_CELL_STAGE[args.scheme],
                         "kernel": ("x, y, z face passes + stage_combine_kernel"
                                    if launch[0] in {5: (12, 13, 14), 7: (13, 14, 15, 16, 17)}[args.scheme]
                                    else "zflux_kernel + stage_kernel") + " (WENO%d)" % args.scheme,
                         "stage_ms": stage_ms,
                         "peak_source": "FP64 FMA probe kernel measured in this run (hydro_measure_fp64_peak); "
                                        "MEASURED_PEAKS.json has no FP64 figure; nominal 152 SM x 2 DFMA/clk x "
                                        "2.07 GHz = 0.629 T/s"},
            "hbm": {"achieved_gbs": hbm_achieved, "peak_gbs": hbm_peak, "frac": hbm_achieved / hbm_peak,
                    "bytes_per_cell_update": HBM_BYTES_PER_CELL_UPDATE, "peak_source": "MEASURED_PEAKS.json"},
            "e2e": e2e,
            "cpu_baseline": cpu,
            "clocks": clk.summary(),
            "gpu_launches": step_launches * args.steps + 1,   # + the t_end setter
            "kernel_ms_per_step": {"step_begin": kms[0] / args.steps, "stage1": kms[1] / args.steps,
                                   "stage2": kms[2] / args.steps, "stage3": kms[3] / args.steps,
                                   "step_end": kms[4] / args.steps},
        }
        line.update(extra)
        print(json.dumps(line), flush=True)
    if pg is not None:
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
