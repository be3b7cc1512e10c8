"""Benchmark: cell x band x direction updates/s and time-to-converge of the
steady nongray phonon-BTE hot path on one GB300 (or N replicas).

Workload (one "step"): the 2D nongray square -- 128 x 128 cells on
2 um x 2 um, 15 synthetic silicon-like bands, 64 directions (8 Gauss-Legendre
polar x 8 azimuths), left wall 310 K, right wall 300 K, top/bottom diffuse --
solved from T = 300 K to eps_T < 1e-6 with FP32 sweeps and FP64 reductions
(forward), followed by the discrete adjoint of the probe-temperature misfit
(64 seeded probes) to a relative change of 1e-6.  ``value`` counts the
updates of every forward and adjoint source iteration.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]

With torchrun (N > 1) every rank solves its own replica of the workload (the
single-instance path does not shard; "replicas only").
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "square2d_128x128_B15_D64_fwd+adj_eps1e-6"
METRIC = "cell*band*direction updates/s (fwd+adj to eps_T<1e-6, FP32 sweeps)"
TOL = 1e-6
L2_FLUSH_BYTES = 512 << 20
TIME_EVERY = 8   # sweeps timed with CUDA events: one in every TIME_EVERY iterations


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def probes_and_obs(p, seed=20250330):
    rng = np.random.Generator(np.random.PCG64(seed))
    act = np.flatnonzero(p.mask)
    probes = np.sort(rng.choice(act, size=64, replace=False))
    T_obs = 300.0 + rng.uniform(0.0, 10.0, probes.size)
    return probes, T_obs


class ClockSampler:
    """nvidia-smi clocks/throttle sampling during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(self.dev)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for name, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# dram__bytes_read.sum + dram__bytes_write.sum of one launch, from the ncu
# capture summarised in profiles/ (keyed by the exact kernel; a kernel changed
# since the capture has no entry)
NCU_TRAFFIC = {
    # profiles/sweep2dp_square128.md: 177.9 KB read + 0.8 KB written (128 x 128 square, tile 3:4:4)
    ("sweep2dp_kernel<float, 4, 8, 0, 0>", "3:4:4"): 178688,
}


def measured_hbm_peak():
    """HBM copy bandwidth (GB/s) measured on this GPU pool, else the fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            v = float(json.load(f)["hbm_gbs"])
        return v, "measured: MEASURED_PEAKS.json hbm_gbs (STREAM-style copy)"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback: 6.8 TB/s"


def timed_sweep_scale(stats):
    """Timed sweeps are a sample (one in TIME_EVERY per poll interval): the
    factor from the sampled sweep time to all sweeps of these solves."""
    timed = sum(s["sweep_launches"] for s in stats)
    total = sum(s["iterations"] for s in stats)
    return total / timed if timed else 0.0


def sweep_kernel_name(p, st):
    """The sweep kernel a solve ran (forward and adjoint share it), as ncu
    names it."""
    dw = st["dirs_per_lane"]
    if st["tile_kind"] == 3:
        return f"sweep2dp_kernel<float, {dw}, 8, 0, 0>"
    if st["tile_kind"] == 2:
        rb = next(r for r in (1, 2, 3, 4, 5) if 32 * r >= p.n[1])
        return f"sweep2d_kernel<float, {dw}, {rb}, false>"
    return f"sweep_kernel<float, {dw}, 1, false, false>"


def cpu_baseline_oracle(iters: int = 20):
    """The FP64 oracle (single thread) on a bounded sample of the workload:
    `iters` forward source iterations of the full 128x128 square."""
    import bte_inputs as bi
    import oracle
    p = bi.square_2d()
    t0 = time.perf_counter()
    oracle.solve(p, max_iter=iters, tol=0.0)
    dt = time.perf_counter() - t0
    units = iters * p.n_active * p.B * p.D
    return {"value": units / dt, "unit": "updates/s", "cores": 1, "kind": "oracle",
            "sample": f"{iters} forward source iterations of the full 128x128x15x64 square "
                      f"({units:.3g} updates, {dt:.1f} s, FP64, 1 thread)"}


def run_reference(args, ws, rank):
    """Reference arm: the FP64 CPU oracle as it stands, timed on the host."""
    if rank != 0:
        return 0
    import bte_inputs as bi
    import oracle
    oracle.build()
    p = bi.square_2d()
    k_iter = 2
    units_step = k_iter * p.n_active * p.B * p.D
    for _ in range(args.warmup):
        oracle.solve(p, max_iter=1, tol=0.0)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.solve(p, max_iter=k_iter, tol=0.0)
    dt = time.perf_counter() - t0
    val = units_step * args.steps / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": "updates/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "reference": "FP64 CPU oracle (oracle/bte_oracle.c), 1 thread",
                   "step": f"{k_iter} forward source iterations (bounded sample)"},
        "cpu_baseline": {"value": val, "unit": "updates/s", "cores": 1, "kind": "oracle",
                         "sample": f"{args.steps} steps x {k_iter} source iterations of the full square"},
        "e2e": {"value": val, "unit": "updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "gpu_launches": 0,
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-iters", type=int, default=20)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--store-e-every-iter", action="store_true")
    ap.add_argument("--tile", default="0:0:0",
                    help="sweep tile kind:dirs_per_lane:dirs_per_cta (0:0:0 = autotuned); profiling runs pin "
                         "the tile the autotuner chose, since timings under a profiler are not representative")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    ws, rank, local = dist_env()

    if args.impl == "reference":
        return run_reference(args, ws, rank)

    import torch
    import torch.distributed as dist
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if ws > 1:
            dist.barrier()

    # the CPU baseline runs before any GPU work (no fork after CUDA init)
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_oracle(args.cpu_iters)

    import __graft_entry__
    __graft_entry__.build()
    import bte_inputs as bi
    import paper_2503_23657_gb300 as m

    p = bi.square_2d()
    probes, T_obs = probes_and_obs(p)
    probes_d = torch.as_tensor(probes, device="cuda")
    T_obs_d = torch.as_tensor(T_obs, device="cuda")
    plan = m.Plan(p)
    stream = torch.cuda.current_stream()
    sp = stream.cuda_stream
    T = torch.zeros(p.n_cells, dtype=torch.float64, device="cuda")
    g = torch.zeros(p.n_cells, dtype=torch.float64, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    per_update = p.n_active * p.B * p.D

    tile_kind, tile_dw, tile_cw = (int(x) for x in args.tile.split(":"))

    def step(T, g):
        rc, sf = plan.solve(T, precision=m.BTE_FP32, tol=TOL, max_iter=100000, stream=sp,
                            store_e_every_iter=args.store_e_every_iter, tile_kind=tile_kind,
                            dirs_per_lane=tile_dw, dirs_per_cta=tile_cw)
        g.zero_()
        g[probes_d] = T[probes_d] - T_obs_d
        rc, g_tau, g_Tw, g_Q, sa = plan.adjoint(g, tol=TOL, max_iter=100000)
        return sf, sa

    # the sweep of every 8th iteration of the timed steps is bracketed by CUDA
    # events on its stream (inside the captured graphs): the dominant kernel's
    # mean duration, sampled over the whole timed region
    plan.set_sweep_timing(TIME_EVERY)
    for _ in range(args.warmup):
        step(T, g)
    torch.cuda.synchronize()

    clocks = ClockSampler(torch.cuda.current_device())
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    torch.cuda.nvtx.range_push("bench_timed")   # lets a profiler select the timed steps
    times, fstats, astats = [], [], []
    for _ in range(args.steps):
        flush.fill_(1.0)   # evict the previous step's working set from L2
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sf, sa = step(T, g)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
        fstats.append(sf)
        astats.append(sa)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    barrier()
    clk = clocks.stop()

    units = sum((f["iterations"] + a["iterations"]) * per_update for f, a in zip(fstats, astats))
    t_total = sum(times) / 1e3
    t_max = t_total
    units_all = units
    if ws > 1:
        tt = torch.tensor([t_total], dtype=torch.float64, device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        uu = torch.tensor([units], dtype=torch.float64, device="cuda")
        dist.all_reduce(uu, op=dist.ReduceOp.SUM)
        t_max, units_all = float(tt), float(uu)
    value = units_all / t_max
    launches = sum(f["kernel_launches"] + a["kernel_launches"] for f, a in zip(fstats, astats))

    # forward-only and FP64 comparison (not part of the timed region)
    fwd_ups = statistics.median(f["updates_per_s"] for f in fstats)
    fwd_ms = statistics.median(f["seconds"] for f in fstats) * 1e3
    T64 = torch.zeros_like(T)
    plan.solve(T64, precision=m.BTE_FP64, tol=TOL, max_iter=100000, stream=sp)
    rc, s64 = plan.solve(T64, precision=m.BTE_FP64, tol=TOL, max_iter=100000, stream=sp)
    dT_fp64 = float((T - T64).abs().max() / T64.abs().max())

    plan.set_sweep_timing(0)
    # dominant kernel: the sweep (forward and adjoint launches of the same
    # kernel), its mean launch duration from the CUDA events of the timed steps
    fwd_sweep_s = sum(f["sweep_seconds"] for f in fstats)
    fwd_sweeps = sum(f["sweep_launches"] for f in fstats)
    adj_sweep_s = sum(a["sweep_seconds"] for a in astats)
    adj_sweeps = sum(a["sweep_launches"] for a in astats)
    sweep_ms = (fwd_sweep_s + adj_sweep_s) / (fwd_sweeps + adj_sweeps) * 1e3
    dw = fstats[-1]["dirs_per_lane"]
    kernel = sweep_kernel_name(p, fstats[-1])
    # algorithmic HBM bytes per cell x band x direction update: one FP32
    # write of e, plus per cell the T read (8 B) and S, q writes (32 B)
    # shared by its B x D updates
    bytes_per_update = 4.0 + 40.0 / (p.B * p.D)
    sweep_bytes = bytes_per_update * per_update
    achieved = sweep_bytes / (sweep_ms * 1e-3) / 1e9
    peak_hbm, peak_src = measured_hbm_peak()
    tile = f"{fstats[-1]['tile_kind']}:{dw}:{fstats[-1]['dirs_per_cta']}"
    traffic = NCU_TRAFFIC.get((kernel, tile))
    flops_per_update = 7.0   # 3 FMA + 1 MUL per update (upwind update + weighted sum)
    sm_count = torch.cuda.get_device_properties(0).multi_processor_count
    smax = 2070.0
    peak_fp32 = sm_count * 128 * 2 * smax * 1e6 / 1e12   # TFLOP/s, FP32 FMA pipes at max SM clock
    alu_achieved = flops_per_update * per_update / (sweep_ms * 1e-3) / 1e12
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak_hbm, "unit": "GB/s",
                "frac": achieved / peak_hbm, "traffic": traffic,
                "kernel": kernel, "tile": tile, "peak_source": peak_src,
                "algorithmic": f"{bytes_per_update:.4f} B x {per_update} cell*band*direction updates per launch "
                               f"(e write per update + per-cell T, S, q); the kernel itself keeps e on chip "
                               f"(e is regenerated once after convergence), so DRAM traffic is far lower",
                "sweep_ms": sweep_ms, "sweep_launches_timed": fwd_sweeps + adj_sweeps,
                "fwd_sweep_ms": fwd_sweep_s / max(fwd_sweeps, 1) * 1e3,
                "adj_sweep_ms": adj_sweep_s / max(adj_sweeps, 1) * 1e3,
                "sweep_share_of_step": (fwd_sweep_s * timed_sweep_scale(fstats) +
                                        adj_sweep_s * timed_sweep_scale(astats)) / t_total,
                "alu": {"achieved": alu_achieved, "peak": peak_fp32, "unit": "TFLOP/s",
                        "frac": alu_achieved / peak_fp32,
                        "peak_source": f"derived: {sm_count} SMs x 128 FP32 lanes x 2 flop x {smax:.0f} MHz"}}

    # end to end through the C ABI with host buffers (pinned), copies inside
    T_init_h = torch.full((p.n_cells,), 300.0, dtype=torch.float64).pin_memory()
    T_h = torch.zeros(p.n_cells, dtype=torch.float64).pin_memory()
    g_h = torch.zeros(p.n_cells, dtype=torch.float64).pin_memory()
    e2e_units, e2e_t = 0, 0.0
    for i in range(max(2, args.steps)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rc, sf = plan.solve(T_h, T_init=T_init_h, precision=m.BTE_FP32, tol=TOL, max_iter=100000, stream=sp,
                            tile_kind=tile_kind, dirs_per_lane=tile_dw, dirs_per_cta=tile_cw)
        g_h.zero_()
        g_h[probes] = T_h[probes] - torch.as_tensor(T_obs)
        rc, g_tau, g_Tw, g_Q, sa = plan.adjoint(g_h, tol=TOL, max_iter=100000)
        t1 = time.perf_counter()
        if i > 0:
            e2e_units += (sf["iterations"] + sa["iterations"]) * per_update
            e2e_t += t1 - t0
    e2e_value = e2e_units / e2e_t * (ws if ws > 1 else 1)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "updates/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_max * 1e3 / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "cells": p.n_cells, "bands": p.B, "directions": p.D,
                       "tol_eps_T": TOL, "l2": f"flushed before every step ({L2_FLUSH_BYTES >> 20} MB write)",
                       "parallelism": "replicas" if ws > 1 else "single",
                       "store_e_every_iter": bool(args.store_e_every_iter),
                       "tile": f"{fstats[-1]['tile_kind']}:{dw}:{fstats[-1]['dirs_per_cta']}"},
            "fwd_iterations": fstats[-1]["iterations"], "adj_iterations": astats[-1]["iterations"],
            "fwd_time_to_converge_ms": fwd_ms, "fwd_updates_per_s": fwd_ups,
            "fwd_adj_ms_per_step": statistics.median(times),
            "fp64_fwd_updates_per_s": s64["updates_per_s"], "fp64_fwd_time_to_converge_ms": s64["seconds"] * 1e3,
            "fp64_fwd_iterations": s64["iterations"], "speedup_fp32_vs_fp64_fwd": fwd_ups / s64["updates_per_s"],
            "T_fp32_vs_fp64_rel": dT_fp64,
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": "updates/s",
                    "h2d_bytes_per_step": 2 * 8 * p.n_cells, "d2h_bytes_per_step": 8 * p.n_cells + 8 * (p.B + 7)},
            "gpu_launches": launches,
            "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
