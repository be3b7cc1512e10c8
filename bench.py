"""Benchmark: cell x band x direction updates/s and time-to-converge of the
steady nongray phonon-BTE hot path on one GB300 (or N replicas).

Default workload (one "step"): the inverse FinFET-like problem -- a masked
160 x 80 x 64 grid (2.5 nm cells; substrate, oxide with tau x 0.1, a 20 nm x
40 nm fin, Joule source in the fin's top 10 nm), 15 synthetic silicon-like
bands, 128 directions (8 Gauss-Legendre polar x 16 azimuths), bottom face
isothermal, every other face diffuse -- solved from T = 300 K to eps_T < 1e-6
with FP32 sweeps and FP64 reductions (forward), followed by the discrete
adjoint of the misfit of 64 seeded probe temperatures to a relative change of
1e-6 (gradients w.r.t. the 15 tau_b, the substrate temperature and the source
amplitude).  ``value`` counts the updates of every forward and adjoint source
iteration.  The same line reports the batched ensemble (256 uneven 2D
squares) solved in FP32 and in FP64 on the GPU: the FP32 batched form's
speedup over the FP64 path and its error (``ensemble`` key).

Other workloads (--workload): ``square`` (2D nongray square 128^2, 64
directions, forward + adjoint), ``slab`` (1D gray slab, 200 cells, FP64 to
1e-10), ``hotspot`` (3D cube 64^3, 15 bands x 128 directions, Gaussian
source, forward to 1e-6), ``ensemble`` (256 uneven 2D squares solved as one
batch, forward to 1e-6 per instance).

  python bench.py [--gpus N --steps K --warmup W] [--impl reference] [--workload W]

With torchrun (N > 1) every rank solves its own replica of the workload (the
single-instance path does not shard; "replicas only").
"""
from __future__ import annotations

import argparse
import json
import re
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cell*band*direction updates/s (fwd+adj to eps_T<1e-6, FP32 sweeps)"

# workload -> (problem maker, name, tol, FP64?, adjoint?)
WORKLOADS = {
    "square": (lambda bi: bi.square_2d(), "square2d_128x128_B15_D64_fwd+adj_eps1e-6", 1e-6, False, True),
    "slab": (lambda bi: bi.gray_slab(), "slab1d_200_B1_D16_fwd_eps1e-10_fp64", 1e-10, True, False),
    "hotspot": (lambda bi: bi.hotspot_3d(), "hotspot3d_64^3_B15_D128_fwd_eps1e-6", 1e-6, False, False),
    "finfet": (lambda bi: bi.finfet_3d(), "finfet3d_160x80x64_B15_D128_fwd+adj_eps1e-6", 1e-6, False, True),
    "finfet_specular": (lambda bi: bi.finfet_specular_3d(),
                        "finfet3d_specbase_160x80x64_B15_D128_fwd+adj_eps1e-6", 1e-6, False, True),
    "ensemble": (lambda bi: bi.ensemble_2d(), "ensemble2d_256x(32..160)^2_B15_D64_fwd_eps1e-6", 1e-6, False, False),
    "hotspot_transient": (lambda bi: bi.hotspot_3d(), "hotspot3d_64^3_B15_D128_transient_10x10ps_eps1e-6", 1e-6,
                          False, False),
}
# implicit-Euler workloads: time step (s) and steps per bench step, each step
# solved to eps_T < tol from the previous one (the paper's Conclusion names
# transient transport as its extension)
TRANSIENT = {"hotspot_transient": (1e-11, 10)}
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


# dram__bytes_read.sum + dram__bytes_write.sum of one launch of the sweep
# kernel, from an ncu capture of that kernel (one launch, --clock-control
# none), keyed by the kernel, the tile and a fingerprint of the kernel's
# sources at capture time: a kernel edited since its capture has no entry and
# reports null.  Full-size captures where the launch fits the capture rules;
# otherwise a capture with fewer bands, scaled to all bands (traffic grows in
# proportion to the bands: every band is an independent set of CTAs).
NCU_TRAFFIC = {
    # FinFET 160x80x64, 15 bands, forward launch, full size (one-pass capture),
    # mean of two launches: 1203.2 MB read + 2193.8 MB written (two 8-warp
    # CTAs per SM: the per-CTA wrap planes of all 240 resident CTAs and the
    # partial sums leave L2)
    ("sweep3dp_kernel<float, 8, 1, 0, 1, 0>", "3:8:8:2:4:2", "4ca13341a79c"): 3396967040,
    # 64^3 hotspot, 15 bands, forward launch, full size, mean of two launches:
    # 66.5 MB read + 251.7 MB written
    ("sweep3dp_kernel<float, 8, 1, 0, 0, 0>", "3:8:8:2:4:1", "4ca13341a79c"): 318187904,
    # FinFET with specular base side faces, forward launch, full size, mean
    # of two launches: 1328.4 MB read + 2366.5 MB written
    ("sweep3dp_kernel<float, 8, 1, 0, 1, 1>", "3:8:8:2:4:2", "4ca13341a79c"): 3694982656,
}
KERNEL_SOURCES = {
    "sweep3dp_kernel": ["sweep3dp.cuh", "bte_internal.cuh", "finalize.cuh", "tma.cuh"],
    "sweep2dp_kernel": ["sweep2dp.cuh", "bte_internal.cuh", "finalize.cuh", "tma.cuh"],
}


def kernel_fingerprint(kernel):
    """Short hash of the sources a sweep kernel is compiled from."""
    import hashlib
    base = kernel.split("<")[0]
    files = KERNEL_SOURCES.get(base)
    if not files:
        return None
    h = hashlib.sha1()
    for f in files:
        with open(os.path.join(ROOT, "paper_2503_23657_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:12]


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
    phi = 0 if p.phi is None or p.Q_amp == 0.0 else 1
    if st["tile_kind"] == 3 and p.dim == 3:
        spec = int(any(int(t) == 2 for t in p.bc_type[:6]))   # the variant with specular faces
        return f"sweep3dp_kernel<float, {dw}, {phi}, 0, {int(st['lane_axis'] == 2)}, {spec}>"
    if st["tile_kind"] == 3:
        return f"sweep2dp_kernel<float, {dw}, 8, {phi}, 0, {st['source_staged']}>"
    if st["tile_kind"] == 2:
        rb = next(r for r in (1, 2, 3, 4, 5) if 32 * r >= p.n[1])
        return f"sweep2d_kernel<float, {dw}, {rb}, false>"
    return f"sweep_kernel<float, {dw}, lz, {int(p.dim == 3)}, 0>"


def oracle_iters(units_per_iter, seconds=15.0, rate=4e7):
    """Source iterations of the oracle that take about `seconds` on one core."""
    return max(1, int(round(seconds * rate / max(units_per_iter, 1))))


def oracle_sample(p, seconds, rate=4e7):
    """A bounded sample of workload `p` for the single-thread oracle: whole
    source iterations of the full problem when one takes less than `seconds`,
    else one iteration of the problem restricted to its first bands (every
    band is an independent set of sweeps; at least one band).  Returns the
    sampled problem, its iteration count and a description."""
    per_band = p.n_active * p.D
    if p.B * per_band <= seconds * rate:
        return p, oracle_iters(p.B * per_band, seconds, rate), "all bands"
    nb = max(1, min(p.B, int(seconds * rate / per_band)))
    q = p.copy(C=p.C[:nb], v=p.v[:nb], tau=p.tau[:nb])
    return q, 1, f"the first {nb} of {p.B} bands"


def oracle_iterations(q, k, transient=None):
    """k source iterations of the oracle on problem q: of the steady problem,
    or of the first implicit-Euler step (transient = (dt, steps))."""
    import oracle
    if transient:
        oracle.transient(q, transient[0], 1, max_iter=k, tol=0.0)
    else:
        oracle.solve(q, max_iter=k, tol=0.0)


def cpu_baseline_oracle(probs, iters=0, transient=None):
    """The FP64 oracle (single thread) on a bounded sample of the workload:
    forward source iterations of (the first instances of) it, restricted to
    its first bands where one full iteration would take too long."""
    import oracle
    oracle.build()
    t0 = time.perf_counter()
    units = 0
    what = "all bands"
    for p in probs:
        q, k, what = oracle_sample(p, 15.0)
        k = iters or k
        oracle_iterations(q, k, transient)
        units += k * q.n_active * q.B * q.D
        if time.perf_counter() - t0 > 20.0:
            break
    dt = time.perf_counter() - t0
    return {"value": units / dt, "unit": "updates/s", "cores": 1, "kind": "oracle",
            "sample": f"{k} forward source iteration(s) of {len(probs) if len(probs) == 1 else 'the first'} "
                      f"instance(s) of the workload, {what} ({units:.3g} updates, {dt:.1f} s, FP64, 1 thread)"}


def run_reference(args, ws, rank):
    """Reference arm: the FP64 CPU oracle as it stands, timed on the host."""
    if rank != 0:
        return 0
    import bte_inputs as bi
    import oracle
    oracle.build()
    make, name, tol, fp64, adj = WORKLOADS[args.workload]
    probs = make(bi)
    probs = probs if isinstance(probs, list) else [probs]
    p, k_iter, what = oracle_sample(probs[0], 3.0)
    units_step = k_iter * p.n_active * p.B * p.D
    tr = TRANSIENT.get(args.workload)
    for _ in range(args.warmup):
        oracle_iterations(p, 1, tr)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle_iterations(p, k_iter, tr)
    dt = time.perf_counter() - t0
    val = units_step * args.steps / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": "updates/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": name, "reference": "FP64 CPU oracle (oracle/bte_oracle.c), 1 thread",
                   "step": f"{k_iter} forward source iteration(s) of {p.name}, {what} (bounded sample)"},
        "cpu_baseline": {"value": val, "unit": "updates/s", "cores": 1, "kind": "oracle",
                         "sample": f"{args.steps} steps x {k_iter} source iteration(s) of {p.name}, {what}"},
        "e2e": {"value": val, "unit": "updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "gpu_launches": 0,
    }
    print(json.dumps(line), flush=True)
    return 0


def roofline_object(kernel, tile, sweep_ms, updates_per_launch, B, D, extra):
    """The sweep's HBM-equivalent rate: algorithmic bytes per launch (one FP32
    e write per update + T, S, q per cell) over the measured launch time."""
    import torch
    bytes_per_update = 4.0 + 40.0 / (B * D)
    achieved = bytes_per_update * updates_per_launch / (sweep_ms * 1e-3) / 1e9
    peak_hbm, peak_src = measured_hbm_peak()
    flops_per_update = 7.0   # 3 FMA + 1 MUL per update (upwind update + weighted sum)
    sm_count = torch.cuda.get_device_properties(0).multi_processor_count
    smax = 2070.0
    peak_fp32 = sm_count * 128 * 2 * smax * 1e6 / 1e12
    alu_achieved = flops_per_update * updates_per_launch / (sweep_ms * 1e-3) / 1e12
    r = {"bound": "hbm", "achieved": achieved, "peak": peak_hbm, "unit": "GB/s", "frac": achieved / peak_hbm,
         "traffic": NCU_TRAFFIC.get((kernel, tile, kernel_fingerprint(kernel))), "kernel": kernel, "tile": tile,
         "kernel_sources": kernel_fingerprint(kernel), "peak_source": peak_src,
         "algorithmic": f"{bytes_per_update:.4f} B x {updates_per_launch} cell*band*direction updates per launch "
                        f"(e write per update + per-cell T, S, q); the kernel keeps e on chip (e is regenerated "
                        f"once after convergence), so DRAM traffic is far lower",
         "sweep_ms": sweep_ms,
         "alu": {"achieved": alu_achieved, "peak": peak_fp32, "unit": "TFLOP/s", "frac": alu_achieved / peak_fp32,
                 "peak_source": f"derived: {sm_count} SMs x 128 FP32 lanes x 2 flop x {smax:.0f} MHz"}}
    r.update(extra)
    return r


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="finfet", choices=sorted(WORKLOADS))
    ap.add_argument("--no-ensemble", action="store_true",
                    help="finfet: skip the FP32-vs-FP64 batched-ensemble comparison")
    ap.add_argument("--instances", type=int, default=256, help="ensemble: number of instances (a profiler "
                                                                  "capture uses a small batch)")
    ap.add_argument("--bands", type=int, default=0, help="keep only the first N bands (0 = all): the small "
                                                          "case of a workload for a full profiler capture")
    ap.add_argument("--cpu-iters", type=int, default=0, help="oracle iterations of the CPU baseline (0 = ~15 s)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 GPU comparison run")
    ap.add_argument("--store-e-every-iter", action="store_true")
    ap.add_argument("--tile", default="0:0:0:0",
                    help="sweep tile kind:dirs_per_lane:dirs_per_cta:source_staging[:warps_z[:lane_axis]] "
                         "(0:0:0:0 = autotuned; warps_z, lane_axis: the 3D plane-pipeline kernel's warps along "
                         "the plane axis and its row axis, 1 = y, 2 = z); "
                         "profiling runs pin the tile the autotuner chose, since timings under a profiler are "
                         "not representative")
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

    import bte_inputs as bi
    make, name, tol, fp64, with_adj = WORKLOADS[args.workload]
    probs = bi.ensemble_2d(n_instances=args.instances) if args.workload == "ensemble" else make(bi)
    probs = probs if isinstance(probs, list) else [probs]
    if args.workload == "ensemble" and args.instances != 256:
        name = name.replace("256x", f"{args.instances}x")
    if args.bands:
        probs = [q.copy(C=q.C[:args.bands], v=q.v[:args.bands], tau=q.tau[:args.bands]) for q in probs]
        name = re.sub(r"_B\d+_", f"_B{probs[0].B}_", name)

    # the CPU baseline runs before any GPU work (no fork after CUDA init)
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        p0 = probs[0]
        cpu = cpu_baseline_oracle(probs, args.cpu_iters, TRANSIENT.get(args.workload))

    import __graft_entry__
    __graft_entry__.build()
    import paper_2503_23657_gb300 as m

    ctx = dict(args=args, ws=ws, rank=rank, dist=dist, torch=torch, m=m, name=name, tol=tol, fp64=fp64,
               with_adj=with_adj, cpu=cpu)
    if args.workload == "ensemble":
        line = run_ensemble(probs, ctx)
    elif args.workload in TRANSIENT:
        line = run_transient(probs[0], ctx)
    else:
        line = run_single(probs[0], ctx)
        if args.workload == "finfet" and ws == 1 and not args.no_ensemble:
            line["ensemble"] = ensemble_fp32_vs_fp64(ctx)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()
    return 0


def timed_steps(ctx, step, flush):
    """W untimed steps, then exactly K steps between barriers + syncs; returns
    per-step device times (ms), step results, clocks."""
    torch, args, ws, dist = ctx["torch"], ctx["args"], ctx["ws"], ctx["dist"]
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    clocks = ClockSampler(torch.cuda.current_device())
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    torch.cuda.nvtx.range_push("bench_timed")   # lets a profiler select the timed steps
    times, res = [], []
    for _ in range(args.steps):
        flush.fill_(1.0)   # evict the previous step's working set from L2
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        res.append(step())
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    if ws > 1:
        dist.barrier()
    return times, res, clocks.stop()


def aggregate(ctx, units, t_total):
    """Whole-job numbers over the replicas: units summed over ranks, time the
    slowest rank's."""
    torch, ws, dist = ctx["torch"], ctx["ws"], ctx["dist"]
    if ws > 1:
        dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
        tt = torch.tensor([t_total], dtype=torch.float64, device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        uu = torch.tensor([units], dtype=torch.float64, device=dev)
        dist.all_reduce(uu, op=dist.ReduceOp.SUM)
        return float(uu), float(tt)
    return units, t_total


def base_line(ctx, value, t_max, dtype, config):
    args = ctx["args"]
    return {"metric": METRIC, "value": value, "unit": "updates/s", "n_gpus": ctx["ws"], "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_max * 1e3 / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": dtype, "data": "synthetic", "config": config}


def run_single(p, ctx):
    torch, m, args, tol = ctx["torch"], ctx["m"], ctx["args"], ctx["tol"]
    prec = m.BTE_FP64 if ctx["fp64"] else m.BTE_FP32
    if ctx["with_adj"]:
        if getattr(p, "probes", None) is not None and p.T_obs is not None:
            probes, T_obs = np.asarray(p.probes), np.asarray(p.T_obs)
        else:
            probes, T_obs = probes_and_obs(p)
    else:
        probes, T_obs = np.zeros(0, dtype=np.int64), np.zeros(0)
    probes_d = torch.as_tensor(probes, device="cuda")
    T_obs_d = torch.as_tensor(T_obs, device="cuda")
    plan = m.Plan(p)
    stream = torch.cuda.current_stream()
    sp = stream.cuda_stream
    T = torch.zeros(p.n_cells, dtype=torch.float64, device="cuda")
    g = torch.zeros(p.n_cells, dtype=torch.float64, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    per_update = p.n_active * p.B * p.D
    tile_kind, tile_dw, tile_cw, tile_st, tile_wz, tile_ax = (
        int(x) for x in (args.tile + ":0:0:0:0:0:0").split(":")[:6])

    def step():
        rc, sf = plan.solve(T, precision=prec, tol=tol, max_iter=100000, stream=sp,
                            store_e_every_iter=args.store_e_every_iter, tile_kind=tile_kind,
                            dirs_per_lane=tile_dw, dirs_per_cta=tile_cw, source_staging=tile_st,
                            warps_z=tile_wz, lane_axis=tile_ax)
        sa = None
        if ctx["with_adj"]:
            g.zero_()
            g[probes_d] = T[probes_d] - T_obs_d
            rc, g_tau, g_Tw, g_Q, sa = plan.adjoint(g, tol=tol, max_iter=100000)
        return sf, sa

    # the sweep of every TIME_EVERY-th iteration of the timed steps is bracketed
    # by CUDA events on its stream (inside the captured graphs): the dominant
    # kernel's mean duration, sampled over the whole timed region
    plan.set_sweep_timing(TIME_EVERY)
    times, res, clk = timed_steps(ctx, step, flush)
    plan.set_sweep_timing(0)
    fstats = [r[0] for r in res]
    astats = [r[1] for r in res if r[1] is not None]
    units = sum(f["iterations"] * per_update for f in fstats) + sum(a["iterations"] * per_update for a in astats)
    t_total = sum(times) / 1e3
    units_all, t_max = aggregate(ctx, units, t_total)
    value = units_all / t_max
    launches = sum(f["kernel_launches"] for f in fstats) + sum(a["kernel_launches"] for a in astats)

    fwd_ups = statistics.median(f["updates_per_s"] for f in fstats)
    fwd_ms = statistics.median(f["seconds"] for f in fstats) * 1e3
    extra = {}
    if not ctx["fp64"] and not args.no_fp64:
        # forward in FP64 on the GPU (not part of the timed region)
        T64 = torch.zeros_like(T)
        plan.solve(T64, precision=m.BTE_FP64, tol=tol, max_iter=100000, stream=sp)
        rc, s64 = plan.solve(T64, precision=m.BTE_FP64, tol=tol, max_iter=100000, stream=sp)
        extra = {"fp64_fwd_updates_per_s": s64["updates_per_s"], "fp64_fwd_time_to_converge_ms": s64["seconds"] * 1e3,
                 "fp64_fwd_iterations": s64["iterations"], "speedup_fp32_vs_fp64_fwd": fwd_ups / s64["updates_per_s"],
                 "T_fp32_vs_fp64_rel": float((T - T64).abs().max() / T64.abs().max())}

    # dominant kernel: the sweep (forward and adjoint launches of the same
    # kernel), its mean launch duration from the CUDA events of the timed steps
    fwd_sweep_s = sum(f["sweep_seconds"] for f in fstats)
    fwd_sweeps = sum(f["sweep_launches"] for f in fstats)
    adj_sweep_s = sum(a["sweep_seconds"] for a in astats)
    adj_sweeps = sum(a["sweep_launches"] for a in astats)
    sweep_ms = (fwd_sweep_s + adj_sweep_s) / max(fwd_sweeps + adj_sweeps, 1) * 1e3
    dw = fstats[-1]["dirs_per_lane"]
    tile = f"{fstats[-1]['tile_kind']}:{dw}:{fstats[-1]['dirs_per_cta']}:{2 - fstats[-1]['source_staged']}"
    if fstats[-1]["warps_z"]:
        tile += f":{fstats[-1]['warps_z']}:{fstats[-1]['lane_axis']}"
    kernel = sweep_kernel_name(p, fstats[-1])
    roofline = roofline_object(kernel, tile, sweep_ms, per_update, p.B, p.D, {
        "sweep_launches_timed": fwd_sweeps + adj_sweeps,
        "fwd_sweep_ms": fwd_sweep_s / max(fwd_sweeps, 1) * 1e3,
        "adj_sweep_ms": adj_sweep_s / max(adj_sweeps, 1) * 1e3 if astats else None,
        "sweep_share_of_step": (fwd_sweep_s * timed_sweep_scale(fstats) +
                                (adj_sweep_s * timed_sweep_scale(astats) if astats else 0.0)) / t_total})

    # end to end through the C ABI with host buffers (pinned), copies inside
    T_init_h = torch.full((p.n_cells,), float(p.T_init), dtype=torch.float64).pin_memory()
    T_h = torch.zeros(p.n_cells, dtype=torch.float64).pin_memory()
    g_h = torch.zeros(p.n_cells, dtype=torch.float64).pin_memory()
    T_obs_t = torch.as_tensor(T_obs)
    e2e_units, e2e_t = 0, 0.0
    for i in range(max(2, min(args.steps, 5))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rc, sf = plan.solve(T_h, T_init=T_init_h, precision=prec, tol=tol, max_iter=100000, stream=sp,
                            tile_kind=tile_kind, dirs_per_lane=tile_dw, dirs_per_cta=tile_cw, source_staging=tile_st,
                            warps_z=tile_wz, lane_axis=tile_ax)
        u = sf["iterations"] * per_update
        if ctx["with_adj"]:
            g_h.zero_()
            g_h[probes] = T_h[probes] - T_obs_t
            rc, g_tau, g_Tw, g_Q, sa = plan.adjoint(g_h, tol=tol, max_iter=100000)
            u += sa["iterations"] * per_update
        t1 = time.perf_counter()
        if i > 0:
            e2e_units += u
            e2e_t += t1 - t0
    e2e_value = e2e_units / e2e_t * (ctx["ws"] if ctx["ws"] > 1 else 1)

    config = {"workload": ctx["name"], "cells": p.n_cells, "solid_cells": p.n_active, "bands": p.B,
              "directions": p.D, "tol_eps_T": tol,
              "l2": f"flushed before every step ({L2_FLUSH_BYTES >> 20} MB write)",
              "parallelism": "replicas" if ctx["ws"] > 1 else "single",
              "store_e_every_iter": bool(args.store_e_every_iter), "tile": tile}
    line = base_line(ctx, value, t_max, "f64" if ctx["fp64"] else "f32", config)
    # the stopping measure eps_T = RMS(dT)/T_max understates the change when
    # the temperature range is small: the same RMS change over T_max - T_min
    act = torch.as_tensor(p.mask > 0, device="cuda")
    Ta = T[act]
    t_range = float(Ta.max() - Ta.min())
    dT_rms = fstats[-1]["eps_T"] * fstats[-1]["T_max"]
    line.update({"fwd_iterations": fstats[-1]["iterations"],
                 "adj_iterations": astats[-1]["iterations"] if astats else None,
                 "fwd_time_to_converge_ms": fwd_ms, "fwd_updates_per_s": fwd_ups,
                 "step_ms_median": statistics.median(times),
                 "eps_T_final": fstats[-1]["eps_T"],
                 "dT_rms_over_T_range_final": dT_rms / t_range if t_range > 0 else None})
    line.update(extra)
    line.update({
        "roofline": roofline, "cpu_baseline": ctx["cpu"],
        "e2e": {"value": e2e_value, "unit": "updates/s",
                "h2d_bytes_per_step": (2 if ctx["with_adj"] else 1) * 8 * p.n_cells,
                "d2h_bytes_per_step": 8 * p.n_cells + (8 * (p.B + 7) if ctx["with_adj"] else 0)},
        "gpu_launches": launches, "clocks": clk})
    return line


def run_transient(p, ctx):
    """Implicit-Euler time steps (bte_transient): a bench step is `steps` time
    steps of length dt from the equilibrium at 300 K, each solved to eps_T <
    tol (FP32 sweeps, FP64 temperatures); the value counts the source
    iterations of all of them."""
    torch, m, args, tol = ctx["torch"], ctx["m"], ctx["args"], ctx["tol"]
    dt, nsteps = TRANSIENT[args.workload]
    plan = m.Plan(p)
    sp = torch.cuda.current_stream().cuda_stream
    T = torch.zeros(p.n_cells, dtype=torch.float64, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    per_update = p.n_active * p.B * p.D
    tile_kind, tile_dw, tile_cw, tile_st, tile_wz, tile_ax = (
        int(x) for x in (args.tile + ":0:0:0:0:0:0").split(":")[:6])
    topt = dict(tile_kind=tile_kind, dirs_per_lane=tile_dw, warps_z=tile_wz, lane_axis=tile_ax)

    def step():
        rc, st = plan.transient(dt, nsteps, T, precision=m.BTE_FP32, tol=tol, stream=sp, **topt)
        return st

    plan.set_sweep_timing(TIME_EVERY)
    times, res, clk = timed_steps(ctx, step, flush)
    plan.set_sweep_timing(0)
    units = sum(st["iterations"] for st in res) * per_update
    t_total = sum(times) / 1e3
    units_all, t_max = aggregate(ctx, units, t_total)
    last = res[-1]
    # the sweep launches of the last time step's solve, event-timed
    sweep_ms = last["sweep_seconds"] / max(last["sweep_launches"], 1) * 1e3
    dw = last["dirs_per_lane"]
    tile = f"{last['tile_kind']}:{dw}:{last['dirs_per_cta']}:{2 - last['source_staged']}"
    if last["warps_z"]:
        tile += f":{last['warps_z']}:{last['lane_axis']}"
    if last["tile_kind"] == 3 and p.dim == 3:
        spec = int(any(int(t) == 2 for t in p.bc_type[:6]))
        kernel = f"sweep3dp_kernel<float, {dw}, {0 if p.phi is None else 1}, 0, {int(last['lane_axis'] == 2)}, " \
                 f"{2 + spec}>"
    else:
        kernel = f"sweep_kernel<float, {dw}, lz, {int(p.dim == 3)}, 0>"
    roofline = roofline_object(kernel, tile, sweep_ms, per_update, p.B, p.D, {
        "sweep_launches_timed": last["sweep_launches"],
        "extra_source_bytes_per_update": 4.0,
        "note": "the extra source (e of the previous step over dt) is read once per update (4 B), beyond the "
                "steady sweep's algorithmic bytes"})
    extra = {}
    if not args.no_fp64:
        T64 = torch.zeros_like(T)
        rc, s64 = plan.transient(dt, nsteps, T64, precision=m.BTE_FP64, tol=tol, stream=sp)
        extra = {"fp64_iterations": s64["iterations"],
                 "T_fp32_vs_fp64_rel": float((T - T64).abs().max() / T64.abs().max())}
    # end to end with host buffers
    T_h = torch.zeros(p.n_cells, dtype=torch.float64).pin_memory()
    e2e_units, e2e_t = 0, 0.0
    for i in range(max(2, min(args.steps, 4))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rc, st = plan.transient(dt, nsteps, T_h, precision=m.BTE_FP32, tol=tol, stream=sp, **topt)
        t1 = time.perf_counter()
        if i > 0:
            e2e_units += st["iterations"] * per_update
            e2e_t += t1 - t0
    config = {"workload": ctx["name"], "cells": p.n_cells, "solid_cells": p.n_active, "bands": p.B,
              "directions": p.D, "tol_eps_T": tol, "dt_s": dt, "time_steps_per_step": nsteps,
              "l2": f"flushed before every step ({L2_FLUSH_BYTES >> 20} MB write)",
              "parallelism": "replicas" if ctx["ws"] > 1 else "single", "tile": tile}
    line = base_line(ctx, units_all / t_max, t_max, "f32", config)
    line.update({"iterations_per_step": statistics.median(st["iterations"] for st in res)})
    line.update(extra)
    line.update({
        "roofline": roofline, "cpu_baseline": ctx["cpu"],
        "e2e": {"value": e2e_units / e2e_t if e2e_t > 0 else None, "unit": "updates/s",
                "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 8 * p.n_cells},
        "gpu_launches": sum(st["kernel_launches"] for st in res), "clocks": clk})
    return line


def ensemble_fp32_vs_fp64(ctx):
    """The batched ensemble (256 uneven 2D squares, 15 bands x 64 directions)
    solved to eps_T < 1e-6 per instance in FP32 (sweeps; FP64 reductions) and
    in FP64 on the GPU, outside the timed steps: the FP32 batched form's
    speedup over the FP64 GPU path and the FP32 temperatures' error against
    the FP64 ones.  Each precision first runs one graph replay (tile
    autotuning and graph capture), then the timed solve."""
    torch, m = ctx["torch"], ctx["m"]
    import bte_inputs as bi
    probs = bi.ensemble_2d()
    plans = [m.Plan(p) for p in probs]
    batch = m.Batch(plans)
    n = sum(p.n_cells for p in probs)
    res = {}
    for prec in (m.BTE_FP32, m.BTE_FP64):
        T = torch.zeros(n, dtype=torch.float64, device="cuda")
        batch.solve(T, precision=prec, tol=1e-6, max_iter=32, check=False)
        rc, st, bs = batch.solve(T, precision=prec, tol=1e-6, max_iter=100000)
        res[prec] = (T, st, bs)
    (T32, st32, bs32), (T64, st64, bs64) = res[m.BTE_FP32], res[m.BTE_FP64]
    o = batch.offsets
    errs = [float((T32[o[i]:o[i + 1]] - T64[o[i]:o[i + 1]]).abs().max() / T64[o[i]:o[i + 1]].abs().max())
            for i in range(len(probs))]
    out = {"workload": WORKLOADS["ensemble"][1], "instances": len(probs), "cells": n,
           "fp32_time_to_converge_ms": bs32["seconds"] * 1e3, "fp64_time_to_converge_ms": bs64["seconds"] * 1e3,
           "speedup_fp32_vs_fp64": bs64["seconds"] / bs32["seconds"],
           "fp32_updates_per_s": bs32["updates_per_s"], "fp64_updates_per_s": bs64["updates_per_s"],
           "T_fp32_vs_fp64_rel_max": max(errs),
           "iterations_equal_fp32_fp64": sum(int(a["iterations"] == b["iterations"]) for a, b in zip(st32, st64)),
           "converged_fp32_fp64": [bs32["converged"], bs64["converged"]],
           "gpu_launches_fp32": bs32["kernel_launches"]}
    batch.close()
    for pl in plans:
        pl.close()
    return out


def run_ensemble(probs, ctx):
    torch, m, args, tol = ctx["torch"], ctx["m"], ctx["args"], ctx["tol"]
    if ctx["ws"] > 1:
        # the instances are independent: each rank solves its share, nothing
        # is exchanged on the data path (the whole job is fixed: strong scaling)
        probs = probs[ctx["rank"]::ctx["ws"]]
    plans = [m.Plan(p) for p in probs]
    batch = m.Batch(plans)
    n = sum(p.n_cells for p in probs)
    T = torch.zeros(n, dtype=torch.float64, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    per_iter = [p.n_active * p.B * p.D for p in probs]

    def step():
        rc, st, bs = batch.solve(T, precision=m.BTE_FP32, tol=tol, max_iter=100000)
        return st, bs

    times, res, clk = timed_steps(ctx, step, flush)
    units = sum(sum(s["iterations"] * u for s, u in zip(st, per_iter)) for st, bs in res)
    t_total = sum(times) / 1e3
    units_all, t_max = aggregate(ctx, units, t_total)
    value = units_all / t_max
    launches = sum(bs["kernel_launches"] for st, bs in res)
    st, bs = res[-1]
    its = sorted(s["iterations"] for s in st)

    # FP64 batch (not timed above) and the FP32 error against it
    extra = {}
    if not args.no_fp64:
        T64 = torch.zeros_like(T)
        batch.solve(T64, precision=m.BTE_FP64, tol=tol, max_iter=100000)
        rc, st64, bs64 = batch.solve(T64, precision=m.BTE_FP64, tol=tol, max_iter=100000)
        errs = [float((T[batch.offsets[i]:batch.offsets[i + 1]] - T64[batch.offsets[i]:batch.offsets[i + 1]]).abs().max()
                      / T64[batch.offsets[i]:batch.offsets[i + 1]].abs().max()) for i in range(len(probs))]
        extra = {"fp64_time_to_converge_ms": bs64["seconds"] * 1e3, "fp64_updates_per_s": bs64["updates_per_s"],
                 "speedup_fp32_vs_fp64": bs64["seconds"] / bs["seconds"],
                 "T_fp32_vs_fp64_rel_max": max(errs),
                 "iterations_equal_fp32_fp64": sum(int(a["iterations"] == b["iterations"]) for a, b in zip(st, st64))}

    # the batched sweep phase (all size classes, fork to join) with every
    # instance active: fixed iterations with the sweep phase event-timed
    batch.set_sweep_timing(True)
    Tz = torch.zeros_like(T)
    rc, stz, bsz = batch.solve(Tz, precision=m.BTE_FP32, tol=0.0, max_iter=256)
    batch.set_sweep_timing(False)
    sweep_ms = bsz["sweep_seconds"] / max(bsz["sweep_iterations"], 1) * 1e3
    tiles = sorted({f"3:{s['dirs_per_lane']}:{s['dirs_per_cta']}" for s in stz})
    roofline = roofline_object("sweep2dp_batch_kernel (all size classes, concurrent)", ",".join(tiles), sweep_ms,
                               sum(per_iter), probs[0].B, probs[0].D,
                               {"sweep_phases_timed": bsz["sweep_iterations"],
                                "timing": "sweep phase of the first iteration of each 32-iteration graph, "
                                          "fixed-iteration run with every instance active"})

    # end to end with a host output buffer (pinned), copy inside
    T_h = torch.zeros(n, dtype=torch.float64).pin_memory()
    e2e_units, e2e_t = 0, 0.0
    for i in range(3):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rc, st2, bs2 = batch.solve(T_h, precision=m.BTE_FP32, tol=tol, max_iter=100000)
        t1 = time.perf_counter()
        if i > 0:
            e2e_units += sum(s["iterations"] * u for s, u in zip(st2, per_iter))
            e2e_t += t1 - t0
    # effective Knudsen number of each instance, (sum C v^2 tau / sum C v) / L (descriptive)
    kn = sorted(float(np.sum(q.C * q.v ** 2 * q.tau) / np.sum(q.C * q.v) / q.length[0]) for q in probs)
    config = {"workload": ctx["name"], "instances_this_rank": len(probs), "cells_this_rank": n, "bands": probs[0].B,
              "Kn_eff_min_median_max": [kn[0], kn[len(kn) // 2], kn[-1]],
              "directions": probs[0].D, "tol_eps_T": tol, "size_classes": bs["classes"],
              "l2": f"flushed before every step ({L2_FLUSH_BYTES >> 20} MB write)",
              "parallelism": "instances sharded over ranks" if ctx["ws"] > 1 else "single",
              "tiles": ",".join(tiles)}
    line = base_line(ctx, value, t_max, "f32", config)
    if ctx["ws"] > 1:
        line["scaling"] = "strong"
    line.update({"time_to_converge_ms": bs["seconds"] * 1e3, "iterations_min_median_max": [its[0], its[len(its) // 2], its[-1]],
                 "converged": bs["converged"]})
    line.update(extra)
    line.update({"roofline": roofline, "cpu_baseline": ctx["cpu"],
                 "e2e": {"value": e2e_units / e2e_t, "unit": "updates/s", "h2d_bytes_per_step": 0,
                         "d2h_bytes_per_step": 8 * n},
                 "gpu_launches": launches, "clocks": clk})
    return line


if __name__ == "__main__":
    sys.exit(main())
