#!/usr/bin/env python
"""Benchmark of the STBA LM iteration on one GB300 (or N replicas under torchrun).

Workload: the unordered Internet-like scene -- 1000 cameras on a hemisphere of radius 20, 200k points in
a 10^3 box, Zipf(2) tracks on [2, 50] (1.11M observations), 10 clusters of 100 cameras, mixed precision
(FP32 Jacobians and Schur accumulation, FP32 factorisation with FP64 refinement, FP64 cost sums).
A step is one full LM iteration (residuals and Jacobians, virtual points and correction, S' build,
per-cluster factorisation and solve, point update, cost, accept / reject).  L2 is flushed between timed
steps (a 512 MB write outside the timed events).

Prints one JSON line.  --impl reference times the FP64 CPU oracle on the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "STBA LM iter/s and obs/s vs full-RCS LM on 1 GB300 at equal final RMSE"
CONFIG = "c1_internet"
SGC_GAMMA, SGC_BETA = 100, 10.0
REORDER_LAUNCHES = 16  # kernels of one stba_set_clusters (device re-ordering, listing of the pair chunks)
WORKLOADS = {
    "c1_internet": ("c1_internet: 1000 cameras (hemisphere r=20), 200k points (10^3 box), Zipf(2) tracks on [2,50] "
                    "over nearby viewpoints, clusters drawn every iteration by stochastic graph clustering "
                    "(Gamma 100, beta 10), mixed precision"),
    "c4_large": ("c4_large: 20000 cameras (hemisphere r=60), 4M points (30^3 box), Zipf(2) tracks on [2,80] over "
                 "nearby viewpoints, clusters drawn every iteration by stochastic graph clustering (Gamma 100, "
                 "beta 10), mixed precision"),
    "c2_slam": ("c2_slam: 5000 cameras along a 2 km closed trajectory with 3 crossings, 500k points, tracks of "
                "2-20 consecutive frames, 27 clusters of 45-297 cameras, mixed precision"),
}
WORKLOAD = WORKLOADS[CONFIG]
FP32_PEAK_TFLOPS_DERIVED = 152 * 128 * 2 * 2.070e9 / 1e12   # SMs x FP32 lanes x 2 flops x max SM clock (fallback)


def env_rank():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def max_over_ranks(value, device=None):
    """The largest value over the ranks of the process group (a job's time is its slowest rank's); the value
    itself without a group or with one rank."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def source_hash():
    """Hash of the CUDA sources; the DRAM traffic in profiles/traffic.json is used only while it matches."""
    import glob
    import hashlib
    h = hashlib.sha256()
    for f in sorted(glob.glob(os.path.join(ROOT, "paper_2008_00446_gb300", "csrc", "*"))):
        h.update(os.path.basename(f).encode())
        h.update(open(f, "rb").read())
    return h.hexdigest()[:16]


def stage_traffic(stage, config):
    """DRAM bytes per iteration of a stage from profiles/traffic.json, or None unless that capture was of the
    same sources and the same workload."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            t = json.load(f)
    except (OSError, ValueError):
        return None
    if t.get("source_hash") != source_hash() or not str(t.get("workload", "")).startswith(config + ","):
        return None
    return t.get("stage_dram_bytes_per_iteration", {}).get(stage)


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() in ("active", "1", "yes"):
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": max(mx), "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------------------------------------
# CPU oracle (the reference arm and the cpu_baseline leg)
# ----------------------------------------------------------------------------------------------------------
ORACLE_CHILD = r"""
import json, os, sys, time
sys.path.insert(0, sys.argv[1])
import numpy as np
import scenes
from oracle import camera, stba
s = scenes.make_config(sys.argv[2])
iters = int(sys.argv[3])
F = camera.cost(s.cameras, s.points, s.obs_cam, s.obs_pt, s.obs_uv)
t = time.perf_counter()
c, p, lam, F, hist = stba.solve(s.cameras, s.points, s.obs_cam, s.obs_pt, s.obs_uv, s.clusters, iters)
dt = time.perf_counter() - t
print(json.dumps({"seconds": dt, "iters": iters, "q": int(s.q), "F": F}))
"""


def run_oracle(config, iters, threads=1):
    """One oracle run in a child process with `threads` BLAS threads (the SciPy-sparse products are
    single-threaded either way; dense Cholesky factors and products use the threads)."""
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = str(threads)
    env.pop("CUDA_VISIBLE_DEVICES", None)
    r = subprocess.run([sys.executable, "-c", ORACLE_CHILD, ROOT, config, str(iters)], capture_output=True,
                       text=True, env=env)
    if r.returncode != 0:
        raise RuntimeError(r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def reference_arm(args):
    rank, world, _ = env_rank()
    if rank != 0:
        return
    secs = []
    q = None
    # each step is one oracle LM iteration of the full workload (tens of seconds); stop adding steps once
    # the run would exceed about three minutes
    t_start = time.perf_counter()
    cores = os.cpu_count() or 1
    for i in range(args.steps):
        out = run_oracle(CONFIG, 1, threads=cores)
        secs.append(out["seconds"])
        q = out["q"]
        el = time.perf_counter() - t_start
        if el + el / (i + 1) > 180.0:
            break
    steps = len(secs)
    tot = sum(secs)
    v = steps / tot
    sample = (f"{steps} step(s), each one STBA LM iteration of the full workload (FP64 SciPy-sparse oracle, "
              f"{cores} BLAS threads) with the scene's fixed azimuth-wedge clustering instead of a new draw")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "iter/s", "n_gpus": args.gpus,
        "steps": steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "l2_flush": False},
        "obs_per_s": v * q,
        "cpu_baseline": {"value": v, "unit": "iter/s", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": "iter/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


# ----------------------------------------------------------------------------------------------------------
STAGES = ["linearise", "s_build", "factorisation", "cluster_solve", "point_update_cost"]


def stage_roofline(info0, stage_ms, q, n, m, hbm, alu, config):
    """Algorithmic bytes (inputs read once, outputs written once) of every stage of one iteration, its HBM
    fraction at the measured stage time, the DRAM traffic ratio where a capture of the same sources and
    workload exists, and the factorisation's flops against the measured FP32 and TF32 peaks.  Returns the
    per-stage table and the dominant stage's roofline object."""
    s_lower = info0["s_lower_elems"]
    nv = info0["nv"]
    bytes_stage = {
        "linearise": q * (8 + 4 + 4) + n * 24 + m * 72 + nv * 9 * 4 * 2 + n * 9 * 4,
        "s_build": q * (8 + 4 + 4) + n * 24 + m * 72 + nv * 9 * 4 + s_lower * 4 + m * 9 * 4 * 2,
        "factorisation": s_lower * (8 + 4),   # FP64 lower triangles read once, FP32 factor written once
        "cluster_solve": s_lower * 4 * (1 + 2 * 1) + m * 9 * 8,
        "point_update_cost": q * (8 + 4 + 4) * 2 + n * 24 * 2 + m * 72 * 2 + n * 9 * 4 + n * 24,
    }
    fp32_peak = alu["fp32_tflops"] if alu else FP32_PEAK_TFLOPS_DERIVED
    fp32_src = ("measured: stba_measure_peaks FP32 FMA chains (of measured)" if alu else
                "derived: 152 SMs x 128 FP32 lanes x 2 flops x 2070 MHz (fallback)")
    stages = {}
    for i, nm in enumerate(STAGES):
        t = float(stage_ms[i])
        b = float(bytes_stage[nm])
        gbs = b / (t / 1e3) / 1e9
        e = {"ms": t, "algorithmic_bytes": b, "achieved_gbs": gbs, "hbm_frac": gbs / hbm}
        tr = stage_traffic(nm, config)
        if tr is not None:
            e["traffic_bytes"] = tr
            e["traffic_ratio"] = tr / b
        stages[nm] = e
    fl = float(info0["factor_flops"])
    tfl = fl / (float(stage_ms[2]) / 1e3) / 1e12
    f = stages["factorisation"]
    f.update(flops=fl, achieved_tflops=tfl, fp32_peak_tflops=fp32_peak, fp32_frac=tfl / fp32_peak)
    if alu:   # a 3xTF32 product (FP32 accuracy) runs at a third of the dense TF32 rate
        f.update(tf32_peak_tflops=alu["tf32_tflops"], tensor_3xtf32_frac=tfl / (alu["tf32_tflops"] / 3.0))
    dom = STAGES[int(np.argmax(stage_ms))]
    if dom == "factorisation":
        dominant = {"bound": "alu", "stage": dom, "achieved": tfl, "peak": fp32_peak, "unit": "TFLOP/s",
                    "frac": tfl / fp32_peak, "traffic": stage_traffic(dom, config), "peak_source": fp32_src}
    else:
        e = stages[dom]
        dominant = {"bound": "hbm", "stage": dom, "achieved": e["achieved_gbs"], "peak": hbm, "unit": "GB/s",
                    "frac": e["hbm_frac"], "traffic": stage_traffic(dom, config),
                    "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)"}
    return {"stages": stages, "dominant": dominant}


def scene_leg(name, stba, stream, torch, steps=10, compare=True, builder=None, alu=None):
    """One more scene of the metric, measured outside the headline's timed steps: `steps` iterations after 3
    warm-up ones, each with its stba_set_clusters (stochastic-graph-clustering draws on the hemisphere scenes,
    the scene's own uneven segments on the sequential one), CUDA events around each; then the stage times of
    the same iterations and, with `compare`, the equal-RMSE comparison with full-RCS LM on the GPU."""
    import scenes
    t0 = time.perf_counter()
    s = builder() if builder is not None else scenes.make_config(name)
    gen_s = time.perf_counter() - t0
    ctx = stba.stba_create(s.cameras, s.points, s.obs_cam, s.obs_pt, s.obs_uv, s.clusters,
                           precision=stba.STBA_MIXED, stream=stream)
    n_it = 3 + steps
    t0 = time.perf_counter()
    if name == "c2_slam":
        seq = np.tile(np.asarray(s.clusters, np.int32), (n_it, 1))
        draw_ms = 0.0
    else:
        seq, _ = stba.stba_cluster_sgc(ctx, count=n_it, gamma=SGC_GAMMA, beta=SGC_BETA, seed=s.meta["seed"] + 1)
        draw_ms = 1e3 * (time.perf_counter() - t0) / n_it
    for i in range(3):
        stba.stba_set_clusters(ctx, seq[i])
        stba.stba_lm_iteration(ctx, want_info=False)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for i in range(steps):
        ev[i][0].record(stream)
        stba.stba_set_clusters(ctx, seq[3 + i])
        stba.stba_lm_iteration(ctx, want_info=False)
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    ms = [a.elapsed_time(b) for a, b in ev]
    st = np.zeros(5)
    info = {}
    for i in range(steps):
        stba.stba_set_clusters(ctx, seq[3 + i])
        stba.stba_lm_iteration(ctx, want_info=False)
        st += np.array(stba.stba_stage_times(ctx))
        for k_, v_ in stba.stba_problem_info(ctx).items():
            info[k_] = info.get(k_, 0) + v_ / steps
    st /= steps
    lam, F, it = stba.stba_get_state(ctx)
    stba.stba_destroy(ctx)
    hbm = measured_peaks().get("hbm_gbs", 6800.0)
    rf = stage_roofline(info, st, s.q, s.n, s.m, hbm, alu, name)
    step_ms = float(np.median(ms))
    out = {"cameras": int(s.m), "points": int(s.n), "observations": int(s.q), "generate_s": gen_s,
           "clusters_mean": float(info.get("l", 0)), "virtual_points_mean": float(info.get("nv", 0)),
           "ms_per_step": step_ms, "iter_per_s": 1e3 / step_ms, "obs_per_s": 1e3 / step_ms * s.q,
           "draw_ms_host": draw_ms, "stage_ms": {nm: float(v) for nm, v in zip(STAGES, st)},
           "stages": rf["stages"], "final_rmse_px": float(np.sqrt(F / (2 * s.q))), "iterations": it,
           "step": ("set_clusters + one LM iteration; " +
                    ("the scene's uneven contiguous segments" if name == "c2_slam" else
                     "a stochastic-graph-clustering draw (Gamma 100, beta 10)"))}
    if compare:
        out["full_rcs"] = compare_full_rcs(s, stba, stream, 10, torch)
    return out


# ----------------------------------------------------------------------------------------------------------
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default=CONFIG)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-compare", action="store_true", help="skip the full-RCS LM comparison")
    ap.add_argument("--compare-iters", type=int, default=10)
    ap.add_argument("--no-adjoint", action="store_true", help="skip the adjoint timing on the 500-camera scene")
    ap.add_argument("--no-fp64-factor", action="store_true", help="skip the FP64-factor leg")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default factorisation tile")
    ap.add_argument("--no-scenes", action="store_true",
                    help="skip the extra scene legs (20000 cameras, 5000-camera sequential, uniform tracks)")
    ap.add_argument("--no-peaks", action="store_true", help="skip the measured FP32 / TF32 peaks")
    ap.add_argument("--factor", default=None,
                    help="force one factorisation configuration (a name of stba.AUTOTUNE_CANDIDATES) instead of "
                         "the autotuner's choice")
    args = ap.parse_args()
    if args.impl == "reference":
        return reference_arm(args)

    import numpy as np
    import torch

    import scenes
    from paper_2008_00446_gb300 import stba

    rank, world, local = env_rank()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()

    s = scenes.make_config(args.config)
    fkw = {}
    if args.factor:
        t_, u_, p_ = stba.AUTOTUNE_CANDIDATES[args.factor]
        fkw = dict(factor_tile=t_, factor_update=u_, factor_panel=p_)
    ctx = stba.stba_create(s.cameras, s.points, s.obs_cam, s.obs_pt, s.obs_uv, s.clusters,
                           precision=stba.STBA_MIXED, stream=stream, **fkw)
    info0 = stba.stba_problem_info(ctx)
    # Algorithm 1 draws a new clustering every iteration (stochastic graph clustering, Sec. 4.4, with the
    # paper's beta = 10, Gamma = 100).  The camera graph is fixed, so the draws do not depend on the
    # iterations: they are made ahead on host threads, like a data loader, and timed separately.
    e2e_steps = max(3, min(args.steps, 10))
    n_draw = max(args.warmup, 3) + args.steps + e2e_steps
    t0 = time.perf_counter()
    seq, seq_l = stba.stba_cluster_sgc(ctx, count=n_draw, gamma=SGC_GAMMA, beta=SGC_BETA, seed=s.meta["seed"] + 1)
    sgc_s = time.perf_counter() - t0
    sgc = {"gamma": SGC_GAMMA, "beta": SGC_BETA, "draws": n_draw, "host_threads": min(os.cpu_count() or 1, 16),
           "ms_per_draw": 1e3 * sgc_s / n_draw, "clusters_mean": float(np.mean(seq_l))}
    if args.config == "c2_slam":
        # the sequential scene's own uneven segments (45..297 cameras), applied every step
        seq = np.tile(np.asarray(s.clusters, np.int32), (n_draw, 1))
        sgc = {"note": "the scene's uneven contiguous segments, re-applied every step", "clusters_mean":
               float(np.max(s.clusters) + 1)}
    stba.stba_set_clusters(ctx, seq[0])
    tuned, tile_ms = None, {}
    if not args.no_autotune and not args.factor:   # the factorisation configuration, chosen by timing
        tuned, tile_ms = stba.stba_autotune(ctx, 5)
    for i in range(max(args.warmup, 3)):
        stba.stba_set_clusters(ctx, seq[i])
        stba.stba_lm_iteration(ctx, want_info=False)
    torch.cuda.synchronize()
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    sampler = ClockSampler(local)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    sampler.start()
    t_wall = time.perf_counter()
    w0 = max(args.warmup, 3)
    for i in range(args.steps):   # nothing in the loop waits for the device
        flush.fill_(float(i))
        ev[i][0].record(stream)
        stba.stba_set_clusters(ctx, seq[w0 + i])
        stba.stba_lm_iteration(ctx, want_info=False)
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall
    clocks = sampler.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    tot_ms = float(sum(step_ms))
    tot_ms = max_over_ranks(tot_ms, dev)
    lam, F_end, it_end = stba.stba_get_state(ctx)
    value = world * args.steps / (tot_ms / 1e3)

    # stage times and sizes: the same steps again (their clusterings), reading the stage events after each
    stage_tot = np.zeros(5)
    info_tot = {}
    n_stage = min(args.steps, 50)
    boosted = failed = 0   # FP32 pivots raised by static pivoting, failed cluster factorisations
    for i in range(n_stage):
        flush.fill_(float(i))
        stba.stba_set_clusters(ctx, seq[w0 + i])
        it_info = stba.stba_lm_iteration(ctx)
        boosted += it_info["boosted_pivots"]
        failed += it_info["failed_clusters"]
        stage_tot += np.array(stba.stba_stage_times(ctx))
        for k_, v_ in stba.stba_problem_info(ctx).items():
            info_tot[k_] = info_tot.get(k_, 0) + v_
    stage_ms = stage_tot / n_stage
    info0 = {k_: v_ / n_stage for k_, v_ in info_tot.items()}   # per-step means over the clusterings

    # the same iterations without re-clustering (one fixed assignment), for reference
    fixed_ms = []
    for i in range(min(args.steps, 50)):
        flush.fill_(float(i))
        a_ev, b_ev = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a_ev.record(stream)
        stba.stba_lm_iteration(ctx, want_info=False)
        b_ev.record(stream)
        fixed_ms.append((a_ev, b_ev))
    torch.cuda.synchronize()
    fixed_ms = float(np.mean([a.elapsed_time(b) for a, b in fixed_ms]))

    # the same steps with the cluster systems factored in FP64 (option factor_fp64) under the same FP32
    # Jacobians, for the cost of the precision Eq. 13's solve has in the paper's CPU code
    fp64f = None
    if rank == 0 and world == 1 and not args.no_fp64_factor:
        ctx64 = stba.stba_create(s.cameras, s.points, s.obs_cam, s.obs_pt, s.obs_uv, s.clusters,
                                 precision=stba.STBA_MIXED, stream=stream, factor_fp64=1)
        st64 = np.zeros(5)
        ev64 = []
        n64 = min(args.steps, 20)
        for i in range(3 + n64):
            flush.fill_(float(i))
            a_ev, b_ev = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a_ev.record(stream)
            stba.stba_set_clusters(ctx64, seq[w0 + i % args.steps])
            stba.stba_lm_iteration(ctx64, want_info=False)
            b_ev.record(stream)
            if i >= 3:
                ev64.append((a_ev, b_ev))
                st64 += np.array(stba.stba_stage_times(ctx64))
        torch.cuda.synchronize()
        st64 /= n64
        fp64f = {"ms_per_step": float(np.mean([a.elapsed_time(b) for a, b in ev64])),
                 "stage_ms": {nm: float(v) for nm, v in zip(STAGES, st64)},
                 "note": "factor_fp64 = 1: FP64 LL^T of every S'_k (tile 32, CUDA cores) under the same FP32 "
                         "Jacobians and the same clustering draws (and the same one refinement step)"}
        stba.stba_destroy(ctx64)

    # measured arithmetic peaks (outside the timed region), with the SM clock sampled while they run
    alu = None
    if not args.no_peaks:
        psampler = ClockSampler(local)
        psampler.start()
        fp32s, tf32s = [], []
        t_end = time.perf_counter() + 1.5
        while time.perf_counter() < t_end or not fp32s:
            a_, b_ = stba.stba_measure_peaks(3, stream)
            fp32s.append(a_)
            tf32s.append(b_)
        alu = {"fp32_tflops": max(fp32s), "tf32_tflops": max(tf32s), "runs": len(fp32s), "clocks": psampler.stop(),
               "how": "stba_measure_peaks: FP32 FMA chains on every SM (CUDA cores); tcgen05.mma kind::tf32 "
                      "M128 N256 K8 back to back into TMEM, one CTA per SM (tensor cores); best of the runs"}
    # roofline of the dominant stage and of every stage (stage averages over the timed steps)
    q, n, m = s.q, s.n, s.m
    rf = stage_roofline(info0, stage_ms, q, n, m, measured_peaks().get("hbm_gbs", 6800.0), alu, args.config)
    roofline = rf["dominant"]
    roofline["stage_ms"] = {nm: float(v) for nm, v in zip(STAGES, stage_ms)}
    roofline["stages"] = rf["stages"]
    if alu:
        roofline["measured_alu_peaks"] = alu

    # end to end through the C ABI with host buffers: parameters and the iteration's clustering in, one
    # iteration, parameters out
    cams_h = torch.from_numpy(s.cameras.copy()).pin_memory()
    pts_h = torch.from_numpy(s.points.copy()).pin_memory()
    cams_o = torch.empty_like(cams_h).pin_memory()
    pts_o = torch.empty_like(pts_h).pin_memory()
    stba.stba_get_params(ctx, cams_h, pts_h)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    t0 = time.perf_counter()
    for i in range(e2e_steps):
        stba.stba_set_params(ctx, cams_h, pts_h)
        stba.stba_set_clusters(ctx, seq[w0 + args.steps + i])
        stba.stba_lm_iteration(ctx, want_info=False)
        stba.stba_get_params(ctx, cams_o, pts_o)
    torch.cuda.synchronize()
    e2e_s = max_over_ranks((time.perf_counter() - t0) / e2e_steps, dev)
    nbytes_in = 8 * (cams_h.numel() + pts_h.numel()) + 4 * s.m
    nbytes_out = 8 * (cams_h.numel() + pts_h.numel())

    out = {
        "metric": METRIC, "value": value, "unit": "iter/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": tot_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": WORKLOADS.get(args.config, args.config), "cameras": m, "points": n, "observations": q,
                   "clusters_mean": sgc["clusters_mean"],
                   "virtual_points_mean": float(info0["nv"]), "l2_flush": True, "parallelism": f"replicas{world}"},
        "obs_per_s": value * q,
        "roofline": roofline,
        "e2e": {"value": world / e2e_s, "unit": "iter/s", "h2d_bytes_per_step": nbytes_in,
                "d2h_bytes_per_step": nbytes_out},
        "step": "set_clusters (a stochastic-graph-clustering draw) + one LM iteration (Algorithm 1)",
        "sgc": sgc,
        "autotune": {"kept": tuned, "ms_per_iter": {str(k_): v_ for k_, v_ in tile_ms.items()}},
        "fixed_clusters_ms_per_iter": fixed_ms,
        "factor_pivots": {"boosted_pivots": int(boosted), "failed_clusters": int(failed), "steps": n_stage,
                          "note": "FP32 factor: pivots that rounding made vanish, raised to 2^-12 (static "
                                  "pivoting; the FP64 refinement solves the unmodified system)"},
        "fp64_factor": fp64f,
        "gpu_launches": int(round((info0["launches_per_iter"] + REORDER_LAUNCHES) * args.steps)),
        "clocks": clocks,
        "final": {"rmse_px": float(np.sqrt(F_end / (2 * q))), "lambda": lam, "iterations": it_end},
    }

    if rank == 0 and world == 1 and not args.no_compare:
        out["full_rcs"] = compare_full_rcs(s, stba, stream, args.compare_iters, torch)
    if rank == 0 and world == 1 and not args.no_adjoint:
        out["adjoint"] = time_adjoint(stba, stream, torch)
    if rank == 0 and world == 1 and not args.no_cpu_baseline and args.config == CONFIG:
        cores = os.cpu_count() or 1
        t1 = run_oracle(args.config, 1, threads=1)
        tn = run_oracle(args.config, 1, threads=cores)
        out["cpu_baseline"] = {"value": 1.0 / tn["seconds"], "unit": "iter/s", "cores": cores, "kind": "oracle",
                               "sample": f"one STBA LM iteration of the full workload (FP64 SciPy-sparse oracle, "
                                         f"{cores} BLAS threads = nproc) with the scene's fixed azimuth-wedge "
                                         "clustering",
                               "single_thread": {"value": 1.0 / t1["seconds"], "unit": "iter/s", "cores": 1}}
    stba.stba_destroy(ctx)
    if rank == 0 and world == 1 and not args.no_scenes and args.config == CONFIG:
        # the other scenes of the metric (outside the timed steps): the 20000-camera scene, the 5000-camera
        # sequential scene, and the headline scene with tracks drawn uniformly among the cameras that see a point
        import scenes as _sc
        c1kw = dict(_sc.CONFIGS["c1_internet"][1], tracks="uniform", name="internet_uniform")
        out["scenes"] = {
            "c4_large": scene_leg("c4_large", stba, stream, torch, alu=alu),
            "c2_slam": scene_leg("c2_slam", stba, stream, torch, alu=alu),
            "c1_uniform_tracks": scene_leg("c1_uniform_tracks", stba, stream, torch, alu=alu,
                                           builder=lambda: _sc.make_hemisphere_scene(**c1kw)),
        }
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        torch.distributed.destroy_process_group()


def compare_full_rcs(s, stba, stream, iters, torch, max_stba_iters=100):
    """Full-RCS LM on the same GPU against STBA, from the same start.  Full RCS runs `iters` iterations as
    (a) one cluster holding every camera (the dense reduced camera system, when it fits: 9 m <= 27000) and
    (b) block-Jacobi preconditioned CG on the full Schur system (matrix-free).  STBA takes a new clustering
    every iteration (Algorithm 1) -- stochastic graph clustering draws (Sec. 4.4, beta = 10, Gamma = 100),
    and, for comparison, spatial partitions (azimuth wedges with a random phase) -- and runs until its RMSE
    reaches 1.001 x the better full-RCS final RMSE (or max_stba_iters).  Every timed STBA iteration
    includes its stba_set_clusters.  Per-iteration device time, final RMSE and time to the target, the
    latter twice: iteration by iteration with the host reading the RMSE after each (as the loop that finds
    the target must), and the same number of iterations enqueued back to back."""
    import numpy as np

    import scenes

    def run(clusters, seq, n_it, target=None, **kw):
        ctx = stba.stba_create(s.cameras, s.points, s.obs_cam, s.obs_pt, s.obs_uv, clusters,
                               precision=stba.STBA_MIXED, stream=stream, **kw)
        rm, ts, cg = [], [], []
        for t in range(n_it):
            torch.cuda.synchronize()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            if seq is not None:
                stba.stba_set_clusters(ctx, seq[t])
            info = stba.stba_lm_iteration(ctx)
            b.record(stream)
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
            cg.append(info["linear_iterations"])
            _, F, _ = stba.stba_get_state(ctx)
            rm.append(float(np.sqrt(F / (2 * s.q))))
            if target is not None and rm[-1] <= target:
                break
        stba.stba_destroy(ctx)
        return {"ms_per_iter": float(np.median(ts)), "rmse": rm, "cum_ms": [float(x) for x in np.cumsum(ts)],
                "cg_iters": cg}

    res = {}
    one = np.zeros(s.m, np.int32)
    if 9 * s.m <= 27000:
        res["full_rcs_dense"] = run(one, None, iters)
    res["full_rcs_pcg"] = run(one, None, iters, linear_solver=stba.STBA_SOLVER_PCG_FULL)
    best = min(r["rmse"][-1] for r in res.values())
    target = 1.001 * best
    out = {"rmse_target": target}
    g = stba.stba_graph_create(s.m, s.n, s.obs_cam, s.obs_pt)
    seq_sgc, _ = stba.stba_graph_cluster_batch(g, max_stba_iters, gamma=100, beta=10.0, seed=s.meta["seed"] + 2)
    g.close()
    seqs = {"stba_sgc": seq_sgc}
    if s.meta.get("kind") in ("ring", "hemisphere"):
        seqs["stba_spatial"] = scenes.cluster_sequence(s, max_stba_iters, seed=s.meta["seed"] + 1)
    def run_pipelined(seq, n_it):
        # the same iterations with nothing waiting for the host between them (Algorithm 1's stop test runs on
        # the device): one pair of events around all of them
        ctx = stba.stba_create(s.cameras, s.points, s.obs_cam, s.obs_pt, s.obs_uv, seq[0], precision=stba.STBA_MIXED,
                               stream=stream)
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for t in range(n_it):
            stba.stba_set_clusters(ctx, seq[t])
            stba.stba_lm_iteration(ctx, want_info=False)
        b.record(stream)
        torch.cuda.synchronize()
        _, F, _ = stba.stba_get_state(ctx)
        stba.stba_destroy(ctx)
        return a.elapsed_time(b), float(np.sqrt(F / (2 * s.q)))

    for name, seq in seqs.items():
        st = run(seq[0], seq, max_stba_iters, target=target)
        hit = [i for i, r in enumerate(st["rmse"]) if r <= target]
        out[name] = {"iters_run": len(st["rmse"]), "ms_per_iter": st["ms_per_iter"], "final_rmse": st["rmse"][-1],
                     "time_to_target_ms": st["cum_ms"][hit[0]] if hit else None,
                     "iters_to_target": hit[0] + 1 if hit else None}
        if hit:
            ms, rm = run_pipelined(seq, hit[0] + 1)
            out[name]["time_to_target_pipelined_ms"] = ms
            out[name]["rmse_pipelined_run"] = rm
    # the iterations to the target depend on the clustering draws: four more independent draw sequences
    g = stba.stba_graph_create(s.m, s.n, s.obs_cam, s.obs_pt)
    its, tts = [out["stba_sgc"]["iters_to_target"]], [out["stba_sgc"]["time_to_target_ms"]]
    for k in range(1, 5):
        seq_k, _ = stba.stba_graph_cluster_batch(g, max_stba_iters, gamma=100, beta=10.0,
                                                 seed=s.meta["seed"] + 2 + 100003 * k)
        st = run(seq_k[0], seq_k, max_stba_iters, target=target)
        hit = [i for i, r in enumerate(st["rmse"]) if r <= target]
        its.append(hit[0] + 1 if hit else None)
        tts.append(st["cum_ms"][hit[0]] if hit else None)
    g.close()
    ok = [t for t in tts if t is not None]
    out["stba_sgc_draw_sequences"] = {"iters_to_target": its, "time_to_target_ms": tts,
                                      "median_time_to_target_ms": float(np.median(ok)) if ok else None,
                                      "note": "five independent stochastic-graph-clustering draw sequences "
                                              "(the first is stba_sgc); None = not reached in max iterations"}
    # the method with its split system solved by PCG instead of the cluster factorisations (Sec. 6); on the
    # smaller scenes only (each of its iterations costs tens of CG passes over the observations)
    if s.m <= 2000:
        st = run(seq_sgc[0], seq_sgc, max_stba_iters, target=target, linear_solver=stba.STBA_SOLVER_PCG_CLUSTERS)
        hit = [i for i, r in enumerate(st["rmse"]) if r <= target]
        out["stba_sgc_split_pcg"] = {"iters_run": len(st["rmse"]), "ms_per_iter": st["ms_per_iter"],
                                     "final_rmse": st["rmse"][-1], "cg_iters_median": float(np.median(st["cg_iters"])),
                                     "time_to_target_ms": st["cum_ms"][hit[0]] if hit else None,
                                     "iters_to_target": hit[0] + 1 if hit else None}
    for name, r in res.items():
        h = [i for i, x in enumerate(r["rmse"]) if x <= target]
        out[name] = {"iters": len(r["rmse"]), "ms_per_iter": r["ms_per_iter"], "final_rmse": r["rmse"][-1],
                     "time_ms": r["cum_ms"][-1], "time_to_target_ms": r["cum_ms"][h[0]] if h else None,
                     "cg_iters": r["cg_iters"] if name.endswith("pcg") else None}
    return out


def time_adjoint(stba, stream, torch, reps=3):
    """The differentiable configuration: 500 cameras, 50k points (about 280k observations), 5 recorded
    STBA iterations in mixed precision, then stba_adjoint of the camera-centre loss (recomputes each
    accepted step and runs the adjoint kernels).  Medians over `reps` runs after one warm-up."""
    import numpy as np

    import scenes
    s = scenes.make_config("c3_diff")
    iters = scenes.CONFIGS["c3_diff"][3]
    rng = np.random.default_rng(7)
    a_c = torch.tensor(rng.normal(0, 1, (s.m, 9)), device="cuda")
    fw, bw, fw_dev, bw_dev = [], [], [], []
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    for r in range(reps + 1):
        ctx = stba.stba_create(s.cameras, s.points, s.obs_cam, s.obs_pt, s.obs_uv, s.clusters,
                               precision=stba.STBA_MIXED, stream=stream)
        stba.stba_record(ctx, iters)   # allocates the tape and the reverse pass's buffers
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ev[0].record(stream)
        for _ in range(iters):
            stba.stba_lm_iteration(ctx, want_info=False)
        ev[1].record(stream)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        stba.stba_adjoint(ctx, a_c)
        ev[2].record(stream)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        stba.stba_destroy(ctx)
        if r > 0:
            fw.append(t1 - t0)
            bw.append(t2 - t1)
            fw_dev.append(ev[0].elapsed_time(ev[1]) * 1e-3)
            bw_dev.append(ev[1].elapsed_time(ev[2]) * 1e-3)
    med = lambda v: 1e3 * float(np.median(v))   # noqa: E731
    return {"workload": "c3_diff: 500 cameras, 50k points, Zipf(2) tracks on [2,50], 5 clusters, mixed precision",
            "observations": int(s.q), "iterations": iters, "forward_ms": med(fw_dev), "adjoint_ms": med(bw_dev),
            "forward_wall_ms": med(fw), "adjoint_wall_ms": med(bw),
            "timing": "CUDA events on the context's stream (the adjoint's span includes the host reads of the "
                      "recorded step records between its kernels); *_wall_ms: host wall clock around the calls. "
                      "The adjoint allocates nothing: its buffers come with stba_record."}


if __name__ == "__main__":
    main()
