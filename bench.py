"""Benchmark of the fused ZNCC + DT + WTA path on the paper-shaped workload.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]
                    [--storage f32|f16|i8] [--workload paper_1280x384]

One step = one pass of the whole path (window statistics, ZNCC fused with the first
horizontal DT pair, the remaining DT passes, WTA fused into the last vertical pair) over one
synthetic 1280x384 pair, D = 128, 9x9 window, sigma_s = 20, sigma_r = 0.1, 3 iterations.
Inputs are resident in HBM; L2 is flushed (a 256 MB write) before every timed step and the
flush is outside the step's CUDA events. Rank 0 prints one JSON line. With the default
workload on one GPU the line also carries, measured after the timed region: "precision" (the
same pair with F32, F16 and FastDT I8 storage: step time and disparity mismatch against the
FP64 oracle), "serving" (Poisson requests of mixed size and disparity range through the
serving calls, continuous batching against one pair per launch: p50/p99, throughput, the p99
latency breakdown and a saturation leg) and "configs" (the lines of --workload plain_320x96,
batch_uneven16 and precision_sweep, run as child processes); --no-extras leaves them out.

--impl reference times the FP64 CPU oracle (the only reference this method has) on the host
cores, one full pair per step.
"""

from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Gdisp/s & fps at 1280x384 D=128 (ZNCC+DT+WTA); served p50/p99 vs plain"
SIG_S, SIG_R, ITERS = 20.0, 0.1, 3
WORKLOADS = {
    "paper_1280x384": dict(h=384, w=1280, d=128, win=9),
    "precision_1920x1080": dict(h=1080, w=1920, d=256, win=11),
    "plain_320x96": dict(h=96, w=320, d=32, win=9),
}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(x: float, device) -> float:
    """The largest x over the ranks of the process group (x itself without one): the step time
    of a replica run is its slowest rank's."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(units_per_rank: int, world: int, seconds: float) -> float:
    """Whole-job disparities per second (Gdisp/s) of `world` replicas that each processed
    units_per_rank in `seconds` (the max over ranks)."""
    return world * units_per_rank / seconds / 1e9


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


# bytes per stored volume element of each storage type (I8: the FastDT code of Sec. IV-C)
STORAGE_BYTES = {"f32": 4, "f16": 2, "i8": 1}


def storage_code(Z, name):
    return {"f32": Z.ZNCC_F32, "f16": Z.ZNCC_F16, "i8": Z.ZNCC_I8}[name]


def workload_desc(name, storages=None):
    """The workload: the pair, its sizes and the DT parameters. The volume's storage type is
    the implementation's (the line's `dtype` / `storage` keys), so that both arms name the same
    workload; a sweep over storage types names them."""
    wl = WORKLOADS[name]
    return (f"{name}: {wl['w']}x{wl['h']} D={wl['d']} win={wl['win']}x{wl['win']} DT "
            f"sigma_s={SIG_S} sigma_r={SIG_R} iters={ITERS if name != 'plain_320x96' else 0}"
            + (f" {storages} volume storage" if storages else "") +
            "; seeded synthetic pair (blurred noise, slanted planes, 5% occlusion bands, gain/offset/noise)")


# ---------------------------------------------------------------------------------------
# clocks sampled during the timed region

class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.out = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.out, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.out.close()

    def summary(self):
        if self.proc is None or not self.path:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax = float(parts[2])
                except ValueError:
                    continue
                for nm, val in zip(names, parts[5:9]):
                    if val.lower() == "active":
                        reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------------------
# the CPU oracle (the cpu_baseline leg and the reference arm)

def time_oracle(pair, wl, iters, max_seconds=12.0, min_runs=1, max_runs=5, cores=None):
    import oracle
    cores = cores or host_cores()
    oracle.load()
    times = []
    t_start = time.perf_counter()
    while len(times) < max_runs:
        t0 = time.perf_counter()
        oracle.run(pair.left, pair.right, wl["d"], wl["win"] // 2, SIG_S, SIG_R, iters,
                   nthreads=cores)
        times.append(time.perf_counter() - t0)
        if len(times) >= min_runs and time.perf_counter() - t_start > max_seconds:
            break
    return times, cores


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    from synth import config_pair
    wl = WORKLOADS[args.workload]
    pair = config_pair(args.workload)
    iters = ITERS if args.workload != "plain_320x96" else 0
    import oracle
    cores = host_cores()
    oracle.load()
    for _ in range(args.warmup):
        oracle.run(pair.left, pair.right, wl["d"], wl["win"] // 2, SIG_S, SIG_R, iters,
                   nthreads=cores)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.run(pair.left, pair.right, wl["d"], wl["win"] // 2, SIG_S, SIG_R, iters,
                   nthreads=cores)
    dt = (time.perf_counter() - t0) / args.steps
    units = wl["w"] * wl["h"] * wl["d"]
    value = units / dt / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": "Gdisp/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(dt * 1e3, 3), "fps": round(1.0 / dt, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_desc(args.workload),
                   "l2": "n/a (CPU)"},
        "cpu_baseline": {"value": round(value, 6), "unit": "Gdisp/s", "cores": cores,
                         "kind": "oracle",
                         "sample": f"one full {wl['w']}x{wl['h']} D={wl['d']} pair per step"},
        "e2e": {"value": round(value, 6), "unit": "Gdisp/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------------------------------

def algorithmic_bytes(kind, wl, elt_bytes):
    """Algorithmic HBM bytes of one launch of a kernel kind (cost-volume traffic; the images,
    statistics and weights are below 1%)."""
    n = wl["w"] * wl["h"] * wl["d"]
    return {
        "dt_hpair": 2 * elt_bytes * n,        # read + write the volume
        "dt_vpair": 2 * elt_bytes * n,
        "dt_vpair_wta": elt_bytes * n,         # read only; WTA keys stay in L2
        "zncc_cost_hpair": elt_bytes * n,      # write only
        "zncc_cost": elt_bytes * n,
        # no volume (iters = 0): the two images in, the disparity map out
        "zncc_cost_wta": 4 * wl["w"] * wl["h"],
    }.get(kind)


# Lane operations per volume element in the path's model (window sums and Eq. (2) ~10, two
# per DT pass over 4 * iters passes, WTA ~2): the ALU side of the whole step's roofline.
ALU_OPS_ZNCC, ALU_OPS_PER_PASS, ALU_OPS_WTA = 10, 2, 2
ALU_LANES_PER_SM = 128


def step_roofline(n, iters, elt_bytes, ms, peak_gbs, peak_src, clocks):
    """Both bounds of a whole fused step: HBM (the volume written once by the cost kernel, read
    and written by every middle pass pair, read by the last: (4 * iters - 2) transfers) and
    ALU (the lane-operation model above against SMs x 128 lanes x the SM clock under load)."""
    import torch
    hbm_bytes = elt_bytes * n * max(0, 4 * iters - 2)
    hbm_us = hbm_bytes / (peak_gbs * 1e9) * 1e6
    ops = n * (ALU_OPS_ZNCC + ALU_OPS_PER_PASS * 4 * iters + (ALU_OPS_WTA if iters else 0))
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    mhz = (clocks or {}).get("sm_mhz") or (clocks or {}).get("sm_max_mhz") or 2070.0
    peak_ops = sms * ALU_LANES_PER_SM * mhz * 1e6
    step_us = ms * 1e3
    return {"step_us": round(step_us, 2),
            "hbm": {"bytes": hbm_bytes, "min_us": round(hbm_us, 2), "peak_gbs": peak_gbs,
                    "peak_source": peak_src, "frac": round(hbm_us / step_us, 4) if hbm_bytes else None},
            "alu": {"lane_ops_per_elt": ops / n, "lane_ops": ops, "min_us": round(ops / peak_ops * 1e6, 2),
                    "peak_tops": round(peak_ops / 1e12, 2), "sms": sms, "sm_mhz": mhz,
                    "frac": round(ops / peak_ops * 1e6 / step_us, 4)}}


def load_traffic(kind, digest, workload, storage):
    """DRAM bytes per launch of a kernel kind from the committed ncu capture, if it was taken
    on this workload and storage type with the current kernel sources."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        with open(path) as f:
            t = json.load(f)
    except (OSError, ValueError):
        return None
    ent = t.get("kernels", {}).get(kind)
    if (not ent or t.get("source_digest") != digest or t.get("workload_key") != workload
            or t.get("storage") != storage):
        return None
    return ent.get("bytes_per_launch")


def run_gb300(args):
    import torch
    import torch.distributed as dist

    from paper_2212_00476_gb300 import build as zbuild
    from paper_2212_00476_gb300 import zncc as Z
    from synth import config_pair

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    wl = WORKLOADS[args.workload]
    iters = ITERS if args.workload != "plain_320x96" else 0
    storage = storage_code(Z, args.storage)
    elt_bytes = STORAGE_BYTES[args.storage]
    pair = config_pair(args.workload)
    H, W, D = wl["h"], wl["w"], wl["d"]

    stream = torch.cuda.Stream(device=dev)
    ctx = Z.ZnccContext(W, H, D, wl["win"], stream=stream)
    left = torch.from_numpy(pair.left).to(dev)
    right = torch.from_numpy(pair.right).to(dev)
    disp = torch.empty((H, W), dtype=torch.int16, device=dev)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)

    def step():
        ctx.zncc_run(left, right, disp, SIG_S, SIG_R, iters, storage)

    tuned = None
    if args.tuning:                             # fixed launch shapes, e.g. for a profiler run
        from paper_2212_00476_gb300 import autotune
        settings = {k: int(v) for k, v in (kv.split("=") for kv in args.tuning.split(","))}
        autotune.apply(ctx, settings)
        tuned = {"settings": settings}
    elif not args.no_autotune:
        from paper_2212_00476_gb300 import autotune
        with torch.cuda.stream(stream):
            tuned = autotune.tune(ctx, left, right, disp, SIG_S, SIG_R, iters, storage)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            flush.zero_()
            step()
    torch.cuda.synchronize()

    # ---- timed region: K steps, per-step CUDA events on the context's stream ----
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    n0 = Z.launch_count()
    with ClockSampler(local) as clk:
        time.sleep(0.3)
        t_wall0 = time.perf_counter()
        with torch.cuda.stream(stream):
            for i in range(args.steps):
                flush.zero_()
                starts[i].record(stream)
                step()
                ends[i].record(stream)
        torch.cuda.synchronize()
        t_wall = time.perf_counter() - t_wall0
    launches = Z.launch_count() - n0
    if world > 1:
        dist.barrier()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    ms = max_over_ranks(sum(step_ms) / len(step_ms), dev)
    clocks = clk.summary()

    # ---- per-kernel durations: the same steps again, each kernel between CUDA events ----
    ctx.profile_enable(True)
    with torch.cuda.stream(stream):
        for _ in range(args.steps):
            flush.zero_()
            step()
    prof = ctx.profile_read()
    ctx.profile_enable(False)
    kinds = {k: v for k, v in prof.items() if algorithmic_bytes(k, wl, elt_bytes)}
    dom = max(kinds, key=lambda k: kinds[k][0])
    dom_ms = kinds[dom][0] / kinds[dom][1]
    dom_bytes = algorithmic_bytes(dom, wl, elt_bytes)
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except (OSError, ValueError):
        pass
    peak = peaks.get("hbm_gbs")
    peak_src = "measured" if peak else "fallback"
    peak = peak or 6800.0
    achieved = dom_bytes / (dom_ms * 1e-3) / 1e9

    # ---- end to end through the public host-buffer call ----
    lh = torch.from_numpy(pair.left).pin_memory().numpy()
    rh = torch.from_numpy(pair.right).pin_memory().numpy()
    dh = torch.empty((H, W), dtype=torch.int16).pin_memory().numpy().view(np.uint16)
    for _ in range(max(1, args.warmup)):
        ctx.zncc_run_host(lh, rh, dh, SIG_S, SIG_R, iters, storage)
    e2e_times = []
    for _ in range(args.steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx.zncc_run_host(lh, rh, dh, SIG_S, SIG_R, iters, storage)
        e2e_times.append(time.perf_counter() - t0)
    e2e_s = max_over_ranks(sum(e2e_times) / len(e2e_times), dev)

    units = W * H * D
    value = replica_throughput(units, world, ms * 1e-3)
    line = {
        "metric": METRIC, "value": round(value, 3), "unit": "Gdisp/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 4),
        "fps": round(world * 1e3 / ms, 2), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "storage": args.storage, "data": "synthetic",
        "config": {"workload": workload_desc(args.workload),
                   "l2": "flushed before every timed step (256 MB write outside the step events)",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                   "step_ms_min": round(min(step_ms), 4), "wall_ms_per_step_incl_flush":
                   round(t_wall * 1e3 / args.steps, 4),
                   "launch_shapes": tuned["settings"] if tuned else "defaults"},
        "roofline": {"bound": "hbm" if iters > 0 else "alu (HBM fraction shown for reference)",
                     "kernel": dom, "achieved": round(achieved, 1),
                     "peak": peak, "peak_source": peak_src, "unit": "GB/s",
                     "frac": round(achieved / peak, 4),
                     "traffic": load_traffic(dom, zbuild._sources_digest(), args.workload, args.storage),
                     "algorithmic_bytes_per_launch": dom_bytes,
                     "launch_ms": round(dom_ms, 5)},
        "roofline_step": step_roofline(W * H * D, iters, elt_bytes, ms, peak, peak_src, clocks),
        "kernels_ms_per_step": {k: round(v[0] / args.steps, 5) for k, v in prof.items()},
        "kernels_on_second_stream": {"kinds": [k for k in ("dt_coef", "ahat_pair") if k in prof],
                                     "note": "timed on the second stream beside the cost kernel, "
                                             "so their spans overlap it and are not additive"},
        "e2e": {"value": round(replica_throughput(units, world, e2e_s), 3), "unit": "Gdisp/s",
                "h2d_bytes_per_step": 2 * W * H, "d2h_bytes_per_step": 2 * W * H,
                "ms_per_step": round(e2e_s * 1e3, 4)},
        "gpu_launches": int(launches),
        "clocks": clocks,
    }

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        times, cores = time_oracle(pair, wl, iters)
        tb = sum(times) / len(times)
        line["cpu_baseline"] = {"value": round(units / tb / 1e9, 6), "unit": "Gdisp/s",
                                "cores": cores, "kind": "oracle",
                                "sample": f"{len(times)} full {W}x{H} D={D} pair(s), "
                                          f"{tb:.2f} s each"}
        if iters == 0:              # the small plain workload: one host core as well
            t1, _ = time_oracle(pair, wl, iters, max_seconds=5.0, max_runs=20, cores=1)
            line["cpu_baseline"]["single_core"] = {"value": round(units / (sum(t1) / len(t1)) / 1e9, 6),
                                                   "unit": "Gdisp/s", "cores": 1,
                                                   "sample": f"{len(t1)} full pair(s)"}
    if rank == 0 and world == 1 and args.workload == "paper_1280x384" and not args.no_extras:
        line["precision"] = precision_leg(Z, ctx, pair, wl, iters, left, right, disp, flush, stream, args)
        sweep, sat = serving_legs(Z, Z.ZNCC_F32, [SERVE_RATE, SERVE_RATE_BUSY], SERVE_REQUESTS,
                                  sat_n=SERVE_SAT_REQUESTS)
        head, busy = sweep
        line["serving"] = {
            "config": SERVE_CONFIG + f"; {SERVE_REQUESTS} requests at {SERVE_RATE:g} and at "
                                     f"{SERVE_RATE_BUSY:g} req/s; saturation: {SERVE_SAT_REQUESTS} "
                                     "requests queued at once",
            "rate_req_per_s": SERVE_RATE,
            "p50_ms": head["batched"]["p50_ms"], "p99_ms": head["batched"]["p99_ms"],
            "throughput_req_per_s": head["batched"]["served_req_per_s"],
            "throughput_gdisp_s": head["batched"]["served_gdisp_s"],
            "p99_breakdown": head["batched"]["p99_breakdown"],
            "plain": {"p50_ms": head["one_pair_per_launch"]["p50_ms"],
                      "p99_ms": head["one_pair_per_launch"]["p99_ms"],
                      "throughput_req_per_s": head["one_pair_per_launch"]["served_req_per_s"],
                      "throughput_gdisp_s": head["one_pair_per_launch"]["served_gdisp_s"],
                      "p99_breakdown": head["one_pair_per_launch"]["p99_breakdown"]},
            "busy": {"rate_req_per_s": SERVE_RATE_BUSY,
                     "batched": {k: busy["batched"][k] for k in ("p50_ms", "p99_ms", "served_req_per_s")},
                     "plain": {k: busy["one_pair_per_launch"][k] for k in ("p50_ms", "p99_ms", "served_req_per_s")}},
            "saturation": sat,
        }
    if rank == 0 and world == 1 and args.workload == "paper_1280x384" and not args.no_extras:
        ctx.close()
        torch.cuda.synchronize()
        line["configs"] = other_configs(args)
    if rank == 0:
        print(json.dumps(line))
    ctx.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


OTHER_CONFIGS = [("plain_320x96", ["--workload", "plain_320x96"]),
                 ("batch_uneven16", ["--workload", "batch_uneven16"]),
                 ("precision_1920x1080", ["--workload", "precision_sweep"])]


def other_configs(args):
    """The other configurations of the paper-shaped workload family, each in a child process
    after the timed region (so that their lines reach the record of a default run): the plain
    320x96 pair (ZNCC + WTA, latency), 16 uneven pairs batched under a CUDA graph against one
    pair per launch, and the 1920x1080 precision sweep (F32 / F16 / FastDT I8 against the FP64
    oracle). A child that fails is recorded with its error instead."""
    out = {}
    for name, extra in OTHER_CONFIGS:
        cmd = [sys.executable, os.path.abspath(__file__), *extra, "--steps", "10", "--warmup", "3",
               "--no-cpu-baseline"]
        if args.no_autotune:
            cmd.append("--no-autotune")
        t0 = time.perf_counter()
        try:
            p = subprocess.run(cmd, capture_output=True, text=True, timeout=600)
            lines = [x for x in p.stdout.splitlines() if x.startswith("{")]
            if p.returncode != 0 or not lines:
                out[name] = {"error": f"exit {p.returncode}: {(p.stderr or p.stdout)[-400:]}"}
            else:
                out[name] = json.loads(lines[-1])
        except (subprocess.TimeoutExpired, OSError, ValueError) as e:
            out[name] = {"error": f"{type(e).__name__}: {e}"}
        out[name]["wall_s"] = round(time.perf_counter() - t0, 1)
    return out


def precision_leg(Z, ctx, pair, wl, iters, left, right, disp, flush, stream, args, steps=10):
    """The same pair with F32, F16 and FastDT I8 volume storage: step time (CUDA events, L2
    flushed, each storage autotuned) and the disparity map against the FP64 oracle's: the share
    of pixels that differ, and of those whose oracle best-vs-second gap is at least 1e-5 A_hat
    (away from near-ties)."""
    import torch

    import oracle
    ref, gap = oracle.run(pair.left, pair.right, wl["d"], wl["win"] // 2, SIG_S, SIG_R, iters)
    A = oracle.ones_response(pair.left, SIG_S, SIG_R, iters)
    clear = gap >= 1e-5 * A
    out = {"reference": "FP64 oracle map of the same pair",
           "pixels": int(ref.size), "pixels_away_from_ties": int(clear.sum())}
    for name in ("f32", "f16", "i8"):
        st = storage_code(Z, name)
        tuned = None
        if not args.no_autotune:
            from paper_2212_00476_gb300 import autotune
            with torch.cuda.stream(stream):
                tuned = autotune.tune(ctx, left, right, disp, SIG_S, SIG_R, iters, st)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        with torch.cuda.stream(stream):
            for _ in range(3):
                ctx.zncc_run(left, right, disp, SIG_S, SIG_R, iters, st)
            for a, b in ev:
                flush.zero_()
                a.record(stream)
                ctx.zncc_run(left, right, disp, SIG_S, SIG_R, iters, st)
                b.record(stream)
        torch.cuda.synchronize()
        ms = sum(a.elapsed_time(b) for a, b in ev) / steps
        got = disp.cpu().numpy().view(np.uint16)
        diff = got != ref
        out[name] = {"ms_per_step": round(ms, 4),
                     "gdisp_s": round(wl["w"] * wl["h"] * wl["d"] / (ms * 1e-3) / 1e9, 3),
                     "mismatch_rate": round(float(diff.mean()), 7),
                     "mismatch_rate_away_from_ties": round(float((diff & clear).sum() / max(1, clear.sum())), 7),
                     "launch_shapes": tuned["settings"] if tuned else "defaults"}
    # leave the context with the F32 shapes the timed region used
    if not args.no_autotune:
        from paper_2212_00476_gb300 import autotune
        with torch.cuda.stream(stream):
            autotune.tune(ctx, left, right, disp, SIG_S, SIG_R, iters, Z.ZNCC_F32)
    return out


def run_batch(args):
    """16 seeded pairs of uneven size, disparity range and window (sizes from {640x192,
    1280x384, 1242x375, 1920x1080}, D from {64, 128, 192}, windows from {7, 9, 11}) through
    one batched fused run per step, replayed from a captured CUDA graph; compared with the
    same pairs run one zncc_run after another."""
    import torch

    from paper_2212_00476_gb300 import zncc as Z
    from synth import batch_specs, make_pair

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    specs = batch_specs(16, 300)
    stream = torch.cuda.Stream(device=dev)
    ctxs, L, R, D, units, pairs = [], [], [], [], 0, []
    for sp in specs:
        p = make_pair(sp["h"], sp["w"], sp["max_disp"], sp["seed"], disp="planes", occlusion_frac=0.05)
        pairs.append(p)
        ctxs.append(Z.ZnccContext(sp["w"], sp["h"], sp["max_disp"], sp["win"], stream=stream))
        L.append(torch.from_numpy(p.left).to(dev))
        R.append(torch.from_numpy(p.right).to(dev))
        D.append(torch.empty((sp["h"], sp["w"]), dtype=torch.int16, device=dev))
        units += sp["w"] * sp["h"] * sp["max_disp"]
    storage = storage_code(Z, args.storage)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)

    def batched():
        Z.zncc_run_batch(ctxs, L, R, D, SIG_S, SIG_R, ITERS, storage)

    def sequential():
        for c, l, r, d in zip(ctxs, L, R, D):
            c.zncc_run(l, r, d, SIG_S, SIG_R, ITERS, storage)

    def timed(fn, graph=None):
        with torch.cuda.stream(stream):
            for _ in range(args.warmup):
                flush.zero_()
                graph.replay() if graph else fn()
        ms = []
        for _ in range(args.steps):
            with torch.cuda.stream(stream):
                flush.zero_()
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(stream)
                graph.replay() if graph else fn()
                b.record(stream)
            b.synchronize()
            ms.append(a.elapsed_time(b))
        return sum(ms) / len(ms)

    tuned = {}
    if not args.no_autotune:                   # launch shapes tuned per pair shape (cached)
        from paper_2212_00476_gb300 import autotune
        with torch.cuda.stream(stream):
            for c, l, r, d in zip(ctxs, L, R, D):
                res = autotune.tune(c, l, r, d, SIG_S, SIG_R, ITERS, storage)
                tuned[autotune.shape_key(c, ITERS, storage)] = res["settings"]
    with torch.cuda.stream(stream):
        batched()                              # allocations and launch plans before capture
        sequential()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        batched()
    n0 = Z.launch_count()
    ms_graph = timed(None, g)
    ms_batch = timed(batched)
    launches = (Z.launch_count() - n0) // max(1, args.steps + args.warmup)
    ms_seq = timed(sequential)
    line = {
        "metric": "aggregate Gdisp/s, 16 uneven pairs (ZNCC+DT+WTA), batched vs one pair per launch",
        "value": round(units / (ms_graph * 1e-3) / 1e9, 3), "unit": "Gdisp/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_graph, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": args.storage,
        "data": "synthetic",
        "config": {"workload": "batch_uneven16: " + ", ".join(
            f"{sp['w']}x{sp['h']}/D{sp['max_disp']}/w{sp['win']}" for sp in specs),
            "disparities_per_step": units, "iters": ITERS,
            "l2": "flushed before every timed step (256 MB write outside the step events)"},
        "batched_graph_ms": round(ms_graph, 4), "batched_ms": round(ms_batch, 4),
        "one_pair_per_launch_ms": round(ms_seq, 4),
        "speedup_vs_one_pair_per_launch": round(ms_seq / ms_graph, 3),
        "launches_per_batched_step": int(launches),
        "launch_shapes": tuned or "defaults",
    }
    if not args.no_cpu_baseline:               # the oracle pair by pair, about 12 s of it
        import oracle
        oracle.load()
        cores = host_cores()
        done, t_all, per_pair = 0, 0.0, []
        for sp, p in zip(specs, pairs):
            t0 = time.perf_counter()
            oracle.run(p.left, p.right, sp["max_disp"], sp["win"] // 2, SIG_S, SIG_R, ITERS, nthreads=cores)
            dt = time.perf_counter() - t0
            t_all += dt
            done += sp["w"] * sp["h"] * sp["max_disp"]
            per_pair.append(f"{sp['w']}x{sp['h']}/D{sp['max_disp']}/w{sp['win']}: {dt:.2f} s")
            if t_all > 12.0:
                break
        line["cpu_baseline"] = {"value": round(done / t_all / 1e9, 6), "unit": "Gdisp/s", "cores": cores,
                                "kind": "oracle", "sample": f"the first {len(per_pair)} of the 16 pairs, "
                                                            "one after another: " + "; ".join(per_pair)}
    print(json.dumps(line))
    for c in ctxs:
        c.close()
    return 0


def run_precision(args):
    """FP32 vs FP16 vs FastDT (I8) volume storage at 1920x1080, D = 256, 11x11, 3 DT
    iterations against the FP64 oracle: the largest |aggregated cost - oracle| / A_hat over the
    whole volume (F32, F16: the unfused chain zncc_cost_volume + dt_aggregate, which rounds
    every stored pair to the storage type), and the disparity maps of the fused path: the
    share of pixels that differ from the oracle's map, all pixels and those whose oracle
    best-second gap is at least 1e-5 * A_hat (I8 also against the oracle's FastDT chain), and
    the share of valid pixels within one disparity of the ground truth, next to the oracle's.
    Also the fused path's time per pair for each storage type."""
    import torch

    import oracle
    from paper_2212_00476_gb300 import zncc as Z
    from synth import config_pair

    wl = WORKLOADS["precision_1920x1080"]
    H, W, D, win = wl["h"], wl["w"], wl["d"], wl["win"]
    pair = config_pair("precision_1920x1080")
    t0 = time.perf_counter()
    ref, gap, cref = oracle.run(pair.left, pair.right, D, win // 2, SIG_S, SIG_R, ITERS, want_cost=True)
    ahat = oracle.ones_response(pair.left, SIG_S, SIG_R, ITERS)
    ref_fast, _ = oracle.run_fastdt(pair.left, pair.right, D, win // 2, SIG_S, SIG_R, ITERS)
    t_oracle = time.perf_counter() - t0

    def gt_accuracy(m):
        return round(float((np.abs(m.astype(np.int64) - pair.gt) <= 1)[pair.valid].mean()), 6)
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    ctx = Z.ZnccContext(W, H, D, win)
    left = torch.from_numpy(pair.left).to(dev)
    right = torch.from_numpy(pair.right).to(dev)
    disp = torch.empty((H, W), dtype=torch.int16, device=dev)
    clear = gap >= 1e-5 * ahat
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)
    result = {}

    def volume_error(tdt, st):
        vol = torch.empty((H, W, D), dtype=tdt, device=dev)
        ctx.zncc_cost_volume(left, right, vol, st)
        ctx.dt_aggregate(left, vol, SIG_S, SIG_R, ITERS, st)
        torch.cuda.synchronize()
        worst, worst_normal = 0.0, None
        for y0 in range(0, H, 60):
            g = vol[y0:y0 + 60].float().cpu().numpy().astype(np.float64)
            a = ahat[y0:y0 + 60, :, None]
            e = np.abs(g - cref[y0:y0 + 60]) / a
            worst = max(worst, float(e.max()))
            normal = np.broadcast_to(a >= 2.0 ** -14, e.shape)
            if normal.any():
                worst_normal = max(worst_normal or 0.0, float(e[normal].max()))
        return worst, worst_normal

    for name, st, tdt in (("f32", Z.ZNCC_F32, torch.float32), ("f16", Z.ZNCC_F16, torch.float16),
                          ("i8", Z.ZNCC_I8, None)):
        worst, worst_normal = None, None
        if tdt is not None:                 # the FastDT codes exist only inside the fused path
            worst, worst_normal = volume_error(tdt, st)
        ms = []
        for i in range(args.warmup + args.steps):
            flush.zero_()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            ctx.zncc_run(left, right, disp, SIG_S, SIG_R, ITERS, st)
            b.record()
            b.synchronize()
            if i >= args.warmup:
                ms.append(a.elapsed_time(b))
        got = disp.cpu().numpy().view(np.uint16)
        diff = got != ref
        result[name] = {"max_abs_err_over_ahat": worst,
                        "max_abs_err_over_ahat_where_ahat_ge_2^-14": worst_normal,
                        "map_mismatch_rate": round(float(diff.mean()), 6),
                        "map_mismatch_rate_clear_pixels": round(float(diff[clear].mean()), 6),
                        "gt_within_1px": gt_accuracy(got),
                        "fused_ms_per_pair": round(sum(ms) / len(ms), 4),
                        "fused_gdisp_s": round(W * H * D / (sum(ms) / len(ms) * 1e-3) / 1e9, 3)}
        if name == "i8":
            result[name]["map_mismatch_rate_vs_oracle_fastdt"] = round(float((got != ref_fast).mean()), 6)
    ctx.close()
    line = {
        "metric": "precision: FP32 vs FP16 vs FastDT 8-bit volume storage vs the FP64 oracle, "
                  "1920x1080 D=256 11x11",
        "value": result["f16"]["map_mismatch_rate"], "unit": "share of pixels (F16 map vs oracle)",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": workload_desc("precision_1920x1080", "F32/F16/I8"),
                   "oracle_gt_within_1px": {"f64": gt_accuracy(ref), "fastdt": gt_accuracy(ref_fast)},
                   "near_tie_pixels": round(float(1 - clear.mean()), 6),
                   "pixels_with_ahat_below_2^-14": round(float((ahat < 2.0 ** -14).mean()), 6),
                   "volume_error_path": "unfused zncc_cost_volume + dt_aggregate (each stored pair "
                                        "rounded to the storage type, no A_hat normalisation)",
                   "oracle_seconds": round(t_oracle, 2),
                   "l2": "flushed before every timed pair (256 MB write outside the events)"},
        "f32": result["f32"], "f16": result["f16"], "i8": result["i8"],
    }
    print(json.dumps(line))
    return 0


SERVE_RATE, SERVE_RATE_BUSY, SERVE_REQUESTS, SERVE_SAT_REQUESTS = 200.0, 500.0, 1000, 300


def serving_legs(Z, storage, rates, n, sat_n=0, seed=5):
    """Poisson arrivals (seed 5) of requests of size {640x192, 1280x384, 1920x1080} and D
    {64, 128, 256}, 9x9, 3 DT iterations, through the serving calls with continuous batching
    (max_slots 32) and one pair per launch (max_slots 1), under a 40 GB budget. Latency = time
    from a request's scheduled arrival until serve_poll returns its map; one loop submits on
    schedule and polls every outstanding ticket. The images of a (size, D) shape come from one
    seeded pair (seed 500000 + shape index), reused by every request of that shape. Per rate:
    p50/p99/max latency, served throughput, and the server's breakdown of the requests at or
    above p99 (host queue, wait on the stream, uploads, fused run, result copies). sat_n > 0
    adds a saturation leg: sat_n requests offered at 20000 req/s (all queued at once), whose
    served rate is each server's capacity on this mix."""
    from synth.stereo import SERVE_DISPS, SERVE_SIZES, make_pair, serving_requests

    shapes = [(h, w, d) for (h, w) in SERVE_SIZES for d in SERVE_DISPS]
    pool = {sh: make_pair(sh[0], sh[1], sh[2], 500000 + i, disp="planes", occlusion_frac=0.05)
            for i, sh in enumerate(shapes)}
    outs = {sh: np.zeros(sh[:2], np.uint16) for sh in shapes}
    budget = 40 * 10**9
    parts = ("queue_ms", "device_wait_ms", "h2d_ms", "run_ms", "d2h_ms")

    def serve(rate, max_slots, n):
        reqs = serving_requests(n, rate, seed=seed)
        with Z.ZnccServer(budget, max_slots) as srv:
            for sh in shapes:                                   # contexts exist before timing
                p = pool[sh]
                t = srv.submit(p.left, p.right, sh[2], 9, SIG_S, SIG_R, ITERS, storage)
                assert srv.poll(t, outs[sh], 60_000_000) == Z.ZNCC_OK, srv.last_error()
            lat, pending, i, units = [], {}, 0, 0
            t0 = time.perf_counter()
            while i < n or pending:
                now = time.perf_counter() - t0
                while i < n and reqs[i]["t"] <= now:
                    r = reqs[i]
                    sh = (r["h"], r["w"], r["max_disp"])
                    p = pool[sh]
                    pending[srv.submit(p.left, p.right, sh[2], 9, SIG_S, SIG_R, ITERS, storage)] = (sh, r["t"])
                    units += sh[0] * sh[1] * sh[2]
                    i += 1
                done = []
                for tk, (sh, ta) in pending.items():
                    st, tm = srv.poll_timed(tk, outs[sh], 0)
                    if st == Z.ZNCC_OK:
                        lat.append((time.perf_counter() - t0 - ta, sh, tm))
                        done.append(tk)
                    elif st != Z.ZNCC_ENOTREADY:
                        raise RuntimeError(f"request failed: {Z.STATUS_NAMES[st]} {srv.last_error()}")
                for tk in done:
                    del pending[tk]
                if not done:
                    time.sleep(2e-5)
            span = time.perf_counter() - t0
        lat.sort(key=lambda e: e[0])
        q = lambda f: lat[min(len(lat) - 1, int(f * len(lat)))][0] * 1e3
        tail = [e for e in lat[min(len(lat) - 1, int(0.99 * len(lat))):] if e[2]]
        mix = {}
        for e in tail:
            k = f"{e[1][1]}x{e[1][0]}_D{e[1][2]}"
            mix[k] = mix.get(k, 0) + 1
        brk = {k: round(sum(e[2][k] for e in tail) / len(tail), 3) for k in parts} if tail else None
        if brk:
            brk["client_ms"] = round(sum(e[0] * 1e3 - e[2]["total_ms"] for e in tail) / len(tail), 3)
            brk["batch_pairs"] = round(sum(e[2]["batch_pairs"] for e in tail) / len(tail), 2)
            brk["shapes"] = mix
            brk["requests"] = len(tail)
        return {"p50_ms": round(q(0.50), 3), "p99_ms": round(q(0.99), 3), "max_ms": round(lat[-1][0] * 1e3, 3),
                "requests": n, "span_s": round(span, 3), "served_req_per_s": round(n / span, 1),
                "served_gdisp_s": round(units / span / 1e9, 3), "p99_breakdown": brk}

    out = []
    for rate in rates:
        out.append({"rate_req_per_s": rate, "batched": serve(rate, 32, n),
                    "one_pair_per_launch": serve(rate, 1, n)})
    sat = None
    if sat_n:
        sat = {"offered_req_per_s": 20000.0, "requests": sat_n,
               "batched": serve(20000.0, 32, sat_n), "one_pair_per_launch": serve(20000.0, 1, sat_n)}
        for k in ("batched", "one_pair_per_launch"):
            sat[k] = {m: sat[k][m] for m in ("served_req_per_s", "served_gdisp_s", "p50_ms", "p99_ms")}
    return out, sat


SERVE_CONFIG = ("serving: Poisson arrivals seed 5; sizes 640x192/1280x384/1920x1080, D 64/128/256, "
                "9x9, sigma_s 20, sigma_r 0.1, 3 iterations; 40 GB budget; continuous batching "
                "(max_slots 32) vs one pair per launch (max_slots 1)")


def run_serving(args):
    """C5 on its own: the serving legs at every rate of --rates (--requests each) and a
    saturation leg."""
    from paper_2212_00476_gb300 import zncc as Z

    import torch
    torch.cuda.set_device(0)
    storage = storage_code(Z, args.storage)
    rates = [float(r) for r in args.rates.split(",")]
    sweep, sat = serving_legs(Z, storage, rates, args.requests, sat_n=max(SERVE_SAT_REQUESTS, args.requests // 4))
    head = sweep[0]
    line = {
        "metric": f"served p50/p99 latency at {rates[0]:g} req/s (continuous batching vs one pair per launch)",
        "value": head["batched"]["p99_ms"], "unit": "ms (p99)", "n_gpus": 1, "steps": args.requests,
        "warmup": 9, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "storage": args.storage, "data": "synthetic",
        "config": {"workload": SERVE_CONFIG, "l2": "not flushed (a live request stream)"},
        "p50_ms": head["batched"]["p50_ms"], "p99_ms": head["batched"]["p99_ms"],
        "plain_p50_ms": head["one_pair_per_launch"]["p50_ms"],
        "plain_p99_ms": head["one_pair_per_launch"]["p99_ms"],
        "sweep": sweep, "saturation": sat,
    }
    print(json.dumps(line))
    return 0


def run_ablation(args):
    """The paper's Z²-ZNCC vs "original" progressive-scan comparison (Sec. V-B, Fig.
    ZNCC_compare) as an ablation of this repository's kernels: the cost volume of the
    1280x384 pair (seed 2) by the packed-column cost kernel (zncc_cost_volume), by the
    progressive-scan kernel (zncc_cost_volume_scan) and by the tensor-core banded product
    (zncc_cost_volume_mma), F32 volume, window sides 3..15, D = 96 and 128; CUDA events around
    each call, L2 flushed before each. The three give identical values (tested)."""
    import torch

    from paper_2212_00476_gb300 import zncc as Z
    from synth import config_pair

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    pair = config_pair("paper_1280x384")
    H, W = pair.left.shape
    left = torch.from_numpy(pair.left).to(dev)
    right = torch.from_numpy(pair.right).to(dev)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)

    def timed(fn):
        ms = []
        for i in range(args.warmup + args.steps):
            flush.zero_()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            fn()
            b.record()
            b.synchronize()
            if i >= args.warmup:
                ms.append(a.elapsed_time(b))
        return sorted(ms)[len(ms) // 2]

    rows = []
    for D in (96, 128):
        vol = torch.empty((H, W, D), dtype=torch.float32, device=dev)
        for win in (3, 5, 7, 9, 11, 13, 15):
            ctx = Z.ZnccContext(W, H, D, win)
            t_packed = timed(lambda: ctx.zncc_cost_volume(left, right, vol))
            t_scan = timed(lambda: ctx.zncc_cost_volume_scan(left, right, vol))
            t_mma = timed(lambda: ctx.zncc_cost_volume_mma(left, right, vol))
            rows.append({"win": win, "D": D, "packed_ms": round(t_packed, 4), "scan_ms": round(t_scan, 4),
                         "mma_ms": round(t_mma, 4), "speedup": round(t_scan / t_packed, 3),
                         "mma_vs_packed": round(t_packed / t_mma, 3)})
            ctx.close()
        del vol
    at9 = next(r for r in rows if r["win"] == 9 and r["D"] == 128)
    line = {
        "metric": "ZNCC cost volume time, packed-column kernel vs progressive scan (speedup at 9x9, D=128)",
        "value": at9["speedup"], "unit": "x (scan time / packed time)", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "int32 numerator, f32 cost", "data": "synthetic",
        "config": {"workload": "zncc_ablation: 1280x384 pair (seed 2), F32 volume, sides 3..15, D 96 and 128",
                   "l2": "flushed before every timed call (256 MB write outside the events)",
                   "paper_tx2_d128": "Z2-ZNCC 11.31 ms vs original 18.05 ms at side 3, 34.35 vs 72.09 ms at side 15"},
        "rows": rows,
    }
    print(json.dumps(line))
    return 0


def run_plane_ablation(args):
    """The plane-resident fused path (each disparity plane kept in shared memory through the
    cost, every DT pass pair and the WTA; ZNCC_TUNE_PLANE = 1) against the streaming path (the
    cost volume in device memory) on the pair shapes it applies to: 320x96 and 640x192 pairs of
    the configuration generator (seed 3), 9x9 window, 3 DT iterations, F32; CUDA events around
    each fused run, L2 flushed before each. The two give the same disparity maps (tested; the
    mismatch share is reported)."""
    import numpy as np
    import torch

    from paper_2212_00476_gb300 import zncc as Z
    from synth import make_pair

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)
    rows = []
    for (H, W, D) in ((96, 320, 32), (96, 320, 128), (192, 640, 64), (192, 640, 128), (192, 640, 256)):
        p = make_pair(H, W, min(D, 128), seed=3)
        left = torch.from_numpy(p.left).to(dev)
        right = torch.from_numpy(p.right).to(dev)
        row = {"W": W, "H": H, "D": D}
        maps = {}
        for plane in (1, 0):
            ctx = Z.ZnccContext(W, H, D, 9)
            ctx.set_tuning(Z.ZNCC_TUNE_PLANE, plane)
            disp = torch.empty((H, W), dtype=torch.int16, device=dev)
            ms = []
            for i in range(args.warmup + args.steps):
                flush.zero_()
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record()
                ctx.zncc_run(left, right, disp, 20.0, 0.1, 3, Z.ZNCC_F32)
                b.record()
                b.synchronize()
                if i >= args.warmup:
                    ms.append(a.elapsed_time(b))
            t = sorted(ms)[len(ms) // 2]
            row["plane_ms" if plane else "streaming_ms"] = round(t, 4)
            row["plane_gdisp_s" if plane else "streaming_gdisp_s"] = round(W * H * D / t / 1e6, 2)
            maps[plane] = disp.cpu().numpy()
            ctx.close()
        row["map_mismatch"] = float(np.mean(maps[0] != maps[1]))
        rows.append(row)
    at = next(r for r in rows if r["W"] == 640 and r["D"] == 128)
    line = {
        "metric": "fused ZNCC+DT+WTA time, plane-resident path vs streaming path (ratio at 640x192, D=128)",
        "value": round(at["streaming_ms"] / at["plane_ms"], 3), "unit": "x (streaming time / plane time)",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "plane_ablation: 320x96 and 640x192 pairs (seed 3), 9x9, 3 iterations, F32",
                   "l2": "flushed before every timed call (256 MB write outside the events)"},
        "rows": rows,
    }
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["gb300", "reference"], default="gb300")
    ap.add_argument("--storage", choices=["f32", "f16", "i8"], default="f32")
    ap.add_argument("--workload", choices=sorted(WORKLOADS) + ["batch_uneven16", "serving", "precision_sweep",
                                                           "zncc_ablation", "plane_ablation"],
                    default="paper_1280x384")
    ap.add_argument("--rates", default="200,500,1000,2000", help="serving: arrival rates (req/s)")
    ap.add_argument("--requests", type=int, default=2000, help="serving: requests per rate")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="default workload: skip the precision and serving legs of the JSON line")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--tuning", default="", help="fixed launch shapes instead of autotuning, "
                    "e.g. row_minb2=0,row_spb=8")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "gb300":
        args.warmup = 3
    if args.impl == "reference":
        if args.workload not in WORKLOADS:
            print(json.dumps({"impl": "reference", "unavailable": f"the reference arm times the oracle on "
                              f"the single-pair workloads {sorted(WORKLOADS)} only"}))
            return 0
        return run_reference(args)
    if args.workload == "serving":
        return run_serving(args)
    if args.workload == "precision_sweep":
        return run_precision(args)
    if args.workload == "zncc_ablation":
        return run_ablation(args)
    if args.workload == "plane_ablation":
        return run_plane_ablation(args)
    if args.workload == "batch_uneven16":
        return run_batch(args)
    return run_gb300(args)


if __name__ == "__main__":
    sys.exit(main())
