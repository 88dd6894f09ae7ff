#!/usr/bin/env python
"""Throughput of the data-parallel pc-engine: pattern-mode updates per second.

Workload: the far-field 4-mode configuration (probe 128 x 128, 4 probe modes,
900 Fermat-spiral positions, 640 x 640 object, 5 % bandwidth, sigma = 1.5,
1e6 photons) from the seeded generator. One step is one full iteration of the
engine over all positions: exit waves, propagation, the Gaussian intensity
model and modulus constraint, back-propagation, the object / probe
scatter-add update, the complex constraint (active in every timed step) and
the FP64 error. Inputs are resident in HBM when timing starts; L2 is flushed
with a 256 MiB write before every timed step (outside the step's events).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (launched by torch.distributed.run) every rank runs an independent
replica of the workload (the engine does not shard one reconstruction across
GPUs); the value is the sum over ranks divided by the slowest rank's time.
--impl reference times the FP64 CPU oracle on the host cores instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

# the CPU oracle legs report rates on a stated number of cores: BLAS / OpenMP pools default to one
# thread (set before numpy loads its BLAS)
for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import numpy as np  # noqa: E402

ROOT = os.path.dirname(os.path.abspath(__file__))


def cpu_threads():
    """Threads the CPU oracle legs may use (the BLAS pool size set above or by the caller)."""
    try:
        return max(1, int(os.environ.get("OPENBLAS_NUM_THREADS", "1")))
    except ValueError:
        return 1
sys.path.insert(0, ROOT)

METRIC = "pattern-mode updates/s"
FP32_LANES_PER_SM = 128
N_SMS = 152
SM_MAX_MHZ = 2070.0
L2_FLUSH_BYTES = 256 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-time-to-nrmse", action="store_true",
                    help="skip the warm-start time-to-NRMSE record that the benchmark workload's line carries")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="far128x4",
                    help="far128x4: the benchmark workload; the others for reference runs")
    return ap.parse_args()


MONO_LINES5 = [1.0, 1.0125, 1.025, 1.0375, 1.05]
MONO_WHITE32 = [1.0 + 0.75 * j / 31 for j in range(32)]
MONO_WHITE32_W = [math.exp(-0.5 * ((a - 1.3) / 0.2) ** 2) for a in MONO_WHITE32]

WORKLOADS = {
    "far128x4": (1, "far-field 4-mode pc-engine iteration (probe 128^2, K=4, N=900 Fermat spiral, "
                    "object 640^2, 5% bandwidth, sigma 1.5, 1e6 photons)"),
    "near256x8": (2, "near-field 8-mode pc-engine iteration (Fresnel F=10, probe 256^2, K=8, N=256 raster, "
                     "object 1024^2, sigma 2, 1e5 photons)"),
    "far64x1": (0, "far-field single-mode pc-engine iteration (probe 64^2, N=100 raster, object 192^2, "
                   "sigma 1, 1e5 photons)"),
    "far128x4-rpie": (1, "far128x4 with the rPIE step rule (alpha 0.2 object, 0.5 probe)",
                      dict(step_rule="rpie", rpie_alpha_obj=0.2, rpie_alpha_probe=0.5)),
    "far128x4-mb32": (1, "far128x4 as the mini-batch (sequential) engine: batches of 32 positions in a Philox "
                         "order, one fused launch and one update per batch (29 per iteration), rPIE steps",
                      dict(minibatch=32, order_seed=11, step_rule="rpie", rpie_alpha_obj=0.2,
                           rpie_alpha_probe=0.5)),
    "far128x4-dm": (1, "far128x4 with the pc-DM engine (exit-wave state per position and mode in HBM)",
                    dict(engine="dm")),
    "mono128": (1, "numerical monochromatisation (CGLS, k=25) of the 900 broadband 128^2 patterns of far128x4, "
                   "5-line spectrum of 5% bandwidth about the shortest wavelength (the one the data were "
                   "generated with), one CTA per pattern",
                dict(mono=(MONO_LINES5, [0.2] * 5, 25))),
    "mono128-white": (1, "numerical monochromatisation (CGLS, k=25) of 900 patterns of 128^2 with a white-light "
                         "spectrum: 32 lines over a factor 1.75 (400-700 nm about 400 nm), Gaussian weights; the "
                         "patterns of far128x4 stand in for white-light data (the cost does not depend on b)",
                      dict(mono=(MONO_WHITE32, MONO_WHITE32_W, 25))),
    "mono256-white": (2, "numerical monochromatisation (CGLS, k=25) of 256 patterns of 256^2 with the 32-line "
                         "white-light spectrum (one cluster of four CTAs per pattern); the patterns of near256x8 "
                         "stand in for white-light data (the cost does not depend on b)",
                      dict(mono=(MONO_WHITE32, MONO_WHITE32_W, 25))),
    "batch64": (3, "64 independent reconstructions of uneven sizes (probe 64-256, 100-1600 positions, K 1-4, "
                   "far/near 50/50, sigma 0.5-3), one CUDA graph launch per iteration"),
    "unet128": (None, "warm-start U-Net forward (inference) over 64 synthetic 128^2 patterns, C = 32, random-"
                      "initialised weights: one step = one estimate (the network's seven 3x3 convolutions on "
                      "tcgen05, pooling, upsampling, the sigma head, the stitch into a 256^2 object, the median)"),
    "warmstart": (4, "time to intensity NRMSE <= 0.05 against the noise-free patterns: flat start with the true "
                     "sigma vs the learned warm start (U-Net trained on 200k forward-model patterns, 64 sampled "
                     "patterns stitched, median sigma); electron-like crystal, probe 128^2, 64x64 raster step 2 px, "
                     "object 256^2, sigma 2, intensity-blur engine model; variant with 1.0 rad peaks at 2e4 "
                     "counts/pattern (at 0.1 rad / 200 counts the comparison is degenerate; that case reports "
                     "the sigma estimate)"),
}
_WORKLOAD = "far128x4"


def workload():
    from synth import make_problem

    prob = make_problem(WORKLOADS[_WORKLOAD][0])
    params = dict(prob.params, windows=[(1, 1 << 30)])  # complex constraint in every step
    if len(WORKLOADS[_WORKLOAD]) > 2:
        params.update(WORKLOADS[_WORKLOAD][2])
    return prob, params


def config_of(prob, extra=None):
    p = prob.params
    cfg = {"workload": WORKLOADS[_WORKLOAD][1],
           "M": p["M"], "K": p["K"], "N": p["N"], "object": [p["obj_h"], p["obj_w"]], "geometry": p["geometry"],
           "blur": p["blur_domain"], "kernel_size": p["kernel_size"], "complex_constraint": "every step",
           "step": "one iteration over all positions", "l2": "flushed before each timed step (256 MiB write)"}
    if extra:
        cfg.update(extra)
    return cfg


def algorithmic_flops(M, K, N, near, dm=False):
    """Nominal FLOPs of one iteration: 5 M^2 log2(M^2) per 2-D FFT (2 per pattern-mode in the far
    field, 4 in the near field), 26 FLOP per pixel per mode and 55 FLOP per pixel per pattern for
    the elementwise work (exit wave, modulus, blur, ratio, contributions, error). pc-DM propagates
    the estimate as well (one more forward propagation per mode, 12 more FLOP per pixel per mode
    for the reflected wave and the state, one more blur and error pass, 30 FLOP per pixel)."""
    fft = 5.0 * M * M * math.log2(M * M)
    per_mode = ((6 if near else 3) if dm else (4 if near else 2)) * fft + (38.0 if dm else 26.0) * M * M
    return N * K * per_mode + N * (85.0 if dm else 55.0) * M * M


# ------------------------------------------------------------------ clocks
class ClockSampler:
    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except FileNotFoundError:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.2)
        self.proc.terminate()
        self.proc.wait()
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 9:
                rows.append(f)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        loaded = [s for s in sm if mx and s > 0.5 * max(mx)] or sm
        return {"sm_mhz": statistics.median(loaded) if loaded else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------------ distributed helpers
def dist_setup(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist

        backend = "nccl" if args.impl == "ours" else "gloo"
        if backend == "nccl":
            import torch

            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist

        dist.barrier()


def max_over_ranks(ws, value, device=None):
    if ws == 1:
        return value
    import torch
    import torch.distributed as dist

    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------------ CPU oracle timing
def oracle_rate(prob, params, n_positions, iterations=1):
    import oracle

    prm = oracle.Params.from_dict(dict(params, N=n_positions))
    t0 = time.perf_counter()
    oracle.iterate(prob.I[:n_positions], prob.positions[:n_positions], prob.O0, prob.P0, prm, iterations)
    dt = time.perf_counter() - t0
    return n_positions * prob.K * iterations / dt, dt


# ---- the oracle on every host core: independent replicas of one bounded oracle iteration, one per
# worker process (spawned, so no worker inherits a CUDA context); the rate is all units / wall time
_CPU_PROB = None


def _cpu_worker_init(cfg):
    global _CPU_PROB
    from synth import make_problem

    _CPU_PROB = make_problem(cfg)


def _cpu_worker(job):
    n_pos, params = job
    return oracle_rate(_CPU_PROB, params, n_pos)[1]


def oracle_rate_all_cores(cfg, params, n_pos, workers):
    import multiprocessing as mp

    ctx = mp.get_context("spawn")
    with ctx.Pool(workers, initializer=_cpu_worker_init, initargs=(cfg,)) as pool:
        pool.map(_cpu_worker, [(4, params)] * workers, chunksize=1)  # imports and a first small call
        t0 = time.perf_counter()
        pool.map(_cpu_worker, [(n_pos, params)] * workers, chunksize=1)
        wall = time.perf_counter() - t0
    K = params["K"]
    return workers * n_pos * K / wall, wall


def traffic_record(kernel_tag, name="fused_kernel_traffic.json", workload="far128x4"):
    """DRAM bytes per launch of a kernel from a committed ncu summary, if it was taken on the current
    kernel source (hash match) and this workload; None otherwise."""
    path = os.path.join(ROOT, "profiles", name)
    if not os.path.exists(path):
        return None
    try:
        rec = json.load(open(path))
    except ValueError:
        return None
    if rec.get("source_sha256") != kernel_tag or rec.get("bench_workload", "far128x4") != workload:
        return None
    return rec.get("dram_bytes_per_launch_full_size")


def kernel_source_hash(files=("cluster.cuh", "fft.cuh", "fused_common.cuh", "pc_fused_seq.cu"), struct="FusedArgs"):
    """Hash of what a kernel is compiled from: its sources and its argument struct."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2406_06640_gb300", "csrc")
    for f in files:
        h.update(open(os.path.join(csrc, f), "rb").read())
    hdr = open(os.path.join(csrc, "engine.h")).read()
    i = hdr.find("struct " + struct)
    h.update(hdr[i:hdr.find("};", i)].encode() if i >= 0 else b"")
    return h.hexdigest()


def kernel_label(prob, params):
    if prob.M > 128:
        return "staged passes (M=256)"
    geo = "near" if params["geometry"] == "near" else "far"
    if params.get("minibatch", 0):
        return f"pc_seq_kernel<{prob.M}, {geo}> per batch with its update kernels (events around the batch loop)"
    if params.get("engine") == "dm":
        return f"pc_fused_kernel<{prob.M}, {geo}, DM>"
    return f"pc_seq_kernel<{prob.M}, {geo}>"


# ------------------------------------------------------------------ arms
def run_reference(args):
    ws, rank, _ = dist_setup(args)
    if rank != 0:
        return 0
    if _WORKLOAD.startswith("mono"):
        from synth import make_problem

        scales, weights, k = WORKLOADS[_WORKLOAD][2]["mono"]
        return run_reference_mono(args, make_problem(WORKLOADS[_WORKLOAD][0]), scales, weights, k)
    if _WORKLOAD == "unet128":
        return run_reference_unet(args)
    prob, params = workload()
    n_pos = 100
    for _ in range(args.warmup):
        oracle_rate(prob, params, n_pos)
    times = []
    for _ in range(args.steps):
        _, dt = oracle_rate(prob, params, n_pos)
        times.append(dt)
    total = sum(times)
    units = n_pos * prob.K * args.steps
    value = units / total
    line = {"metric": METRIC, "value": value, "unit": METRIC, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": config_of(prob, {"sample": f"each step: one oracle iteration over the first {n_pos} "
                                                 f"of the {prob.N} positions"}),
            "cpu_baseline": {"value": value, "unit": METRIC, "cores": cpu_threads(), "kind": "oracle",
                             "sample": f"{args.steps} steps of one FP64 oracle iteration over {n_pos} positions x "
                                       f"{prob.K} modes (numpy/scipy, single-threaded)"},
            "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def mono_flops(M, J, k):
    """Algorithmic FLOPs of k CGLS steps on one pattern: C and C^T each hold 4 J M^2 non-zeros
    (a multiply and an add each), applied 2 k + 1 times, plus 10 M^2 per step for the vector updates
    and norms."""
    return (2 * k + 1) * 8.0 * J * M * M + 10.0 * k * M * M


def run_reference_unet(args):
    """The oracle's network forward (FP64 numpy) on one 128^2 pattern per step."""
    from oracle import unet

    params = unet.init_params(32, seed=1)
    x = np.random.default_rng(0).random((1, 128, 128, 1)) * 10
    for _ in range(args.warmup):
        unet.forward(params, x)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        unet.forward(params, x)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = args.steps / total
    line = {"metric": "warm-start estimate patterns/s", "value": value, "unit": "patterns/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": WORKLOADS[_WORKLOAD][1], "sample": "each step: the network forward on one pattern"},
            "cpu_baseline": {"value": value, "unit": "patterns/s", "cores": cpu_threads(), "kind": "oracle",
                             "sample": f"{args.steps} oracle network forwards of one 128^2 pattern (numpy, FP64)"},
            "e2e": {"value": value, "unit": "patterns/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_reference_mono(args, prob, scales, weights, k):
    from oracle import mono

    n_pat = 2
    B = prob.I[:n_pat].astype(np.float64)
    for _ in range(args.warmup):
        mono.monochromatise(B, scales, weights, k)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        mono.monochromatise(B, scales, weights, k)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = n_pat * args.steps / total
    unit = "patterns/s"
    line = {"metric": "monochromatised patterns/s", "value": value, "unit": unit, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": WORKLOADS[_WORKLOAD][1], "M": prob.M, "J": len(scales), "k": k,
                       "sample": f"each step: the oracle on {n_pat} of the {prob.N} patterns"},
            "cpu_baseline": {"value": value, "unit": unit, "cores": cpu_threads(), "kind": "oracle",
                             "sample": f"{args.steps} steps of the FP64 oracle CGLS on {n_pat} patterns (numpy)"},
            "e2e": {"value": value, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_ours_mono(args):
    """Monochromatisation: one step = one call over every pattern (one launch, one CTA each)."""
    ws, rank, local = dist_setup(args)
    import torch

    from paper_2406_06640_gb300.engine import monochromatise
    from synth import make_problem

    if not torch.cuda.is_available():
        raise SystemExit("bench.py: a CUDA device is required (no CPU fallback)")
    scales, weights, k = WORKLOADS[_WORKLOAD][2]["mono"]
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    prob = make_problem(WORKLOADS[_WORKLOAD][0])
    N, M, J = prob.N, prob.M, len(scales)
    stream = torch.cuda.current_stream(dev)
    b = torch.from_numpy(prob.I).to(dev)
    x = torch.empty_like(b)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    for _ in range(max(args.warmup, 3)):
        monochromatise(b, scales, weights, k, out=x, stream=stream)
    torch.cuda.synchronize(dev)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    sampler = ClockSampler(local) if rank == 0 else None
    if sampler:
        sampler.start()
    barrier(ws)
    torch.cuda.synchronize(dev)
    for i in range(args.steps):
        flush.zero_()
        ev[i][0].record(stream)
        monochromatise(b, scales, weights, k, out=x, stream=stream)
        ev[i][1].record(stream)
    torch.cuda.synchronize(dev)
    barrier(ws)
    clocks = sampler.stop() if sampler else None
    step_ms = [e0.elapsed_time(e1) for e0, e1 in ev]
    t_max = max_over_ranks(ws, sum(step_ms), dev)
    value = ws * N * args.steps / (t_max / 1e3)
    flops = N * mono_flops(M, J, k)
    avg_s = sum(step_ms) / len(step_ms) / 1e3
    achieved = flops / avg_s / 1e12
    peak = N_SMS * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12
    traffic = traffic_record(kernel_source_hash(("mono.cu",), "MonoArgs"), "mono_kernel_traffic.json",
                             _WORKLOAD)
    # end to end: the broadband patterns from pinned host memory, the monochromatic ones back
    b_h = torch.from_numpy(prob.I).pin_memory()
    x_h = torch.empty_like(b_h).pin_memory()
    e2e_steps = max(3, min(args.steps, 10))
    t_e2e = 0.0
    for i in range(e2e_steps + 1):
        flush.zero_()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        b.copy_(b_h, non_blocking=True)
        monochromatise(b, scales, weights, k, out=x, stream=stream)
        x_h.copy_(x, non_blocking=True)
        torch.cuda.synchronize(dev)
        if i > 0:
            t_e2e += time.perf_counter() - t0
    t_e2e = max_over_ranks(ws, t_e2e, dev)
    e2e_value = ws * N * e2e_steps / t_e2e
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        from oracle import mono

        # patterns one after another until about 10 s of CPU work (at least 2)
        n_pat, t0 = 0, time.perf_counter()
        while n_pat < N and (n_pat < 2 or time.perf_counter() - t0 < 10.0):
            mono.monochromatise(prob.I[n_pat:n_pat + 1].astype(np.float64), scales, weights, k)
            n_pat += 1
        dt = time.perf_counter() - t0
        cpu = {"value": n_pat / dt, "unit": "patterns/s", "cores": cpu_threads(), "kind": "oracle",
               "sample": f"the FP64 oracle CGLS on the first {n_pat} of the {N} patterns ({dt:.1f} s, numpy)"}
    if rank == 0:
        line = {"metric": "monochromatised patterns/s", "value": value, "unit": "patterns/s", "n_gpus": ws,
                "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": t_max / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic",
                "config": {"workload": WORKLOADS[_WORKLOAD][1], "N": N, "M": M, "J": J, "k": k,
                           "l2": "flushed before each timed step (256 MiB write)",
                           "parallelism": f"replicas{ws}" if ws > 1 else "single GPU"},
                "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                             "frac": achieved / peak, "traffic": traffic,
                             "kernel": "k_mono_cgls_band (M=256, clusters of 4)" if M == 256 else f"k_mono_cgls<{M}>",
                             "peak_basis": "152 SMs x 128 FP32 lanes x 2 FLOP x 2070 MHz (FMA pipe, max clock)",
                             "flops_per_launch": flops, "avg_launch_ms": avg_s * 1e3},
                "cpu_baseline": cpu,
                "e2e": {"value": e2e_value, "unit": "patterns/s", "h2d_bytes_per_step": b.numel() * 4,
                        "d2h_bytes_per_step": x.numel() * 4},
                "gpu_launches": args.steps, "clocks": clocks,
                "step_ms_min": min(step_ms), "step_ms_max": max(step_ms)}
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist

        dist.destroy_process_group()
    return 0


def run_ours_batch(args):
    """The batched workload: one step = one iteration of every problem (one graph launch)."""
    ws, rank, local = dist_setup(args)
    import torch

    from paper_2406_06640_gb300.engine import ReconstructionBatch
    from synth.generators import cfg3_members, make_cfg3_member

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    t_gen = time.perf_counter()
    descr = cfg3_members()
    problems, objs, prbs, host = [], [], [], []
    units, flops = 0, 0.0
    for i, (M, K, N, geo, sig) in enumerate(descr):
        p = make_cfg3_member(i)
        prm = dict(p.params, windows=[(1, 1 << 30)])
        I = torch.from_numpy(p.I).to(dev)
        problems.append((prm, I, p.positions))
        objs.append(torch.from_numpy(p.O0.astype(np.complex64)).to(dev))
        prbs.append(torch.from_numpy(p.P0.astype(np.complex64)).to(dev))
        host.append((p.O0.astype(np.complex64), p.P0.astype(np.complex64)))
        units += p.N * p.K
        flops += algorithmic_flops(p.M, p.K, p.N, geo == "near")
        del p
    t_gen = time.perf_counter() - t_gen
    stream = torch.cuda.current_stream(dev)
    batch = ReconstructionBatch(problems, stream)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    for _ in range(max(args.warmup, 3)):
        batch.iterate(objs, prbs, 1)
    torch.cuda.synchronize(dev)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    sampler = ClockSampler(local) if rank == 0 else None
    if sampler:
        sampler.start()
    barrier(ws)
    torch.cuda.synchronize(dev)
    for k in range(args.steps):
        flush.zero_()
        ev[k][0].record(stream)
        batch.iterate(objs, prbs, 1)
        ev[k][1].record(stream)
    torch.cuda.synchronize(dev)
    barrier(ws)
    clocks = sampler.stop() if sampler else None
    total_ms = sum(a.elapsed_time(b) for a, b in ev)
    t_max = max_over_ranks(ws, total_ms, dev)
    value = ws * units * args.steps / (t_max / 1e3)
    # end to end: every problem's state from pinned host memory and back, errors read back
    hO = [torch.from_numpy(o).pin_memory() for o, _ in host]
    hP = [torch.from_numpy(q).pin_memory() for _, q in host]
    e2e_steps = 3
    t_e2e = 0.0
    for k in range(e2e_steps + 1):
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for o, h in zip(objs, hO):
            o.copy_(h, non_blocking=True)
        for q, h in zip(prbs, hP):
            q.copy_(h, non_blocking=True)
        batch.iterate(objs, prbs, 1)
        for o, h in zip(objs, hO):
            h.copy_(o, non_blocking=True)
        for q, h in zip(prbs, hP):
            h.copy_(q, non_blocking=True)
        E = batch.errors()
        if k > 0:
            t_e2e += time.perf_counter() - t0
    t_e2e = max_over_ranks(ws, t_e2e, dev)
    state_bytes = sum(o.numel() * 8 for o in objs) + sum(q.numel() * 8 for q in prbs)
    per_step_s = t_max / args.steps / 1e3
    achieved = flops / per_step_s / 1e12
    peak = N_SMS * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12
    # the metric's second half: time to NRMSE <= 0.05, plain engine against warm start + batching
    ttn = None
    if rank == 0 and ws == 1 and _WORKLOAD == "far128x4" and not args.no_time_to_nrmse:
        try:
            ttn = warmstart_record(args, dev, local)
        except Exception as exc:  # the throughput line is still reported
            ttn = {"error": f"{type(exc).__name__}: {exc}"}
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": METRIC, "n_gpus": ws, "steps": args.steps,
                "warmup": max(args.warmup, 3), "ms_per_step": t_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": WORKLOADS["batch64"][1], "problems": len(descr), "pattern_modes": units,
                           "complex_constraint": "every step", "step": "one iteration of all 64 problems",
                           "l2": "flushed before each timed step (256 MiB write)",
                           "generation_s": round(t_gen, 1)},
                "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                             "frac": achieved / peak, "traffic": None, "kernel": "whole batch graph",
                             "flops_per_launch": flops},
                "cpu_baseline": None,
                "e2e": {"value": ws * units * e2e_steps / t_e2e, "unit": METRIC, "h2d_bytes_per_step": state_bytes,
                        "d2h_bytes_per_step": state_bytes + 8 * len(descr)},
                "gpu_launches": args.steps * batch.launches_per_iteration(), "clocks": clocks,
                "nrmse_mean_last": float(np.mean(E))}
        print(json.dumps(line), flush=True)
    batch.close()
    return 0


def conv_forward_flops(S, C):
    """Multiply-add FLOPs of one U-Net forward pass per pattern (stored channel counts)."""
    layers = [(S, 8, C), (S // 2, C, 2 * C), (S // 4, 2 * C, 4 * C), (S // 8, 4 * C, 8 * C),
              (S // 4, 12 * C, 4 * C), (S // 2, 6 * C, 2 * C), (S // 2, 2 * C, 16)]
    return sum(2.0 * h * h * 9 * ci * co for h, ci, co in layers)


WARM_BATCH_SEEDS = (4, 5, 6, 7)  # the batched comparison: four crystals of the variant
WARM_TARGET = 0.05


def _warm_problem(dev, seed, dose, peak):
    import torch

    from synth import make_problem

    pb = make_problem(4, seed=seed, dose=dose, peak=peak)
    prm = dict(pb.params)
    prm.pop("n_iter", None)
    M = prm["M"]
    return dict(pb=pb, prm=prm, M=M, s_true=pb.sim_sigma, I=torch.from_numpy(pb.I).to(dev),
                Ic=torch.from_numpy(pb.I_clean.astype(np.float32)).to(dev), pos=pb.positions.astype(np.int32),
                P0=torch.from_numpy(pb.P0.reshape(1, M, M)).to(dev))


def _engine(prm, sig):
    from paper_2406_06640_gb300.warmstart import eval_kernel_size

    return dict(prm, blur_domain="intensity", sigma1=sig, sigma2=sig, kernel_size=eval_kernel_size(sig))


def warmstart_record(args, dev, local, with_clocks=True):
    """Time to intensity NRMSE <= 0.05 against the noise-free patterns: the plain FP32 engine from a
    flat start (given the true sigma) against the learned warm start (U-Net over 64 sampled patterns,
    stitched object, median sigma), for one reconstruction and for four run as one batch plan; and the
    stated electron workload, where the comparison is degenerate, with the fallback target."""
    import torch

    from paper_2406_06640_gb300.warmstart import (LatticeSpec, WarmStart, WarmStartConfig, subsample_scan,
                                                  time_to_nrmse, time_to_nrmse_batch)

    n_train, spacing = 200_000, 16.0
    rec = {"target": WARM_TARGET, "train_patterns": n_train, "sampled_patterns_per_reconstruction": None}
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def estimate_timed(net, w, idx):
        Isub = w["I"][torch.from_numpy(idx).to(dev)].contiguous()
        torch.cuda.synchronize(dev)
        e0.record()
        Ow, sig = net.estimate(Isub, w["pos"][idx], w["prm"]["obj_h"], w["prm"]["obj_w"])
        e1.record()
        e1.synchronize()
        return Ow, sig, e0.elapsed_time(e1)

    # ---- variant: 1.0 rad peaks, 2e4 counts per pattern
    probs = [_warm_problem(dev, sd, 2e4, 1.0) for sd in WARM_BATCH_SEEDS]
    w0 = probs[0]
    net = WarmStart(w0["P0"][0], WarmStartConfig(S=w0["M"], C=32, batch=64, dose=2e4, target_scale=1.0,
                                                  lattice=LatticeSpec(peak=1.0), seed=1))
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    net.train(n_train)
    torch.cuda.synchronize(dev)
    t_train = time.perf_counter() - t0
    idxs = [subsample_scan(w["pos"], spacing) for w in probs]
    rec["sampled_patterns_per_reconstruction"] = len(idxs[0])
    for _ in range(max(args.warmup, 3)):
        estimate_timed(net, w0, idxs[0])
    sampler = ClockSampler(local) if with_clocks else None
    if sampler:
        sampler.start()
    plain, warm, est_ms = [], [], []
    for _ in range(max(args.steps // 4, 3)):
        O = torch.ones(w0["prm"]["obj_h"], w0["prm"]["obj_w"], dtype=torch.complex64, device=dev)
        plain.append(time_to_nrmse(_engine(w0["prm"], w0["s_true"]), w0["I"], w0["Ic"], w0["pos"], O, w0["P0"].clone(),
                                   w0["s_true"], WARM_TARGET))
        Ow, sig, ms = estimate_timed(net, w0, idxs[0])
        est_ms.append(ms)
        warm.append(time_to_nrmse(_engine(w0["prm"], sig), w0["I"], w0["Ic"], w0["pos"], Ow.clone(), w0["P0"].clone(),
                                  w0["s_true"], WARM_TARGET))
    # batched: the four reconstructions run plain one after another, against warm starts + one batch plan
    plain_b, warm_b = [], []
    for w in probs:
        O = torch.ones(w["prm"]["obj_h"], w["prm"]["obj_w"], dtype=torch.complex64, device=dev)
        plain_b.append(time_to_nrmse(_engine(w["prm"], w["s_true"]), w["I"], w["Ic"], w["pos"], O, w["P0"].clone(),
                                     w["s_true"], WARM_TARGET))
    members, est_b = [], []
    for w, idx in zip(probs, idxs):
        Ow, sig, ms = estimate_timed(net, w, idx)
        est_b.append(ms)
        members.append(dict(params=_engine(w["prm"], sig), intensities=w["I"], clean=w["Ic"], positions=w["pos"],
                            obj=Ow.clone(), probe=w["P0"].clone(), sigma_eval=w["s_true"]))
    rb = time_to_nrmse_batch(members, WARM_TARGET)
    clocks = sampler.stop() if sampler else None
    # end to end through the public calls: the sampled patterns from pinned host memory, object back
    hI = w0["I"][torch.from_numpy(idxs[0]).to(dev)].cpu().pin_memory()
    hO = torch.empty(w0["prm"]["obj_h"], w0["prm"]["obj_w"], dtype=torch.complex64).pin_memory()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    dI = hI.to(dev, non_blocking=True)
    Ow, _ = net.estimate(dI, w0["pos"][idxs[0]], w0["prm"]["obj_h"], w0["prm"]["obj_w"])
    hO.copy_(Ow, non_blocking=True)
    torch.cuda.synchronize(dev)
    e2e_ms = 1e3 * (time.perf_counter() - t0)
    net.close()
    plain_ms = float(np.median([r["engine_ms"] for r in plain]))
    warm_eng = float(np.median([r["engine_ms"] for r in warm]))
    est = float(np.median(est_ms))
    warm_ms = est + warm_eng
    fwd_flops = conv_forward_flops(w0["M"], 32) * len(idxs[0])
    try:
        peak = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["bf16_tflops"]
        peak_src = "measured bf16 burst (MEASURED_PEAKS.json)"
    except (OSError, KeyError, ValueError):
        peak, peak_src = 1900.0, "fallback bf16 burst"
    achieved = fwd_flops / (est / 1e3) / 1e12
    plain_b_ms = float(sum(r["engine_ms"] for r in plain_b))
    warm_b_ms = float(sum(est_b)) + rb["engine_ms"]
    rec["variant"] = {
        "workload": "electron-like crystal with 1.0 rad peaks at 2e4 counts per pattern (probe 128^2, 64x64 raster "
                    "step 2 px, object 256^2, sigma 2), engine with the intensity-blur model of Eq. 2",
        "plain_ms": plain_ms, "warm_ms": warm_ms, "warm_estimate_ms": est, "warm_engine_ms": warm_eng,
        "gain": plain_ms / warm_ms,
        "plain_iterations": [r["iterations"] for r in plain], "warm_iterations": [r["iterations"] for r in warm],
        "reached": all(r["reached"] for r in plain + warm),
        "nrmse_flat_start": plain[0]["curve"][0][1], "nrmse_warm_start": warm[0]["curve"][0][1],
        "plain_curve": [round(c[1], 4) for c in plain[0]["curve"]],
        "warm_curve": [round(c[1], 4) for c in warm[0]["curve"]],
        "sigma_true": w0["s_true"], "train_s": t_train, "train_patterns_per_s": n_train / t_train,
        "batched": {"reconstructions": len(probs), "plain_sequential_ms": plain_b_ms,
                    "warm_estimates_ms": float(sum(est_b)), "warm_batch_engine_ms": rb["engine_ms"],
                    "warm_batched_ms": warm_b_ms, "gain": plain_b_ms / warm_b_ms,
                    "plain_iterations": [r["iterations"] for r in plain_b], "batch_iterations": rb["iterations"],
                    "reached": all(r["reached"] for r in plain_b) and rb["reached"]},
        "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": None, "peak_basis": peak_src,
                     "kernel": f"U-Net forward over {len(idxs[0])} patterns (warm-start estimate, all launches)",
                     "flops_per_launch": fwd_flops},
        "e2e": {"value": e2e_ms + warm_eng, "unit": "ms", "h2d_bytes_per_step": hI.numel() * 4,
                "d2h_bytes_per_step": hO.numel() * 8},
        "clocks": clocks}

    # ---- the stated electron workload (0.1 rad peaks, 200 counts): the flat start already lies below 0.05 and
    # the plain engine moves away from it, so the target is 0.05 above the plain engine's plateau
    w4 = _warm_problem(dev, 4, 200.0, 0.1)
    O = torch.ones(w4["prm"]["obj_h"], w4["prm"]["obj_w"], dtype=torch.complex64, device=dev)
    run = time_to_nrmse(_engine(w4["prm"], w4["s_true"]), w4["I"], w4["Ic"], w4["pos"], O, w4["P0"].clone(),
                        w4["s_true"], -1.0, max_iter=20)
    curve = [c[1] for c in run["curve"]]
    plateau = float(np.mean(curve[-2:]))  # the iterates alternate; the mean of the last two
    fallback = plateau + WARM_TARGET
    net4 = WarmStart(w4["P0"][0], WarmStartConfig(S=w4["M"], C=32, batch=64, dose=200.0, target_scale=0.1,
                                                   lattice=LatticeSpec(peak=0.1), seed=1))
    net4.train(n_train)
    idx4 = subsample_scan(w4["pos"], spacing)
    for _ in range(2):
        estimate_timed(net4, w4, idx4)
    Ow4, sig4, est4 = estimate_timed(net4, w4, idx4)
    net4.close()
    warm4 = time_to_nrmse(_engine(w4["prm"], sig4), w4["I"], w4["Ic"], w4["pos"], Ow4.clone(), w4["P0"].clone(),
                          w4["s_true"], -1.0, max_iter=2)
    first = lambda cv, t: next((i for i, v in enumerate(cv) if v <= t), None)  # noqa: E731
    it_plain = first(curve, fallback)
    it_warm = first([c[1] for c in warm4["curve"]], fallback)
    per_it = run["engine_ms"] / max(run["iterations"], 1)
    rec["configuration4_as_stated"] = {
        "workload": "electron-like crystal, 0.1 rad peaks, 200 counts per pattern (as stated)",
        "nrmse_flat_start": curve[0], "plain_curve": [round(v, 4) for v in curve], "plain_plateau": plateau,
        "target": "0.05 above the plain plateau (0.05 lies below the flat start's value, which the engine only "
                  "moves away from)", "target_value": fallback,
        "plain_iterations": it_plain, "plain_ms": None if it_plain is None else it_plain * per_it,
        "nrmse_warm_start": warm4["curve"][0][1], "warm_iterations": it_warm,
        "warm_ms": None if it_warm is None else est4 + it_warm * per_it,
        "sigma_est": sig4, "sigma_true": w4["s_true"]}
    return rec


def run_ours_unet(args):
    """The warm-start network's inference alone: estimates per second over 64 patterns of 128^2."""
    ws, rank, local = dist_setup(args)
    import torch

    from paper_2406_06640_gb300.warmstart import LatticeSpec, WarmStart, WarmStartConfig

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    M, n, C = 128, 64, 32
    P0 = torch.ones(M, M, dtype=torch.complex64, device=dev)
    net = WarmStart(P0, WarmStartConfig(S=M, C=C, batch=n, dose=2e4, target_scale=1.0, lattice=LatticeSpec(peak=1.0),
                                        seed=1))
    gen = torch.Generator().manual_seed(0)
    hI = (torch.rand(n, M, M, generator=gen) * 10).pin_memory()
    I = hI.to(dev)
    pos = np.stack(np.meshgrid(np.arange(8) * 16, np.arange(8) * 16, indexing="ij"), -1).reshape(-1, 2).astype(np.int32)
    obj = 7 * 16 + M
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    for _ in range(max(args.warmup, 3)):
        net.estimate(I, pos, obj, obj)
    torch.cuda.synchronize(dev)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    sampler = ClockSampler(local) if rank == 0 else None
    if sampler:
        sampler.start()
    barrier(ws)
    for k in range(args.steps):
        flush.zero_()
        ev[k][0].record()
        net.estimate(I, pos, obj, obj)
        ev[k][1].record()
    torch.cuda.synchronize(dev)
    barrier(ws)
    clocks = sampler.stop() if sampler else None
    step_ms = [a.elapsed_time(b) for a, b in ev]
    t_max = max_over_ranks(ws, sum(step_ms), dev)
    value = ws * n * args.steps / (t_max / 1e3)
    # end to end: the patterns from pinned host memory, the stitched object back every step
    hO = torch.empty(obj, obj, dtype=torch.complex64).pin_memory()
    t_e2e = 0.0
    for k in range(args.steps + 1):
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        Ow, _ = net.estimate(hI.to(dev, non_blocking=True), pos, obj, obj)
        hO.copy_(Ow, non_blocking=True)
        torch.cuda.synchronize(dev)
        if k > 0:
            t_e2e += time.perf_counter() - t0
    t_e2e = max_over_ranks(ws, t_e2e, dev)
    net.close()
    flops = conv_forward_flops(M, C) * n
    try:
        peak = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["bf16_tflops"]
        peak_src = "measured bf16 burst (MEASURED_PEAKS.json)"
    except (OSError, KeyError, ValueError):
        peak, peak_src = 1900.0, "fallback bf16 burst"
    avg_s = t_max / args.steps / 1e3
    if rank == 0:
        line = {"metric": "warm-start estimate patterns/s", "value": value, "unit": "patterns/s", "n_gpus": ws,
                "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": t_max / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16",
                "data": "synthetic",
                "config": {"workload": WORKLOADS[_WORKLOAD][1], "patterns": n, "S": M, "C": C,
                           "l2": "flushed before each timed step (256 MiB write)"},
                "roofline": {"bound": "tensor", "achieved": flops / avg_s / 1e12, "peak": peak, "unit": "TFLOP/s",
                             "frac": flops / avg_s / 1e12 / peak, "traffic": None, "peak_basis": peak_src,
                             "kernel": "the seven convolutions' FLOPs over the whole estimate (all launches)",
                             "flops_per_launch": flops},
                "cpu_baseline": None,
                "e2e": {"value": n * args.steps / t_e2e, "unit": "patterns/s", "h2d_bytes_per_step": hI.numel() * 4,
                        "d2h_bytes_per_step": hO.numel() * 8},
                "gpu_launches": None, "clocks": clocks}
        print(json.dumps(line), flush=True)
    return 0


def run_ours_warmstart(args):
    """Learned warm start vs flat start: time to NRMSE <= 0.05 (one GPU; replicas only for N > 1)."""
    ws, rank, local = dist_setup(args)
    import torch

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    rec = warmstart_record(args, dev, local, with_clocks=rank == 0)
    if rank == 0:
        v = rec["variant"]
        line = {"metric": "time to NRMSE <= 0.05 (warm start)", "value": v["warm_ms"], "unit": "ms",
                "n_gpus": ws, "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": v["warm_ms"],
                "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "bf16+f32",
                "data": "synthetic",
                "config": {"workload": WORKLOADS["warmstart"][1], "train_patterns": rec["train_patterns"],
                           "sampled_patterns": rec["sampled_patterns_per_reconstruction"], "target": WARM_TARGET,
                           "l2": "inputs resident; each measurement starts from a fresh object"},
                "roofline": v["roofline"], "cpu_baseline": None, "e2e": v["e2e"], "gpu_launches": None,
                "clocks": v["clocks"], "time_to_nrmse": rec}
        print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    if _WORKLOAD == "batch64":
        return run_ours_batch(args)
    if _WORKLOAD.startswith("mono"):
        return run_ours_mono(args)
    if _WORKLOAD == "warmstart":
        return run_ours_warmstart(args)
    if _WORKLOAD == "unet128":
        return run_ours_unet(args)
    ws, rank, local = dist_setup(args)
    import torch

    from paper_2406_06640_gb300.engine import Reconstruction

    if not torch.cuda.is_available():
        raise SystemExit("bench.py: a CUDA device is required (no CPU fallback)")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    prob, params = workload()
    stream = torch.cuda.current_stream(dev)
    I = torch.from_numpy(prob.I).to(dev)
    O = torch.from_numpy(prob.O0.astype(np.complex64)).to(dev)
    P = torch.from_numpy(prob.P0.astype(np.complex64)).to(dev)
    rec = Reconstruction(params, I, prob.positions, stream)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    units_per_step = prob.N * prob.K

    for _ in range(max(args.warmup, 3)):
        rec.iterate(O, P, 1)
    torch.cuda.synchronize(dev)
    rec.profile(True)
    rec.profile_read()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    sampler = ClockSampler(local) if rank == 0 else None
    if sampler:
        sampler.start()
    barrier(ws)
    torch.cuda.synchronize(dev)
    for k in range(args.steps):
        flush.zero_()
        ev[k][0].record(stream)
        rec.iterate(O, P, 1)
        ev[k][1].record(stream)
    torch.cuda.synchronize(dev)
    barrier(ws)
    clocks = sampler.stop() if sampler else None
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = sum(step_ms)
    fused_ms, fused_launches = rec.profile_read()
    rec.profile(False)
    E_last = rec.error()
    t_max = max_over_ranks(ws, total_ms, dev)
    value = ws * units_per_step * args.steps / (t_max / 1e3)

    # roofline of the dominant (fused) kernel: algorithmic FLOPs per launch / its event-timed duration
    flops = algorithmic_flops(prob.M, prob.K, prob.N, params["geometry"] == "near", params.get("engine") == "dm")
    fused_avg_s = fused_ms / max(fused_launches, 1) / 1e3
    achieved = flops / fused_avg_s / 1e12
    peak = N_SMS * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12
    traffic = traffic_record(kernel_source_hash()) if _WORKLOAD == "far128x4" else None
    # the FP32 FMA rate measured on this device, beside the nominal peak (units x maximum clock)
    from paper_2406_06640_gb300.binding import measure_fp32_peak

    peak_meas, peak_meas_ms = measure_fp32_peak(stream.cuda_stream)

    # end to end through the public API: object + probe state from pinned host memory, one
    # iteration, error metric and state back to pinned host memory, every step
    O_h = torch.from_numpy(prob.O0.astype(np.complex64)).pin_memory()
    P_h = torch.from_numpy(prob.P0.astype(np.complex64)).pin_memory()
    e2e_steps = max(3, min(args.steps, 10))
    torch.cuda.synchronize(dev)
    t_e2e = 0.0
    for k in range(e2e_steps + 1):
        flush.zero_()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        O.copy_(O_h, non_blocking=True)
        P.copy_(P_h, non_blocking=True)
        rec.iterate(O, P, 1)
        O_h.copy_(O, non_blocking=True)
        P_h.copy_(P, non_blocking=True)
        rec.error()  # synchronises the stream; reads E back to the host
        if k > 0:  # first round trip is a warm-up
            t_e2e += time.perf_counter() - t0
    t_e2e = max_over_ranks(ws, t_e2e, dev)
    e2e_value = ws * units_per_step * e2e_steps / t_e2e
    state_bytes = O.numel() * 8 + P.numel() * 8

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        rate, dt = oracle_rate(prob, params, prob.N)
        single = {"value": rate, "unit": METRIC, "cores": cpu_threads(), "kind": "oracle",
                  "sample": f"one FP64 oracle iteration of the full workload ({prob.N} positions x {prob.K} modes, "
                            f"{dt:.1f} s, numpy/scipy single-threaded)"}
        workers = os.cpu_count() or 1
        n_pos = prob.N // 4
        try:
            rate_all, wall = oracle_rate_all_cores(WORKLOADS[_WORKLOAD][0], params, n_pos, workers)
            cpu = {"value": rate_all, "unit": METRIC, "cores": workers * cpu_threads(), "kind": "oracle",
                   "sample": f"{workers} worker processes, each one FP64 oracle iteration over {n_pos} of the "
                             f"{prob.N} positions x {prob.K} modes (independent replicas, {wall:.1f} s wall, "
                             f"numpy/scipy single-threaded per worker)",
                   "single_core": single}
        except Exception as exc:  # the single-core figure stands alone
            cpu = dict(single, all_cores_error=f"{type(exc).__name__}: {exc}")
    # the metric's second half: time to NRMSE <= 0.05, plain engine against warm start + batching
    ttn = None
    if rank == 0 and ws == 1 and _WORKLOAD == "far128x4" and not args.no_time_to_nrmse:
        try:
            ttn = warmstart_record(args, dev, local)
        except Exception as exc:  # the throughput line is still reported
            ttn = {"error": f"{type(exc).__name__}: {exc}"}
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": METRIC, "n_gpus": ws, "steps": args.steps,
                "warmup": max(args.warmup, 3), "ms_per_step": t_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": config_of(prob, {"parallelism": f"replicas{ws}" if ws > 1 else "single GPU",
                                           "engine": params.get("engine", "pie"),
                                           "step_rule": params.get("step_rule", "normalised"),
                                           "minibatch": params.get("minibatch", 0) or prob.N}),
                "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                             "frac": achieved / peak, "traffic": traffic,
                             "kernel": kernel_label(prob, params),
                             "peak_basis": "152 SMs x 128 FP32 lanes x 2 FLOP x 2070 MHz (FMA pipe, max clock)",
                             "peak_measured": peak_meas, "frac_of_measured": achieved / peak_meas,
                             "peak_measured_basis": f"FFMA loop on this device, CUDA events, {peak_meas_ms:.3f} ms",
                             "flops_per_launch": flops, "avg_launch_ms": fused_avg_s * 1e3},
                "cpu_baseline": cpu,
                "e2e": {"value": e2e_value, "unit": METRIC, "h2d_bytes_per_step": state_bytes,
                        "d2h_bytes_per_step": state_bytes + 8},
                "gpu_launches": args.steps * rec.launches_per_iteration(True),
                "clocks": clocks, "nrmse_last": E_last, "step_ms_min": min(step_ms), "step_ms_max": max(step_ms)}
        if ttn is not None:
            line["time_to_nrmse"] = ttn
        print(json.dumps(line), flush=True)
    rec.close()
    if ws > 1:
        import torch.distributed as dist

        dist.destroy_process_group()
    return 0


def main():
    global _WORKLOAD
    args = parse()
    _WORKLOAD = args.workload
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
