#!/usr/bin/env python
"""Benchmark: one optimisation step of the analytic-PSF Gaussian slice model.

A step = forward (Gaussian and slice preprocessing, Mahalanobis cut, (tile,
record) keys, radix sort, tile evaluation with the fused MSE loss), backward
(tile adjoint, gradient epilogue) and the fused Adam update.

Headline workload (default, --workload large): the 1M-Gaussian large case --
1,000,372 Gaussians, six stacks of 48 x 256 x 256 px at 0.8 x 0.8 x 3.0 mm,
motion U(+-10 deg)/U(+-5 mm), every masked pixel (7.09M) in every step; the
step is the sequence of library calls the torch.autograd.Function front end
(autograd.SliceLoss) makes.  The fetal case (200k Gaussians, 3 x 40 x 192^2 px,
2^18 pixels drawn by the device sampler each step) is measured after it and
reported under the "fetal" key.

Prints one JSON line.  `value` counts (pixel, Gaussian) pairs inside the
1e-7 cut (the pairs the method needs) per second of whole-step device time;
`px_per_s` counts slice pixels.  `e2e` is the same metric through the
host-buffer C-ABI call (gsvr_step_host: parameters and pixel list uploaded
from pinned memory, gradient and loss read back every step).  `roofline`
holds, for the dominant tile kernel, the in-cut pairs per launch, the average
launch time (CUDA events), the FP32 operations per pair the method needs (17
for the backward, 7 for the forward) and the FFMA lane-operation rate measured
on the same GPU, so that frac = pairs / time x FP32 per pair / FFMA rate can
be recomputed from the line.  The timed region launches each step's kernels
eagerly (with stage events); `graph` times the same step replayed as one CUDA
graph per iteration (gsvr_graph_capture / gsvr_graph_launch).

--impl reference times the FP64 brute-force CPU oracle on bounded pixel
samples of the same workload (the oracle is this project's reference program).
Multi-GPU (torchrun): every rank reconstructs its own subject (weak scaling,
no data-path collective); rank 0 prints the aggregate.
"""
import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fwd+bwd Gaussian-pixel pairs/s & slice px/s; sec to fixed PSNR vs plain, 1 B300"
UNIT = "pairs/s"
# Algorithmic FP32 work per (pixel, Gaussian) pair inside the cut, as the
# method states it (the 3D form reduced to the slice plane): forward q, exp and
# the weighted sum (7 FP32 + 1 MUFU); backward the same plus the six moment
# contributions of g, g db, g da, g db^2, g db da, g da^2 (17 FP32 + 1 MUFU).
# The roofline pair rate of a kernel is the measured FFMA lane-operation rate
# divided by its count.
FP32_PER_PAIR = {"fwd_eval": 7.0, "bwd_eval": 17.0}
KERNEL_OF = {"fwd_eval": "k_fwd_items", "bwd_eval": "k_bwd_items"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="large", choices=["large", "fetal", "tiny"])
    ap.add_argument("--no-fetal", action="store_true", help="skip the secondary fetal measurement")
    ap.add_argument("--stacks", type=int, default=0, help="keep only the first n stacks (profiling captures)")
    ap.add_argument("--tile", default="16x16",
                    help="HxW or HxWpxP tile (no tuning; P forward pixels per thread) or 'auto': the library's "
                         "autotuner picks the launch shape")
    ap.add_argument("--fetal-tile", default="auto",
                    help="launch shape of the fetal leg of the default run (as --tile; the autotuner by default)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    return ap.parse_args()


def workload(name, seed, n_stacks=0):
    from paper_2512_11624_b300 import inputs
    if name == "large":
        case = inputs.large(seed)
        desc = ("large: %d Gaussians (1.08 mm grid in a brain phantom scaled 2.307x), 6 stacks of 48 x 256 x 256 "
                "px at 0.8 x 0.8 x 3.0 mm (axial, coronal, sagittal, axial turned 45 deg about x, y, z), motion "
                "U(+-10 deg)/U(+-5 mm), every masked pixel (%d) per step, Adam" % (case["N"], int(case["mask"].sum())))
    elif name == "fetal":
        case = inputs.fetal(seed)
        desc = ("fetal: %d Gaussians (0.8 mm grid in a brain phantom), 3 orthogonal stacks of 40 x 192 x 192 px "
                "at 1 x 1 x 3.5 mm, motion U(+-5 deg)/U(+-3 mm), 2^18 sampled px/step, Adam" % case["N"])
    else:
        case = inputs.tiny(seed)
        desc = "tiny: 2000 Gaussians, 1 stack of 8 x 32 x 32 px, all pixels, Adam"
    if n_stacks:
        case = inputs.first_stacks(case, n_stacks)
    return case, desc


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 200 ms."""
    FIELDS = "clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown," \
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown," \
             "clocks_event_reasons.sw_power_cap"

    def __init__(self, gpu_id=None):
        self.rows = []
        self.proc = None
        cmd = ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits", "-lms", "200"]
        if gpu_id is not None:
            cmd += ["-i", str(gpu_id)]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == 7:
                self.rows.append(parts)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows for k in range(4) if r[3 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def parse_tile(spec):
    """'HxW' or 'HxWpxP' -> (tile_h, tile_w, forward pixels per thread, 0 = by width)."""
    m = re.fullmatch(r"(\d+)x(\d+)(?:px(\d+))?", spec)
    if not m:
        raise SystemExit("--tile: HxW, HxWpxP or auto, not %r" % spec)
    return int(m.group(1)), int(m.group(2)), int(m.group(3) or 0)


def kernel_source_sha(kernel):
    """Hash of the source text of one __global__ function (its definition up to the
    matching closing brace) in csrc/gsvr_kernels.cu."""
    src = open(os.path.join(ROOT, "paper_2512_11624_b300", "csrc", "gsvr_kernels.cu")).read()
    at = src.find(" " + kernel + "(")
    while at >= 0 and "__global__" not in src[max(0, src.rfind("\n", 0, at) - 200):at]:
        at = src.find(" " + kernel + "(", at + 1)
    if at < 0:
        return "missing"
    start = src.find("{", at)
    depth, k = 0, start
    while k < len(src):
        depth += {"{": 1, "}": -1}.get(src[k], 0)
        if depth == 0:
            break
        k += 1
    return hashlib.sha1(src[at:k + 1].encode()).hexdigest()[:12]


def profiled_traffic(kernel, workload_name):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, if it was
    taken on the current source of that kernel (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(path):
        return None
    sha = kernel_source_sha(kernel)
    for line in open(path):
        p = line.split()
        if len(p) >= 4 and not line.startswith("#") and p[0] == kernel and p[1] == workload_name and p[2] == sha:
            return float(p[3])
    return None


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        backend = "nccl" if __import__("torch").cuda.is_available() else "gloo"
        dist.init_process_group(backend)
    return ws, rank, local


def reduce_max(x, ws):
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def reduce_sum(x, ws):
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def cpu_oracle_sample(case, pix, n_sample_total):
    """FP64 oracle fwd+bwd (every Gaussian, gradients of all parameters) on the
    listed pixels; returns (seconds, useful pairs in them, threads)."""
    from oracle import oracle
    th = case["theta"].astype(np.float64)
    t0 = time.perf_counter()
    oracle.forward_backward(case["stacks"], th, case["N"], pix, case["I"].astype(np.float64)[pix],
                            1.0 / n_sample_total, want_abs=False)
    dt = time.perf_counter() - t0
    useful = oracle.count_pairs(case["stacks"], th, case["N"], pix)
    return dt, useful, oracle.num_threads()


def run_reference(args, ws, rank):
    if rank != 0:
        return
    case, desc = workload(args.workload, 0)
    from oracle import oracle
    rng = np.random.default_rng(0)
    masked = np.nonzero(case["mask"])[0]
    n_s = min(case["n_sample"], masked.size)
    # per-step pixel count so that warmup + steps fit in ~150 s
    probe = rng.choice(masked, 8, replace=False)
    t_probe, _, _ = cpu_oracle_sample(case, probe, n_s)
    per_px = max(t_probe / 8, 1e-6)
    budget = 150.0 / max(args.steps + args.warmup, 1)
    n_px = int(max(2, min(4096, budget / per_px)))
    times, useful = [], 0
    for k in range(args.warmup + args.steps):
        pix = rng.choice(masked, n_px, replace=False)
        dt, u, cores = cpu_oracle_sample(case, pix, n_s)
        if k >= args.warmup:
            times.append(dt)
            useful += u
    tot = sum(times)
    value = useful / tot
    px_s = n_px * args.steps / tot
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": desc, "parallelism": "replicas" if ws > 1 else "single"},
            "px_per_s": px_s,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "%d random masked pixels per step x every Gaussian, fwd+bwd, float64" % n_px},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def measure(args, gsvr, torch, dev, stream, name, rank, ws, steps, warmup, with_e2e, with_cpu, clocks_on, tile):
    """Times `steps` optimisation steps of one workload; returns its JSON fields."""
    case, desc = workload(name, rank, args.stacks)
    sampled = name == "fetal"  # the fetal case draws 2^18 pixels per step; the others use every masked pixel
    n_mask = int(case["mask"].sum())
    n_s = min(case["n_sample"], n_mask) if sampled else n_mask

    def set_sample(c, k):
        if sampled:
            gsvr.gsvr_sample_pixels(c.ctx, n_s, k)

    def probe_counts(shape):
        probe = gsvr.Context(case, device=dev, stream=stream.cuda_stream)
        gsvr.gsvr_set_tiling(probe.ctx, shape)
        if sampled:
            gsvr.gsvr_sample_pixels(probe.ctx, n_s, 0)
        else:
            gsvr.gsvr_set_pixel_sample(probe.ctx, None)
        probe.forward()
        st = probe.stats()
        probe.close()
        return st

    # launch shape: fixed, or the autotuner's pick (timed fwd+bwd iterations of
    # every candidate on a fixed-capacity context, before and outside the timed region)
    tuning = None
    if tile == "auto":
        st0 = probe_counts(gsvr.tiling(12, 12))
        tune = gsvr.Context(case, device=dev, stream=stream.cuda_stream, tile_h=12, tile_w=12, fixed_capacity=1,
                            cap_records=int(st0["n_records"] * 1.5) + 4096, cap_keys=int(st0["n_keys"] * 4) + 4096)
        if not sampled:
            gsvr.gsvr_set_pixel_sample(tune.ctx, None)
        best, res = gsvr.gsvr_autotune(tune.ctx, None, n_per_subject=n_s if sampled else 0,
                                       iterations=10 if sampled else 3)
        tune.close()
        shape = res[best]
        tuning = {"candidates": len(res), "ms_per_iter_best": round(res[best].ms, 4),
                  "timed": ["%dx%d px%d fwd%d bwd%d order%d: %.4f ms" % (r.tile_h, r.tile_w, r.fwd_px_per_thread,
                                                                          r.fwd_blocks_per_sm, r.bwd_blocks_per_sm,
                                                                          r.queue_order, r.ms) for r in res]}
    else:
        shape = gsvr.tiling(*parse_tile(tile))
    shape_d = {k: v for k, v in shape.as_dict().items() if k != "ms"}
    # capacities from one probe forward, then a fixed-capacity context (no host sync per step)
    st0 = probe_counts(shape)
    ctx = gsvr.Context(case, device=dev, stream=stream.cuda_stream, tile_h=shape.tile_h, tile_w=shape.tile_w,
                       fixed_capacity=1, cap_records=int(st0["n_records"] * 1.3) + 4096,
                       cap_keys=int(st0["n_keys"] * 1.3) + 4096, timing=1, seed=1234 + rank)
    gsvr.gsvr_set_tiling(ctx.ctx, shape)
    if not sampled:
        gsvr.gsvr_set_pixel_sample(ctx.ctx, None)
    M = ctx.M
    ref_slice = case.get("ref_slice", M // 6)
    gsvr.gsvr_set_frozen(ctx.ctx, np.array([1 if i == ref_slice else 0 for i in range(M)], np.uint8))

    def step(k):
        set_sample(ctx, k)
        gsvr.gsvr_forward(ctx.ctx)
        gsvr.gsvr_backward(ctx.ctx)
        gsvr.gsvr_adam_step(ctx.ctx, k + 1)

    # pairs inside the cut per step: counted exactly (count pass over the sampled
    # pixels) outside the timed region, on the parameters before and after the
    # timed steps (the optimisation moves the Gaussians, so the count drifts over
    # a long run; a step's pairs are taken as the mean of the two ends)
    n_count = 3 if sampled else 1

    def count_pairs(k0):
        u_sum = t_sum = 0
        for k in range(n_count):
            set_sample(ctx, k0 + k)
            gsvr.gsvr_forward(ctx.ctx)
            u, e = gsvr.gsvr_count_pairs(ctx.ctx)
            u_sum += u
            t_sum += e
        return u_sum / n_count, t_sum / n_count

    for k in range(warmup):
        step(k)
    useful_start, tile_start = count_pairs(warmup)
    gsvr.gsvr_sync_status(ctx.ctx)
    gsvr.gsvr_timing_reset(ctx.ctx)
    clocks = None
    if clocks_on:
        uuid = None
        try:
            uuid = str(torch.cuda.get_device_properties(dev).uuid)
            uuid = uuid if uuid.startswith("GPU-") else "GPU-" + uuid
        except Exception:
            uuid = None
        clocks = ClockSampler(uuid)
        time.sleep(0.3)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for k in range(steps):
        step(warmup + k)
    e1.record(stream)
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    clk = clocks.stop() if clocks else None
    ms = e0.elapsed_time(e1)
    gsvr.gsvr_sync_status(ctx.ctx)
    kt = gsvr.gsvr_get_kernel_times(ctx.ctx)
    ms_max = reduce_max(ms, ws)

    useful_end, tile_end = count_pairs(warmup + steps)
    useful_per_step = 0.5 * (useful_start + useful_end)
    tile_pairs_per_step = 0.5 * (tile_start + tile_end)
    useful_total = reduce_sum(useful_per_step * steps, ws)
    px_total = reduce_sum(float(n_s) * steps, ws)
    value = useful_total / (ms_max / 1e3)

    # roofline of both tile kernels: in-cut pairs per launch over the kernel's
    # average launch time, against the measured FFMA lane-operation rate / the
    # method's FP32 operations per pair
    ffma_s, ex2_s, n_sm = gsvr.gsvr_alu_peaks(dev)
    ffma2_s = gsvr.gsvr_ffma2_peak(dev)
    kernels = {}
    bwd_eval_per_step = kt["bwd_pairs_evaluated"] / max(kt["calls"]["bwd_eval"], 1)
    evaluated = {"fwd_eval": tile_pairs_per_step, "bwd_eval": bwd_eval_per_step}
    for stg in ("fwd_eval", "bwd_eval"):
        avg_ms = kt["ms"][stg] / max(kt["calls"][stg], 1)
        achieved = useful_per_step / (avg_ms / 1e3) / 1e9
        peak = ffma_s / FP32_PER_PAIR[stg] / 1e9
        kernels[stg] = {"kernel": KERNEL_OF[stg], "pairs_per_launch": useful_per_step, "avg_launch_ms": avg_ms,
                        "fp32_per_pair": FP32_PER_PAIR[stg], "achieved": achieved, "peak": peak,
                        "frac": achieved / peak, "evaluated_pairs_per_launch": evaluated[stg],
                        "useful_fraction": useful_per_step / max(evaluated[stg], 1)}
    dom = max(("fwd_eval", "bwd_eval"), key=lambda k: kt["ms"][k])
    traffic = profiled_traffic(KERNEL_OF[dom], "%s-%dx%d" % (name, shape.tile_h, shape.tile_w))
    roofline = dict(kernels[dom], bound="alu", unit="Gpair/s", traffic=traffic, ffma_lane_ops_per_s=ffma_s,
                    peak_basis="measured FFMA rate %.4e lane-ops/s on this GPU (%d SMs; packed FFMA2 %.3e instr/s, "
                               "ex2.approx %.3e/s) / %.0f FP32 operations per in-cut pair (MEASURED_PEAKS.json "
                               "has no FP32 figure)" % (ffma_s, n_sm, ffma2_s, ex2_s, FP32_PER_PAIR[dom]),
                    other=kernels["fwd_eval" if dom == "bwd_eval" else "bwd_eval"])

    # the same step replayed as one CUDA graph per iteration, timed separately after the eager region
    kg = max(3, min(steps, 200))
    try:
        gsvr.gsvr_graph_capture(ctx.ctx, n_s if sampled else -1)
        gsvr.gsvr_set_step(ctx.ctx, warmup + steps + 3)
        gsvr.gsvr_graph_launch(ctx.ctx, 3)
        gsvr.gsvr_sync_status(ctx.ctx)
        g_err = None
    except gsvr.GsvrError as e:  # reported in the line; the eager measurement stands
        g_err = str(e)
    if ws > 1:
        torch.distributed.barrier()
    if g_err is None:
        torch.cuda.synchronize()
        g0 = torch.cuda.Event(enable_timing=True)
        g1 = torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        gsvr.gsvr_graph_launch(ctx.ctx, kg)
        g1.record(stream)
        torch.cuda.synchronize()
        gsvr.gsvr_sync_status(ctx.ctx)
        g_ms = reduce_max(g0.elapsed_time(g1), ws)
        graph = {"ms_per_step": g_ms / kg, "value": reduce_sum(useful_per_step * kg, ws) / (g_ms / 1e3),
                 "unit": UNIT, "steps": kg}
    else:
        graph = {"error": g_err}

    # end to end through the host-buffer call
    e2e = None
    if with_e2e:
        rng = np.random.default_rng(99 + rank)
        masked = np.nonzero(case["mask"])[0].astype(np.int32)
        ke = max(3, min(steps, 20))
        if sampled:
            lists = [np.sort(rng.choice(masked, n_s, replace=False)).astype(np.int32) for _ in range(ke + 2)]
        else:
            lists = [masked] * (ke + 2)
        theta_h = torch.from_numpy(case["theta"].astype(np.float32)).pin_memory()
        grad_h = torch.empty_like(theta_h).pin_memory()
        loss_h = torch.zeros(1, dtype=torch.float64).pin_memory()
        idx_h = [torch.from_numpy(l).pin_memory() for l in lists[:ke + 2 if sampled else 1]]
        for k in range(2):
            gsvr.gsvr_step_host(ctx.ctx, theta_h, idx_h[k % len(idx_h)], grad_h, loss_h)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(ke):
            gsvr.gsvr_step_host(ctx.ctx, theta_h, idx_h[(2 + k) % len(idx_h)], grad_h, loss_h)
        dt = reduce_max(time.perf_counter() - t0, ws)
        e2e = {"value": reduce_sum(useful_per_step * ke, ws) / dt, "unit": UNIT,
               "h2d_bytes_per_step": int(theta_h.numel() * 4 + n_s * 4),
               "d2h_bytes_per_step": int(grad_h.numel() * 4 + 8), "steps": ke,
               "pairs_per_step": "the eager region's in-cut pairs per step"}

    cpu = None
    if with_cpu and rank == 0 and ws == 1:
        sample = gsvr.gsvr_get_sample(ctx.ctx)
        rng = np.random.default_rng(7)
        n_px = 16
        while True:  # grow the sample until the oracle runs for args.cpu_seconds
            pix = rng.choice(sample, min(n_px, sample.size), replace=False)
            t_cpu, u_cpu, cores = cpu_oracle_sample(case, pix, n_s)
            if t_cpu >= 0.8 * args.cpu_seconds or n_px >= min(65536, sample.size):
                break
            n_px = int(min(65536, n_px * max(2.0, min(32.0, args.cpu_seconds / max(t_cpu, 1e-3)))))
        cpu = {"value": u_cpu / t_cpu, "unit": UNIT, "cores": cores, "kind": "oracle",
               "px_per_s": len(pix) / t_cpu,
               "sample": "%d of the step's pixels x all %d Gaussians, fwd+bwd (all gradients), float64, %.1f s" %
                         (len(pix), case["N"], t_cpu)}

    stats = ctx.stats()
    # HBM-bound stages against the measured copy bandwidth: algorithmic bytes per
    # step (prep: 44 B read + 40 B written per Gaussian; binning: ~68 B per slab
    # candidate record (read 40, write 24, count 4) and 44 B per key (emit 8, two
    # 8-bit radix passes of 8 B read + 8 B write, tile offset 4); Adam: 28 B per
    # parameter) over the stage's CUDA-event time in the timed region
    peaks_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    hbm = json.load(open(peaks_path)).get("hbm_gbs") if os.path.exists(peaks_path) else None
    hbm_basis = "measured copy bandwidth (MEASURED_PEAKS.json hbm_gbs)" if hbm else "fallback 6400 GB/s"
    hbm = float(hbm or 6400.0)
    n_par = 11 * case["N"] + 6 * M
    stage_bytes = {"prep": 84.0 * case["N"], "bin": 68.0 * stats["n_records"] + 44.0 * stats["n_keys"],
                   "adam": 28.0 * n_par}
    hbm_stages = {"peak_gbs": hbm, "peak_basis": hbm_basis}
    for k, b in stage_bytes.items():
        ms_k = kt["ms"][k] / max(steps, 1)
        gbs = b / (ms_k / 1e3) / 1e9 if ms_k > 0 else None
        hbm_stages[k] = {"bytes_per_step": b, "ms_per_step": ms_k, "achieved_gbs": gbs,
                         "frac": gbs / hbm if gbs else None}
    # adjoint memory: what the recompute design keeps against one float32 per in-cut pair
    kept = stats["n_keys"] * (32 + 32 + 4 + 4) + stats["n_records"] * (32 + 8 + 4 + 4)
    memory = {"recompute_bytes": int(kept), "store_per_pair_bytes": int(useful_per_step * 4),
              "note": "recompute keeps records, keys, tile-ordered references and per-key moments; storing one "
                      "float32 factor per in-cut pair is the alternative"}
    out = {"value": value, "ms_per_step": ms_max / steps, "desc": desc, "n_sample": n_s,
           "tile": "%dx%d" % (shape.tile_h, shape.tile_w), "launch_shape": shape_d, "autotune": tuning,
           "l2": "inputs larger than L2 (records + keys + tile records ~%.0f MB per step)" %
                 ((stats["n_records"] * 44 + stats["n_keys"] * 108) / 1e6),
           "px_per_s": px_total / (ms_max / 1e3), "useful_pairs_per_step": useful_per_step,
           "useful_pairs_start_end": [useful_start, useful_end],
           "tile_pairs_per_step": tile_pairs_per_step,
           "useful_fraction": useful_per_step / max(tile_pairs_per_step, 1),
           "stage_ms_per_step": {k: v / steps for k, v in kt["ms"].items()},
           "records_per_step": stats["n_records"], "keys_per_step": stats["n_keys"], "roofline": roofline,
           "hbm_stages": hbm_stages, "graph": graph, "cpu_baseline": cpu, "e2e": e2e, "memory": memory,
           "gpu_launches": kt["kernel_launches"], "clocks": clk}
    ctx.close()
    return out


def main():
    args = parse()
    ws, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, ws, rank)
        return
    import torch
    from paper_2512_11624_b300 import gsvr
    torch.cuda.set_device(local)
    stream = torch.cuda.Stream(device=local)
    head = measure(args, gsvr, torch, local, stream, args.workload, rank, ws, args.steps, args.warmup,
                   not args.no_e2e, not args.no_cpu_baseline, True, args.tile)
    fetal = None
    if args.workload == "large" and not args.no_fetal:
        fs = max(3, min(args.steps * 5, 1000))
        f = measure(args, gsvr, torch, local, stream, "fetal", rank, ws, fs, max(args.warmup, 3), False, False, False,
                    args.fetal_tile)
        fetal = {k: f[k] for k in ("value", "ms_per_step", "desc", "tile", "px_per_s", "useful_pairs_per_step",
                                   "tile_pairs_per_step", "useful_fraction", "stage_ms_per_step", "roofline",
                                   "hbm_stages", "graph", "gpu_launches")}
        fetal["steps"] = fs
    if rank == 0:
        line = {"metric": METRIC, "value": head["value"], "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": head["desc"], "tile": head["tile"], "launch_shape": head["launch_shape"],
                           "autotune": head["autotune"], "parallelism": "replicas" if ws > 1 else "single",
                           "l2": head["l2"]},
                "px_per_s": head["px_per_s"], "useful_pairs_per_step": head["useful_pairs_per_step"],
                "useful_pairs_start_end": head["useful_pairs_start_end"],
                "tile_pairs_per_step": head["tile_pairs_per_step"], "useful_fraction": head["useful_fraction"],
                "stage_ms_per_step": head["stage_ms_per_step"], "records_per_step": head["records_per_step"],
                "keys_per_step": head["keys_per_step"], "roofline": head["roofline"],
                "hbm_stages": head["hbm_stages"], "graph": head["graph"], "cpu_baseline": head["cpu_baseline"],
                "e2e": head["e2e"], "memory": head["memory"], "gpu_launches": head["gpu_launches"],
                "clocks": head["clocks"], "fetal": fetal}
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
