"""Reconstruction studies on synthetic subjects (run on a GPU):

  python -m paper_2512_11624_b300.study batched [--subjects 16] [--iters 2000] [--out FILE]

`batched`: the batched multi-subject workload (`inputs.batched`: 16 subjects of
uneven size).  Every subject is first reconstructed alone (its own context with
an autotuned launch shape, eager iterations on a fixed-capacity context), which
fixes its target PSNR = PSNR after `iters` iterations - 0.5 dB; then all
subjects are reconstructed together in one batched context (autotuned, one CUDA
graph per iteration).  Reported per subject: iterations and device seconds to
the target alone and batched; in aggregate: device seconds for all subjects'
`iters` iterations and useful (pixel, Gaussian) pairs per second both ways.
Evaluations (PSNR every `eval_every` iterations) are outside the timed device
time.
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import time

import numpy as np


def _make_subject(args):
    seed, k = args
    from . import inputs
    rng_seed = seed + k
    cases = inputs.batched(rng_seed, n_subjects=1)
    c = cases[0]
    c["name"] = "subject%d" % k
    return c


def make_subjects(seed, n, workers):
    """Subject k is inputs.batched(seed + k, 1)[0] == inputs.batched(seed, n)[k]."""
    if workers <= 1:
        return [_make_subject((seed, k)) for k in range(n)]
    ctx = mp.get_context("spawn")
    with ctx.Pool(workers) as pool:
        return pool.map(_make_subject, [(seed, k) for k in range(n)])


def useful_pairs_per_iter(ctx, sample):
    from . import gsvr
    sample()
    gsvr.gsvr_forward(ctx.ctx)
    u, e = gsvr.gsvr_count_pairs(ctx.ctx)
    return int(u), int(e)


def run_batched(args):
    t_gen = time.time()
    subjects = make_subjects(args.seed, args.subjects, args.workers)
    t_gen = time.time() - t_gen
    import torch
    from . import gsvr, inputs
    from .recon import BatchedReconstruction, PSNRProbe, Reconstruction
    dev = 0
    torch.cuda.set_device(dev)
    out = {"workload": "batched: %d subjects (seeds %d..%d), N log-uniform [50k, 500k], 3-9 stacks, 24-60 slices, "
                       "128^2-256^2 px, thickness U(2.5, 4.5) mm, motion U(+-15 deg)/U(+-8 mm), 2^18 sampled px "
                       "per subject per iteration" % (args.subjects, args.seed, args.seed + args.subjects - 1),
           "iters": args.iters, "eval_every": args.eval_every, "generate_s": t_gen, "subjects": []}
    probes = [PSNRProbe(c["phantom"], c["N"], device=dev) for c in subjects]
    # alone
    alone_total = 0.0
    alone_useful = 0
    for k, c in enumerate(subjects):
        rec = Reconstruction(c, device=dev, n_sample=args.n_sample, tune=True)
        res = rec.run(args.iters, probe=probes[k], eval_every=args.eval_every)
        hist = res["history"]
        final = hist[-1][3]
        target = final - 0.5
        hit = next(((it, s) for it, s, _, p in hist[1:] if p >= target), (None, None))
        n_mask = int(c["mask"].sum())
        u, e = useful_pairs_per_iter(rec.ctx, lambda: gsvr.gsvr_sample_pixels(rec.ctx.ctx, min(args.n_sample, n_mask),
                                                                                  10 ** 6))
        dev_s = hist[-1][1]
        alone_total += dev_s
        alone_useful += u * args.iters
        sh = rec.shape
        out["subjects"].append({"N": int(c["N"]), "stacks": len(c["stacks"]), "slices": int(c["stacks"][0]["n_slices"]),
                                "W": int(c["stacks"][0]["W"]), "masked_px": n_mask,
                                "shape": "%dx%d px%d order%d" % (sh.tile_h, sh.tile_w, sh.fwd_px_per_thread,
                                                                 sh.queue_order),
                                "psnr_start": hist[0][3], "psnr_final_alone": final, "target": target,
                                "alone": {"ms_per_iter": 1e3 * dev_s / args.iters, "iters_to_target": hit[0],
                                          "s_to_target": hit[1], "useful_pairs_per_iter": u,
                                          "evaluated_pairs_per_iter": e}})
        print("alone %2d: N %6d  %.3f ms/iter  PSNR %.2f -> %.2f  target at %s" %
              (k, c["N"], 1e3 * dev_s / args.iters, hist[0][3], final, hit[0]), flush=True)
        rec.close()
    # batched
    br = BatchedReconstruction(subjects, device=dev, n_sample=args.n_sample, tune=True, graph=not args.no_graph)
    targets = [s["target"] for s in out["subjects"]]
    res = br.run(args.iters, probes=probes, eval_every=args.eval_every, targets=targets)
    hist = res["history"]
    bt = hist[-1][1]
    ub, eb = useful_pairs_per_iter(br.ctx, lambda: gsvr.gsvr_sample_pixels_subjects(br.ctx.ctx, args.n_sample, 10 ** 6))
    for k, s in enumerate(out["subjects"]):
        s["psnr_final_batched"] = hist[-1][3][k]
        s["batched"] = {"iters_to_target": res["iters_to_target"][k], "s_to_target": res["time_to_target"][k]}
    sh = br.shape
    out["batched"] = {"ms_per_iter": 1e3 * bt / args.iters, "device_s": bt, "graph": not args.no_graph,
                      "shape": "%dx%d px%d fwd%d bwd%d order%d" % (sh.tile_h, sh.tile_w, sh.fwd_px_per_thread,
                                                                   sh.fwd_blocks_per_sm, sh.bwd_blocks_per_sm,
                                                                   sh.queue_order),
                      "useful_pairs_per_s": ub * args.iters / bt, "evaluated_pairs_per_iter": eb}
    out["alone"] = {"device_s": alone_total, "useful_pairs_per_s": alone_useful / alone_total}
    all_alone = [s["alone"]["s_to_target"] for s in out["subjects"]]
    all_b = [s["batched"]["s_to_target"] for s in out["subjects"]]
    if all(v is not None for v in all_alone + all_b):
        out["all_targets"] = {"alone_sequential_s": float(sum(all_alone)), "batched_s": float(max(all_b))}
    out["speedup_device_time"] = alone_total / bt
    print("batched: %.3f ms/iter (%d subjects), alone total %.2f s vs batched %.2f s -> %.2fx; useful pairs/s "
          "%.3g alone vs %.3g batched" % (1e3 * bt / args.iters, args.subjects, alone_total, bt, alone_total / bt,
                                          out["alone"]["useful_pairs_per_s"], out["batched"]["useful_pairs_per_s"]),
          flush=True)
    br.close()
    for p in probes:
        p.close()
    if args.out:
        with open(args.out, "w") as f:
            json.dump(out, f, indent=1)
    return out


def main():
    ap = argparse.ArgumentParser()
    sub = ap.add_subparsers(dest="cmd", required=True)
    b = sub.add_parser("batched")
    b.add_argument("--subjects", type=int, default=16)
    b.add_argument("--seed", type=int, default=1000)
    b.add_argument("--iters", type=int, default=2000)
    b.add_argument("--eval-every", type=int, default=25)
    b.add_argument("--n-sample", type=int, default=1 << 18)
    b.add_argument("--workers", type=int, default=8)
    b.add_argument("--no-graph", action="store_true")
    b.add_argument("--out", default="")
    args = ap.parse_args()
    if args.cmd == "batched":
        run_batched(args)


if __name__ == "__main__":
    main()
