"""Reconstruction studies on synthetic subjects (run on a GPU):

  python -m paper_2512_11624_b300.study batched [--subjects 16] [--iters 2000] [--out FILE]
  python -m paper_2512_11624_b300.study learned [--phantoms 2000] [--epochs 20] [--cases 10] [--out FILE]
  python -m paper_2512_11624_b300.study topk [--k 10 20 50 80] [--iters 600] [--out FILE]
  python -m paper_2512_11624_b300.study cnnbench [--batch 256] [--steps 50]
  python -m paper_2512_11624_b300.study init [--model plain|topk] [--density-scales] [--lambdas 0 0.5 1] [--out FILE]
  python -m paper_2512_11624_b300.study metrics [--h 0.8 0.5 0.4]
  python -m paper_2512_11624_b300.study densify [--h0 2.4] [--every 50] [--frac 0.5] [--out FILE]

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

`learned`: the pose network (include/gsvr_cnn.h) is trained on slices that the
forward model renders from phantoms of the canonical-frame family under motion
U(+-20 deg) / U(+-10 mm), then initialises fetal-sized test cases (new seeds;
motion at that range and at the plain workload's U(+-5 deg) / U(+-3 mm)): the
network's pose for every slice with brain content, kept only where it matches
a template volume (the family's seed-0 member) better than the nominal pose
(normalised cross-correlation of the slice with the template rendered at
each pose; the others fall back to nominal), then the plain optimisation
refines.  Reported per case: pose errors (rotation angle, slice-centre
displacement) of the network alone, after refinement and of the plain method
from nominal, the fallback count, and seconds to the target PSNR (plain from
nominal after `iters` iterations - 0.5 dB) both ways, the learned path
including its inference and fallback time.
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
    if args.retire:
        # the batch again, converged subjects leaving it (same targets)
        br.close()
        br = BatchedReconstruction(subjects, device=dev, n_sample=args.n_sample, tune=True, graph=not args.no_graph)
        rr = br.run(args.iters, probes=probes, eval_every=args.eval_every, targets=targets, retire=True)
        rt = rr["time_to_target"]
        for k, s in enumerate(out["subjects"]):
            s["batched_retire"] = {"iters_to_target": rr["iters_to_target"][k], "s_to_target": rt[k]}
        out["batched_retire"] = {"device_s": rr["history"][-1][1],
                                 "s_all_targets": max(rt) if all(v is not None for v in rt) else None}
        print("batched, converged subjects retired: every target after %s s (alone sequential %s s)" %
              (out["batched_retire"]["s_all_targets"], out.get("all_targets", {}).get("alone_sequential_s")),
              flush=True)
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


def _make_fetal(args):
    seed, deg, mm = args
    from . import inputs
    return inputs.fetal(seed, with_truth=True, init="flat", motion_deg=deg, motion_mm=mm, jitter=0.15)


def pose_errors(stacks, est, truth, sel):
    """Rotation angle (deg) between the estimated and true slice rotations and
    displacement (mm) of the slice centre, over the slices in `sel`."""
    from scipy.spatial.transform import Rotation
    c0 = []
    for st in stacks:
        n = st["n_slices"]
        for k in range(n):
            c0.append(st["origin"] + (k - 0.5 * (n - 1)) * st["thickness"] * st["R"][:, 2])
    c0 = np.array(c0)[sel]
    Re, Rt = Rotation.from_rotvec(est[sel, :3]), Rotation.from_rotvec(truth[sel, :3])
    ang = np.rad2deg((Re.inv() * Rt).magnitude())
    te = Re.apply(c0) + est[sel, 3:]
    tt = Rt.apply(c0) + truth[sel, 3:]
    d = np.linalg.norm(te - tt, axis=1)
    return {"deg_mean": float(ang.mean()), "deg_median": float(np.median(ang)), "mm_mean": float(d.mean()),
            "mm_median": float(np.median(d))}


def slice_ncc(pred, obs, msk):
    """Per-slice normalised cross-correlation over the masked pixels (torch)."""
    import torch
    m = msk.float()
    n = m.sum(1).clamp(min=1.0)
    mp = (pred * m).sum(1) / n
    mo = (obs * m).sum(1) / n
    dp = (pred - mp[:, None]) * m
    do = (obs - mo[:, None]) * m
    return (dp * do).sum(1) / torch.sqrt((dp * dp).sum(1) * (do * do).sum(1)).clamp(min=1e-20)


def run_learned(args):
    n_c4, n_c1 = args.cases, args.cases_c1
    specs = [(7000 + k, 20.0, 10.0) for k in range(n_c4)] + [(8000 + k, 5.0, 3.0) for k in range(n_c1)]
    t_gen = time.time()
    if args.workers > 1:
        with mp.get_context("spawn").Pool(args.workers) as pool:
            cases = pool.map(_make_fetal, specs)
    else:
        cases = [_make_fetal(sp) for sp in specs]
    t_gen = time.time() - t_gen
    import torch
    from . import cnn, gsvr, inputs
    from .recon import PSNRProbe, Reconstruction
    dev = 0
    torch.cuda.set_device(dev)
    log = lambda m: print(m, flush=True)  # noqa: E731
    t0 = time.time()
    X, A, Y = cnn.make_training_set(args.phantoms, motions_per_phantom=args.motions, seed=args.seed, log=log)
    t_data = time.time() - t0
    log("training set: %d slices in %.1f s" % (X.shape[0], t_data))
    net = cnn.PoseNet(max_batch=args.batch, seed=args.seed)
    hist = cnn.train(net, X, A, Y, epochs=args.epochs, batch=args.batch, lr=args.lr, seed=args.seed, log=log)
    n_train = int(X.shape[0])
    del X, A, Y
    torch.cuda.empty_cache()
    out = {"training": {"slices": n_train, "phantoms": args.phantoms, "motions_per_phantom": args.motions,
                        "data_s": t_data, "epochs": hist, "batch": args.batch, "lr": args.lr},
           "generate_cases_s": t_gen, "iters": args.iters, "cases": []}
    # template volume for the fallback test: the family's seed-0 member on a 1.5 mm grid
    tmpl_theta, tmpl_N = inputs.grid_gaussians(inputs.BrainPhantom(0), h=1.5, s=1.5)
    for (seed, deg, mm), case in zip(specs, cases):
        M = inputs.n_slices_total(case["stacks"])
        H = W = 192
        truth = case["motion"]
        ref = case["ref_slice"]
        st = torch.cuda.Stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        I = torch.from_numpy(case["I"]).cuda().reshape(M, H, W)
        msk = torch.from_numpy(case["mask"]).cuda().reshape(M, H, W) > 0
        torch.cuda.synchronize()
        t_inf0 = time.perf_counter()
        lo = (H - cnn.IMAGE) // 2
        crop = I[:, lo:lo + cnn.IMAGE, lo:lo + cnn.IMAGE].contiguous()
        content = cnn.content_fraction(crop) > 0.02
        aux_h = cnn.aux_for_stacks(case["stacks"])
        aux = torch.from_numpy(aux_h).cuda()
        pred = cnn.pose_from_output(cnn.predict(net, cnn.normalise_slices(crop), aux).cpu().numpy(), aux_h)
        # fallback test against the template
        tc = {"stacks": case["stacks"], "N": tmpl_N,
              "theta": np.concatenate([tmpl_theta, np.zeros(6 * M)]).astype(np.float32), "I": case["I"],
              "mask": case["mask"]}
        tctx = gsvr.Context(tc, tile_h=12, tile_w=12)
        # candidates per slice: nominal, the network's pose, its translation alone
        trans_only = np.concatenate([np.zeros((M, 3)), pred[:, 3:]], axis=1)
        cands = [np.zeros((M, 6)), pred, trans_only]
        ncc = []
        for poses in cands:
            gsvr.gsvr_set_poses(tctx.ctx, poses.astype(np.float32).reshape(-1))
            tctx.forward()
            ncc.append(slice_ncc(tctx.pred.reshape(M, -1), I.reshape(M, -1), msk.reshape(M, -1)))
        tctx.close()
        score = torch.stack(ncc).cpu().numpy()  # [3][M]
        pick = np.argmax(score, axis=0)
        cont = content.cpu().numpy()
        pick[~cont] = 0
        pick[ref] = 0
        init = np.stack(cands)[pick, np.arange(M)]
        use = pick > 0
        torch.cuda.synchronize()
        t_inf = time.perf_counter() - t_inf0
        sel = content.cpu().numpy().copy()
        sel[ref] = False
        rec_out = {}
        probe = PSNRProbe(case["phantom"], case["N"])
        for name, poses in (("plain", np.zeros((M, 6))), ("learned", init)):
            c = dict(case)
            th = case["theta"].copy()
            th[11 * case["N"]:] = poses.astype(np.float32).reshape(-1)
            c["theta"] = th
            rec = Reconstruction(c, n_sample=1 << 18, fixed=True)
            res = rec.run(args.iters, probe=probe, eval_every=args.eval_every)
            est = rec.ctx.theta[11 * case["N"]:].cpu().numpy().astype(np.float64).reshape(M, 6)
            rec_out[name] = {"history": [(it, s_, p) for it, s_, _, p in res["history"]],
                             "pose_error": pose_errors(case["stacks"], est, truth, sel)}
            rec.close()
        probe.close()
        target = rec_out["plain"]["history"][-1][2] - 0.5
        for name in rec_out:
            h = rec_out[name]["history"]
            hit = next(((it, s_) for it, s_, p in h[1:] if p >= target), (None, None))
            extra = t_inf if name == "learned" else 0.0
            rec_out[name]["iters_to_target"] = hit[0]
            rec_out[name]["s_to_target"] = None if hit[1] is None else hit[1] + extra
            rec_out[name]["psnr_final"] = h[-1][2]
            del rec_out[name]["history"]
        row = {"seed": seed, "motion": [deg, mm], "slices_with_content": int(sel.sum()),
               "fallbacks": int((~use & sel).sum()), "translation_only": int(((pick == 2) & sel).sum()),
               "inference_s": t_inf, "target_psnr": target,
               "selected": pose_errors(case["stacks"], init, truth, sel),
               "network": pose_errors(case["stacks"], pred, truth, sel),
               "nominal": pose_errors(case["stacks"], np.zeros((M, 6)), truth, sel), **rec_out}
        out["cases"].append(row)
        log("case %d (+-%g deg): net %.2f deg %.2f mm | nominal %.2f deg %.2f mm | fallbacks %d/%d | "
            "to target: plain %s s (it %s), learned %s s (it %s) | refined: plain %.2f deg, learned %.2f deg" %
            (seed, deg, row["network"]["deg_mean"], row["network"]["mm_mean"], row["nominal"]["deg_mean"],
             row["nominal"]["mm_mean"], row["fallbacks"], row["slices_with_content"],
             _fmt(rec_out["plain"]["s_to_target"]), rec_out["plain"]["iters_to_target"],
             _fmt(rec_out["learned"]["s_to_target"]), rec_out["learned"]["iters_to_target"],
             rec_out["plain"]["pose_error"]["deg_mean"], rec_out["learned"]["pose_error"]["deg_mean"]))
    net.close()
    if args.out:
        with open(args.out, "w") as f:
            json.dump(out, f, indent=1)
    return out


def conv_flops_per_slice():
    """Multiply-adds x 2 of the six conv layers for one 128 x 128 slice (forward)."""
    ch = [1, 32, 64, 128, 256, 256, 512]
    f, side = 0, 128
    for l in range(6):
        side = (side + 1) // 2
        f += 2 * side * side * ch[l + 1] * 9 * ch[l]
    return f


def run_cnnbench(args):
    """Training-step throughput of the pose network on random slices: CUDA
    events around `steps` steps (forward, loss, backward, Adam) after warm-up;
    FLOPs = 3 x the conv forward FLOPs (forward, input gradient, weight
    gradient) + the fc layers' 6 x multiply-adds; against the measured bf16
    peak (MEASURED_PEAKS.json when present)."""
    import torch
    from . import cnn
    dev = 0
    torch.cuda.set_device(dev)
    B = args.batch
    g = torch.Generator(device="cuda").manual_seed(0)
    x = torch.rand((B, 128, 128), device="cuda", generator=g)
    aux = torch.randn((B, 25), device="cuda", generator=g)
    tgt = torch.randn((B, 6), device="cuda", generator=g) * 0.3
    net = cnn.PoseNet(max_batch=B, seed=1)
    for t in range(1, args.warmup + 1):
        net.loss_backward(x, aux, tgt)
        net.adam_step(t)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for t in range(args.steps):
        net.loss_backward(x, aux, tgt)
        net.adam_step(args.warmup + 1 + t)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    fc = 2 * B * ((2048 + 25) * 256 + 256 * 6)
    flops = 3 * B * conv_flops_per_slice() + 3 * fc
    peak = None
    try:
        import os
        pk = json.load(open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                                         "MEASURED_PEAKS.json")))
        peak = pk.get("bf16_tflops_sustained") or pk.get("bf16_tflops")
    except Exception:
        peak = None
    tf = flops / (ms / 1e3) / 1e12
    out = {"batch": B, "ms_per_step": ms, "slices_per_s": B / (ms / 1e3), "tflops": tf, "peak_tflops": peak,
           "frac": (tf / peak) if peak else None}
    print(json.dumps(out), flush=True)
    net.close()
    return out


def _fmt(v):
    return "-" if v is None else "%.2f" % v


def run_topk(args):
    """The normalised top-K model (Eq. 2 / Eq. 5 ratio over the K nearest
    Gaussians) against the plain sum on the fetal workload: per configuration,
    `iters` iterations (2^18 sampled pixels, Adam with StepLR), device seconds
    per iteration, stage times, PSNR of the volume each model defines (the
    top-K model's probe reads the ratio, the plain one the sum) every
    `eval_every` iterations, and the device seconds to the plain run's final
    PSNR - 0.5 dB.  The ratio's amplitudes are O(1) colours: its initial c is
    the plain initial c divided by the plain sum's grid factor h^3 / ((2 pi)^(3/2) s^3),
    and its c learning rate the plain one divided by the same factor.  A ratio
    model predicts the nearest Gaussians' colours however far they are, so its
    runs also start with zero-amplitude background Gaussians (2.4 mm grid) over
    the 15 mm band of the pixel mask outside the brain.  `loss` / `lambda_reg`
    / `s_target` set the ratio runs' objective (Sec. 2.5): the regulariser's
    weight is the paper's per-pixel-sum weight divided by the sample size (our
    data term is a mean over the sampled pixels), and s_target defaults to
    the Gaussians' initial scale and spacing (0.8 mm; the paper's 1.6 mm goes
    with its 10-80 k Gaussians per brain, ours are 200 k)."""
    import torch
    from . import gsvr, inputs
    from .recon import PLAIN_LR, PSNRProbe, Reconstruction
    torch.cuda.set_device(0)
    case = inputs.fetal(args.seed)
    N = case["N"]
    factor = 1.0 / (2 * np.pi) ** 1.5  # h^3 / ((2 pi)^(3/2) s^3) with h = s = 0.8 mm
    configs = [("plain", None)] + [("topk K=%d" % K, (K, args.delta, args.refresh)) for K in args.k]
    out = []
    target = None
    for name, tk in configs:
        c = dict(case)
        lr = None
        if tk:
            th = case["theta"].copy()
            th[10 * N:11 * N] /= factor
            c["theta"] = th
            bg, nb = inputs.background_gaussians(case["phantom"])
            c = inputs.with_gaussians(c, bg, nb)
            lr = dict(lr_c=PLAIN_LR["lr_c"] / factor)
        # plain: the fixed-capacity context of the other studies (no host
        # synchronisation per iteration); top-K: no capacities involved
        rec = (Reconstruction(c, n_sample=args.n_sample, lr=lr, topk=tk, timing=1) if tk else
               Reconstruction(c, n_sample=args.n_sample, fixed=True))
        if tk:
            gsvr.gsvr_set_objective(rec.ctx.ctx, 1 if args.loss == "l1" else 0, args.lambda_reg / args.n_sample,
                                    args.s_target)
            if args.slice_weights:
                gsvr.gsvr_set_slice_weights(rec.ctx.ctx, 1)
        probe = PSNRProbe(case["phantom"], c["N"], topk=(tk[0], tk[1]) if tk else None)
        if tk:
            gsvr.gsvr_timing_reset(rec.ctx.ctx)
        res = rec.run(args.iters, probe=probe, eval_every=args.eval_every, target_psnr=target)
        hist = res["history"]
        iters = hist[-1][0]
        stage = None
        if tk:
            kt = gsvr.gsvr_get_kernel_times(rec.ctx.ctx)
            stage = {k: kt["ms"][k] / max(iters, 1) for k in ("sample", "prep", "bin", "fwd_eval", "bwd_eval",
                                                              "grad", "adam")}
        row = {"model": name, "K": tk[0] if tk else None, "delta": tk[1] if tk else None,
               "loss": args.loss if tk else "mse", "lambda_reg": args.lambda_reg if tk else 0.0,
               "slice_weights": bool(args.slice_weights and tk),
               "s_target": args.s_target if tk else None,
               "refresh_every": tk[2] if tk else None, "iters": iters, "ms_per_iter": 1e3 * hist[-1][1] / iters,
               "stage_ms_per_iter": stage, "psnr": [(h[0], h[3]) for h in hist],
               "seconds_to_target": res["time_to_target"], "target_psnr": target,
               "pairs_per_s": (args.n_sample * tk[0] / (hist[-1][1] / iters)) if tk else None}
        if target is None:
            target = hist[-1][3] - 0.5
            row["target_psnr"] = target
            row["seconds_to_target"] = next((h[1] for h in hist if h[3] is not None and h[3] >= target), None)
        print(json.dumps(row), flush=True)
        out.append(row)
        probe.close()
        rec.close()
    if args.out:
        json.dump(out, open(args.out, "w"), indent=1)


def density_scales(mu, cell=2.0, smin=0.4, smax=4.0):
    """Isotropic scale per mean from the local density of the means: the count
    of means in each `cell`-mm cube, s = density^(-1/3) (the local spacing),
    clipped to [smin, smax] mm.  mu: (3, N) CUDA tensor."""
    import torch
    lo = mu.min(dim=1, keepdim=True).values
    idx = ((mu - lo) / cell).floor().long()
    dims = idx.max(dim=1).values + 1
    key = (idx[0] * dims[1] + idx[1]) * dims[2] + idx[2]
    cnt = torch.zeros(int(dims.prod()), device=mu.device).scatter_add_(0, key, torch.ones(key.shape, device=mu.device))
    return (cnt[key] / cell ** 3).pow(-1.0 / 3.0).clamp(smin, smax)


def run_init(args):
    """Content-adaptive initialisation (Sec. 2.5) against the grid start on the
    fetal workload.  Every run has the grid's Gaussian count and identity
    rotations and differs in where the means start, their scales and their
    amplitudes.  "grid": means on the 0.8 mm grid inside the brain, scale
    0.8 mm, one flat amplitude (the mean observed brain intensity).
    "adaptive lambda": means drawn by gsvr_init_means from the slices at their
    nominal poses with mixing weight lambda, each amplitude the observed
    intensity of its drawn pixel (the paper does not say how scales and
    colours start); scales 0.8 mm, or with `--density-scales` the local spacing
    of the drawn means (density_scales), since a plain sum of Gaussians adds
    up where means cluster.  Plain sum (`--model plain`): amplitudes carry the
    factor h^3 / ((2 pi)^(3/2) s^3) with h the spacing (= s).  Normalised top-K
    model (`--model topk`, K = `--k`): amplitudes are the colours themselves,
    and zero-colour background Gaussians cover the mask band outside the brain
    as in the top-K study.  Reported per run: the device time of the
    initialisation, PSNR every `eval_every` iterations, and PSNR / SSIM / NCC
    of the volume against the phantom (gsvr_volume_metrics over the phantom's
    voxels) at the start and after `iters` iterations, with the device seconds
    of the iterations."""
    import torch
    from . import gsvr, inputs
    from .recon import PLAIN_LR, PSNRProbe, Reconstruction
    torch.cuda.set_device(0)
    flat = inputs.fetal(args.seed, init="flat")
    N = flat["N"]
    M = inputs.n_slices_total(flat["stacks"])
    topk = args.model == "topk"
    grid_factor = 1.0 / (2 * np.pi) ** 1.5  # h^3 / ((2 pi)^(3/2) s^3) with h = s
    configs = [("grid", None)] + [("adaptive lambda=%g" % lam, lam) for lam in args.lambdas]
    out = []
    for name, lam in configs:
        case = dict(flat)
        init_ms = None
        g = flat["theta"][:11 * N].reshape(11, N).copy()
        if lam is not None:
            ctx = gsvr.Context(flat)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            zero = np.zeros((M, 6), np.float32)
            gsvr.gsvr_init_means(ctx.ctx, N, lam, args.seed + 1, pose=zero)  # warm-up
            torch.cuda.synchronize()
            e0.record()
            mu, pix, _ = gsvr.gsvr_init_means(ctx.ctx, N, lam, args.seed + 1, pose=zero)
            e1.record()
            e1.synchronize()
            init_ms = e0.elapsed_time(e1)
            ctx.close()
            s = density_scales(mu) if args.density_scales else torch.full((N,), 0.8, device=mu.device)
            g[0:3] = mu.cpu().numpy()
            g[3:6] = np.log(s.cpu().numpy())[None, :]
            g[10] = np.asarray(flat["I"], np.float32)[pix.cpu().numpy()] * (1.0 if topk else grid_factor)
        elif topk:
            g[10] /= grid_factor
        case["theta"] = np.concatenate([g.reshape(-1), flat["theta"][11 * N:]]).astype(np.float32)
        if topk:
            bg, nb = inputs.background_gaussians(case["phantom"])
            case = inputs.with_gaussians(case, bg, nb)
            rec = Reconstruction(case, n_sample=args.n_sample, lr=dict(lr_c=PLAIN_LR["lr_c"] / grid_factor),
                                 topk=(args.k, 1e-8, 1))
            probe = PSNRProbe(case["phantom"], case["N"], topk=(args.k, 1e-8))
        else:
            rec = Reconstruction(case, n_sample=args.n_sample, fixed=True)
            probe = PSNRProbe(case["phantom"], N)
        m0 = probe.metrics(rec.ctx.theta)
        res = rec.run(args.iters, probe=probe, eval_every=args.eval_every)
        m1 = probe.metrics(rec.ctx.theta)
        hist = res["history"]
        row = {"model": args.model, "K": args.k if topk else None, "init": name, "lambda_init": lam,
               "density_scales": bool(args.density_scales and lam is not None), "N": N, "init_ms": init_ms,
               "iters": hist[-1][0], "seconds": hist[-1][1], "psnr": [(h[0], h[3]) for h in hist],
               "start": {"psnr": m0[0], "ssim": m0[1], "ncc": m0[2]},
               "end": {"psnr": m1[0], "ssim": m1[1], "ncc": m1[2]}}
        print(json.dumps(row), flush=True)
        out.append(row)
        probe.close()
        rec.close()
    if args.out:
        json.dump(out, open(args.out, "w"), indent=1)


def run_densify(args):
    """Coarse-to-fine densification (the paper's future work, after 3D
    Gaussian Splatting) against the 0.8 mm grid start on the fetal workload,
    plain sum, both in growth mode (capacities follow the Gaussian count).
    "grid": 200,480 Gaussians on the 0.8 mm grid, scale 0.8 mm.  "coarse":
    Gaussians on a `h0`-mm grid with scale h0, then every `every` iterations
    until `stop` the fraction `frac` of Gaussians with the largest mean
    ||dL/dmu|| (the threshold is that quantile of the statistics) is split
    (largest scale above `split_mm`) or cloned, until the grid's count.  Both
    start from one flat amplitude (the mean observed brain intensity) times
    the plain sum's factor h^3 / ((2 pi)^(3/2) s^3).  Reported: the Gaussian
    count and PSNR every `eval_every` iterations, device seconds of the
    iterations and of the densifications (CUDA events), and PSNR / SSIM / NCC
    after `iters` iterations."""
    import torch
    from . import gsvr, inputs
    from .recon import PSNRProbe, Reconstruction
    torch.cuda.set_device(0)
    flat = inputs.fetal(args.seed, init="flat")
    N_grid = flat["N"]
    I, mask = flat["I"], flat["mask"]
    level = float(np.mean(I[mask > 0][I[mask > 0] > 0.2]))
    out = []
    for name in ("grid", "coarse"):
        case = dict(flat)
        if name == "coarse":
            g, N = inputs.grid_gaussians(flat["phantom"], h=args.h0, s=args.h0)
            g = g.reshape(11, N)
            g[10] = level / (2 * np.pi) ** 1.5
            case["N"] = N
            case["theta"] = np.concatenate([g.reshape(-1), flat["theta"][11 * N_grid:]]).astype(np.float32)
        rec = Reconstruction(case, n_sample=args.n_sample)
        probe = PSNRProbe(case["phantom"], case["N"])
        ctx = rec.ctx
        hist = [(0, 0.0, int(ctx.N), probe.psnr(ctx.theta, ctx.N))]
        dev_s = dens_s = 0.0
        events = []
        for it in range(1, args.iters + 1):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(rec.stream)
            rec.step()
            if name == "coarse":
                gsvr.gsvr_densify_accumulate(ctx.ctx)
            e1.record(rec.stream)
            events.append((e0, e1))
            if name == "coarse" and it % args.every == 0 and it <= args.stop and ctx.N < N_grid:
                for a, b in events:
                    b.synchronize()
                    dev_s += a.elapsed_time(b) / 1e3
                events = []
                acc, cnt = gsvr.gsvr_densify_stats(ctx.ctx, ctx.N)
                thr = float(np.quantile(acc[:, 0] / max(cnt, 1), 1.0 - args.frac))
                d0, d1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                d0.record(rec.stream)
                res = ctx.densify(thr, float(np.log(args.split_mm)), max_gaussians=N_grid)
                d1.record(rec.stream)
                d1.synchronize()
                dens_s += d0.elapsed_time(d1) / 1e3
                print(json.dumps({"iteration": it, "densify": res, "threshold": thr}), flush=True)
            if it % args.eval_every == 0:
                for a, b in events:
                    b.synchronize()
                    dev_s += a.elapsed_time(b) / 1e3
                events = []
                hist.append((it, dev_s, int(ctx.N), probe.psnr(ctx.theta, ctx.N)))
        m = probe.metrics(ctx.theta, ctx.N)
        row = {"start": name, "h0_mm": args.h0 if name == "coarse" else 0.8, "N_start": int(case["N"]),
               "N_end": int(ctx.N), "iters": args.iters, "seconds": dev_s, "densify_seconds": dens_s,
               "history": hist, "end": {"psnr": m[0], "ssim": m[1], "ncc": m[2]}}
        print(json.dumps(row), flush=True)
        out.append(row)
        probe.close()
        rec.close()
    if args.out:
        json.dump(out, open(args.out, "w"), indent=1)


def run_metrics_bench(args):
    """Device time of gsvr_volume_metrics on evaluation grids of the fetal
    phantom (0.8 mm and finer), with the float64 DFMA throughput it reaches
    (165 window DFMA per voxel) against the measured DFMA peak."""
    import torch
    from . import gsvr, inputs
    torch.cuda.set_device(0)
    peak = gsvr.gsvr_fp64_peak(0)
    ph = inputs.BrainPhantom(0)
    rows = []
    for h in args.h:
        st, ref, inside = inputs.grid_probe(ph, h)
        shape = (st["n_slices"], st["H"], st["W"])
        Y = torch.from_numpy(ref.reshape(shape)).cuda()
        X = (Y + 0.02 * torch.randn(shape, device="cuda", generator=torch.Generator("cuda").manual_seed(1))).float()
        msk = torch.from_numpy(inside.reshape(shape)).cuda()
        for _ in range(3):
            gsvr.gsvr_volume_metrics(X, Y, msk, 1.0)
        ts = []
        for _ in range(args.reps):
            t0 = time.perf_counter()
            res = gsvr.gsvr_volume_metrics(X, Y, msk, 1.0)
            ts.append(time.perf_counter() - t0)
        t = float(np.median(ts))
        V = int(np.prod(shape))
        row = {"h_mm": h, "shape": shape, "voxels": V, "ms": 1e3 * t, "psnr_ssim_ncc": res,
               "dfma_per_s": 165.0 * V / t, "dfma_peak": peak, "frac": 165.0 * V / t / peak}
        print(json.dumps(row), flush=True)
        rows.append(row)
    return rows


def run_topk_step(args):
    """A few plain top-K iterations (forward + backward) on the fetal workload's
    2^18-pixel sample: the command the top-K kernels are profiled with."""
    import torch
    from . import gsvr, inputs
    torch.cuda.set_device(0)
    ctx = gsvr.Context(inputs.fetal(0))
    gsvr.gsvr_sample_pixels(ctx.ctx, 1 << 18, 0)
    gsvr.gsvr_set_topk(ctx.ctx, args.k, args.delta, 1)
    for _ in range(args.steps):
        ctx.forward()
        ctx.backward()
    gsvr.gsvr_sync_status(ctx.ctx)
    print(json.dumps({"K": args.k, "loss": ctx.loss()}))
    ctx.close()


def run_posefit(args):
    """Train the pose network and report its pose errors against the nominal
    start on held-out rendered slices (phantom seeds disjoint from training) at
    the wide and the fetal motion ranges."""
    import torch
    from . import cnn
    torch.cuda.set_device(0)
    log = lambda m: print(m, flush=True)  # noqa: E731
    t0 = time.time()
    X, A, Y = cnn.make_training_set(args.phantoms, motions_per_phantom=args.motions, seed=args.seed,
                                    workers=args.workers, log=log)
    t_data = time.time() - t0
    net = cnn.PoseNet(max_batch=args.batch, seed=args.seed)
    hist = cnn.train(net, X, A, Y, epochs=args.epochs, batch=args.batch, lr=args.lr, seed=args.seed, log=log)
    out = {"training": {"slices": int(X.shape[0]), "phantoms": args.phantoms, "data_s": t_data, "epochs": hist},
           "held_out": {}}
    del X, A, Y
    for deg, mm in ((20.0, 10.0), (5.0, 3.0)):
        Xv, Av, Yv = cnn.make_training_set(args.eval_phantoms, motions_per_phantom=1, seed=args.seed + 1000,
                                           max_deg=deg, max_mm=mm, workers=args.workers)
        e = cnn.pose_errors_on_set(net, Xv, Av, Yv)
        out["held_out"]["%g deg / %g mm" % (deg, mm)] = {
            "slices": int(Xv.shape[0]), **{k: [float(np.mean(v)), float(np.median(v))] for k, v in e.items()}}
        log(json.dumps({k: out["held_out"]["%g deg / %g mm" % (deg, mm)][k] for k in e}))
    net.close()
    print(json.dumps(out))
    if args.out:
        with open(args.out, "w") as f:
            json.dump(out, f, indent=1)


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
    b.add_argument("--retire", action="store_true")
    b.add_argument("--out", default="")
    lr = sub.add_parser("learned")
    lr.add_argument("--phantoms", type=int, default=2000)
    lr.add_argument("--motions", type=int, default=2)
    lr.add_argument("--epochs", type=int, default=20)
    lr.add_argument("--batch", type=int, default=256)
    lr.add_argument("--lr", type=float, default=1e-3)
    lr.add_argument("--seed", type=int, default=0)
    lr.add_argument("--cases", type=int, default=10)
    lr.add_argument("--cases-c1", type=int, default=5)
    lr.add_argument("--iters", type=int, default=2000)
    lr.add_argument("--eval-every", type=int, default=50)
    lr.add_argument("--workers", type=int, default=8)
    lr.add_argument("--out", default="")
    pf = sub.add_parser("posefit")
    pf.add_argument("--phantoms", type=int, default=2000)
    pf.add_argument("--motions", type=int, default=2)
    pf.add_argument("--epochs", type=int, default=20)
    pf.add_argument("--batch", type=int, default=256)
    pf.add_argument("--lr", type=float, default=1e-3)
    pf.add_argument("--seed", type=int, default=0)
    pf.add_argument("--eval-phantoms", type=int, default=40)
    pf.add_argument("--workers", type=int, default=8)
    pf.add_argument("--out", default="")
    cb = sub.add_parser("cnnbench")
    cb.add_argument("--batch", type=int, default=256)
    cb.add_argument("--steps", type=int, default=50)
    cb.add_argument("--warmup", type=int, default=5)
    tk = sub.add_parser("topk")
    tk.add_argument("--k", type=int, nargs="+", default=[10, 20, 50, 80])
    tk.add_argument("--delta", type=float, default=1e-8)
    tk.add_argument("--refresh", type=int, default=1)
    tk.add_argument("--iters", type=int, default=600)
    tk.add_argument("--eval-every", type=int, default=100)
    tk.add_argument("--n-sample", type=int, default=1 << 18)
    tk.add_argument("--seed", type=int, default=0)
    tk.add_argument("--loss", choices=["mse", "l1"], default="mse")
    tk.add_argument("--lambda-reg", type=float, default=0.0)
    tk.add_argument("--s-target", type=float, default=0.8)
    tk.add_argument("--slice-weights", action="store_true")
    tk.add_argument("--out", default="")
    ts = sub.add_parser("topk-step")
    ts.add_argument("--k", type=int, default=50)
    ts.add_argument("--delta", type=float, default=1e-8)
    ts.add_argument("--steps", type=int, default=3)
    it = sub.add_parser("init")
    it.add_argument("--lambdas", type=float, nargs="+", default=[0.0, 0.5, 1.0])
    it.add_argument("--iters", type=int, default=600)
    it.add_argument("--eval-every", type=int, default=100)
    it.add_argument("--n-sample", type=int, default=1 << 18)
    it.add_argument("--seed", type=int, default=0)
    it.add_argument("--model", choices=["plain", "topk"], default="plain")
    it.add_argument("--k", type=int, default=50)
    it.add_argument("--density-scales", action="store_true")
    it.add_argument("--out", default="")
    dn = sub.add_parser("densify")
    dn.add_argument("--h0", type=float, default=2.4)
    dn.add_argument("--every", type=int, default=50)
    dn.add_argument("--stop", type=int, default=400)
    dn.add_argument("--frac", type=float, default=0.5)
    dn.add_argument("--split-mm", type=float, default=1.2)
    dn.add_argument("--iters", type=int, default=600)
    dn.add_argument("--eval-every", type=int, default=50)
    dn.add_argument("--n-sample", type=int, default=1 << 18)
    dn.add_argument("--seed", type=int, default=0)
    dn.add_argument("--out", default="")
    mb = sub.add_parser("metrics")
    mb.add_argument("--h", type=float, nargs="+", default=[0.8, 0.5, 0.4])
    mb.add_argument("--reps", type=int, default=10)
    args = ap.parse_args()
    if args.cmd == "init":
        run_init(args)
    elif args.cmd == "densify":
        run_densify(args)
    elif args.cmd == "metrics":
        run_metrics_bench(args)
    elif args.cmd == "topk":
        run_topk(args)
    elif args.cmd == "topk-step":
        run_topk_step(args)
    elif args.cmd == "cnnbench":
        run_cnnbench(args)
    elif args.cmd == "batched":
        run_batched(args)
    elif args.cmd == "learned":
        run_learned(args)
    elif args.cmd == "posefit":
        run_posefit(args)


if __name__ == "__main__":
    main()
