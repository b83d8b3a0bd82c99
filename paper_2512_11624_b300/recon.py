"""Reconstruction driver over the library: the joint optimisation of Gaussians
and slice poses (Sec. 2.4 / App. A.1: Adam with per-group learning rates) on
sampled pixels, with PSNR against a reference volume and time to a PSNR target.

`PSNRProbe` reads the Gaussian volume V(x) on an isotropic grid through the
same forward (a stack of grid "slices" with a zero-width PSF reads V itself) and
returns PSNR = -10 log10(MSE) for intensities in [0, 1]; `PSNRProbe.metrics`
reads V at every grid point and returns PSNR, SSIM and NCC over the phantom's
voxels (gsvr_volume_metrics, data range 1).  Iteration time counts
device time of the optimisation steps only (CUDA events around each block of
iterations); evaluations run outside it.
"""
from __future__ import annotations

import numpy as np
import torch

from . import gsvr, inputs


class PSNRProbe:
    """`topk` = (K, delta): read the normalised top-K volume of Eq. 2 instead of
    the plain sum."""

    def __init__(self, phantom, N, device=0, h=0.8, stream=None, topk=None):
        st, ref, inside = inputs.grid_probe(phantom, h)
        self.N = int(N)
        case = {"stacks": [st], "N": self.N, "theta": np.zeros(11 * self.N + 6 * st["n_slices"], np.float32),
                "I": ref, "mask": inside}
        self.ctx = gsvr.Context(case, device=device, stream=stream, tile_h=16, tile_w=16)
        if topk:
            gsvr.gsvr_set_topk(self.ctx.ctx, int(topk[0]), float(topk[1]), 1)
        self.n_points = int(inside.sum())
        self.shape = (st["n_slices"], st["H"], st["W"])
        self._grid_case = dict(case, mask=np.ones_like(inside))
        self._device, self._stream, self._topk = device, stream, topk
        self._full = None
        self._ref = torch.from_numpy(ref.reshape(self.shape)).to("cuda:%d" % device)
        self._inside = torch.from_numpy(inside.reshape(self.shape)).to("cuda:%d" % device)

    def _resize(self, N):
        """Follow a new Gaussian count (after a densification)."""
        N = int(N)
        if N == self.N:
            return
        self.N = N
        zeros = np.zeros(11 * N, np.float32)
        self.ctx.set_gaussians(zeros, N)
        if self._full is not None:
            self._full.set_gaussians(zeros, N)

    def metrics(self, theta_g, N=None):
        """(PSNR, SSIM, NCC) of the volume read at every grid point against the
        phantom, over the phantom's voxels."""
        if N is not None:
            self._resize(N)
        if self._full is None:
            M = int(self._grid_case["stacks"][0]["n_slices"])
            grid = dict(self._grid_case, N=self.N, theta=np.zeros(11 * self.N + 6 * M, np.float32))
            self._full = gsvr.Context(grid, device=self._device, stream=self._stream, tile_h=16, tile_w=16)
            if self._topk:
                gsvr.gsvr_set_topk(self._full.ctx, int(self._topk[0]), float(self._topk[1]), 1)
        self._full.theta[:11 * self.N].copy_(theta_g[:11 * self.N])
        gsvr.gsvr_forward(self._full.ctx)
        gsvr.gsvr_sync_status(self._full.ctx)
        X = self._full.pred.view(self.shape)
        return gsvr.gsvr_volume_metrics(X, self._ref, self._inside, 1.0,
                                        stream=self._stream)

    def psnr(self, theta_g, N=None):
        """theta_g: the first 11 N entries of a parameter vector (CUDA tensor);
        N: its Gaussian count when it changed since the probe was made."""
        if N is not None:
            self._resize(N)
        self.ctx.theta[:11 * self.N].copy_(theta_g[:11 * self.N])
        gsvr.gsvr_forward(self.ctx.ctx)
        mse = self.ctx.loss()
        return float(-10.0 * np.log10(max(mse, 1e-30)))

    def close(self):
        self.ctx.close()
        if self._full is not None:
            self._full.close()


# Learning rates per Adam step on 2^18-pixel mini-batches.  Pose rates are the
# paper's (App. A.1: rotation 2.5e-3, translation 1e-1); the Gaussian rates are
# the paper's x 0.1 for mu, s, q, and for c also x h^3 / ((2 pi)^(3/2) s^3)
# (= 0.0635 on the 0.8 mm grid): the paper's c is the O(1) colour of the
# normalised sum of Eq. 2, the plain sum's amplitude is that colour times this
# factor.  With StepLR x 0.5 every 200 steps the phantom PSNR rises
# monotonically over 2000 steps (a sweep of rates is in the design notes).
PLAIN_LR = dict(lr_mu=2.5e-3, lr_ls=2.5e-3, lr_q=1e-3, lr_c=2e-3 * 0.0635, lr_rot=2.5e-3, lr_trans=1e-1)
PLAIN_STEP_EVERY = 200


# A short list of launch shapes for per-reconstruction tuning (the library's
# full space is gsvr.gsvr_tune_space_default()).
TUNE_SHAPES = [gsvr.tiling(12, 12), gsvr.tiling(8, 16), gsvr.tiling(16, 16), gsvr.tiling(10, 10),
               gsvr.tiling(12, 12, queue_order=1), gsvr.tiling(8, 8)]


def make_context(case, device, stream, n_sample=None, subjects=None, tune=False, margin=2.0, shapes=None):
    """A fixed-capacity context (no host synchronisation per iteration) for
    `case`: record / key counts from one growth-mode forward on a sample,
    capacities `margin` times those, launch shape from the autotuner when
    `tune` (timed on the same sample size).  `subjects` = (stack_subject,
    gauss_count) for a batched case.  Returns (context, launch shape)."""
    def setup(ctx):
        if subjects is not None:
            gsvr.gsvr_set_subjects(ctx.ctx, subjects[0], subjects[1])

    def sample(ctx, step):
        if n_sample:
            if subjects is not None:
                gsvr.gsvr_sample_pixels_subjects(ctx.ctx, n_sample, step)
            else:
                gsvr.gsvr_sample_pixels(ctx.ctx, min(n_sample, int(case["mask"].sum())), step)

    sid = stream.cuda_stream
    probe = gsvr.Context(case, device=device, stream=sid, tile_h=12, tile_w=12)
    setup(probe)
    sample(probe, 0)
    probe.forward()
    st = probe.stats()
    shape = gsvr.gsvr_get_tiling(probe.ctx)
    if tune:
        gsvr.gsvr_reserve(probe.ctx, int(st["n_records"] * margin) + 4096, int(st["n_keys"] * 2 * margin) + 4096)
        best, res = gsvr.gsvr_autotune(probe.ctx, shapes or TUNE_SHAPES, n_per_subject=n_sample or 0, iterations=5)
        shape = res[best]
        sample(probe, 0)
        probe.forward()
        st = probe.stats()
    probe.close()
    ctx = gsvr.Context(case, device=device, stream=sid, tile_h=shape.tile_h, tile_w=shape.tile_w, fixed_capacity=1,
                       cap_records=int(st["n_records"] * margin) + 4096, cap_keys=int(st["n_keys"] * margin) + 4096)
    gsvr.gsvr_set_tiling(ctx.ctx, shape)
    setup(ctx)
    return ctx, shape


def ensure_room(ctx, fill=0.75, grow=1.5):
    """Grow a fixed-capacity context when the last forward used more than
    `fill` of its record or key capacity.  Returns True when it grew."""
    st = ctx.stats()
    if st["n_records"] > fill * st["cap_records"] or st["n_keys"] > fill * st["cap_keys"]:
        gsvr.gsvr_reserve(ctx.ctx, int(max(st["n_records"], 1) * grow / fill), int(max(st["n_keys"], 1) * grow / fill))
        return True
    return False


class Reconstruction:
    """One subject: gsvr context + Adam state; `step` = sample, forward,
    backward, Adam.  `fixed` builds a fixed-capacity context (see make_context),
    `tune` lets the autotuner pick its launch shape, `topk` = (K, delta,
    refresh_every) switches to the normalised top-K model (gsvr_set_topk)."""

    def __init__(self, case, device=0, stream=None, n_sample=None, lr=None, frozen=None,
                 step_every=PLAIN_STEP_EVERY, gamma=0.5, fixed=False, tune=False, topk=None, **cfg):
        self.stream = stream if stream is not None else torch.cuda.Stream(device=device)
        if fixed or tune:
            self.ctx, self.shape = make_context(case, device, self.stream, n_sample, tune=tune)
        else:
            self.ctx = gsvr.Context(case, device=device, stream=self.stream.cuda_stream, **cfg)
            self.shape = gsvr.gsvr_get_tiling(self.ctx.ctx)
        self.fixed = fixed or tune
        if topk:
            gsvr.gsvr_set_topk(self.ctx.ctx, int(topk[0]), float(topk[1]), int(topk[2]) if len(topk) > 2 else 1)
        self.N = int(case["N"])
        self.n_sample = min(int(n_sample), int(np.count_nonzero(case["mask"]))) if n_sample else n_sample
        self.lr = dict(PLAIN_LR, **(lr or {}))
        self.step_every = step_every  # StepLR: learning rates x gamma every step_every iterations (App. A.1)
        self.gamma = gamma
        M = self.ctx.M
        if frozen is None and case.get("ref_slice") is not None:
            frozen = [case["ref_slice"]]
        if frozen:
            f = np.zeros(M, np.uint8)
            f[list(frozen)] = 1
            gsvr.gsvr_set_frozen(self.ctx.ctx, f)
        self.t = 0

    def step(self):
        if self.n_sample:
            gsvr.gsvr_sample_pixels(self.ctx.ctx, self.n_sample, self.t)
        gsvr.gsvr_forward(self.ctx.ctx)
        gsvr.gsvr_backward(self.ctx.ctx)
        self.t += 1
        gsvr.gsvr_adam_step(self.ctx.ctx, self.t, self.lr, step_every=self.step_every or 0, gamma=self.gamma)

    def run(self, iters, probe=None, eval_every=25, target_psnr=None):
        """Returns {"history": [(iteration, device_seconds, loss, psnr)], "time_to_target": s or None}."""
        hist = []
        dev_s = 0.0
        t_hit = None
        if probe is not None:
            hist.append((0, 0.0, None, probe.psnr(self.ctx.theta, self.ctx.N)))
        done = 0
        while done < iters:
            n = min(eval_every, iters - done)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(self.stream)
            for _ in range(n):
                self.step()
            e1.record(self.stream)
            e1.synchronize()
            dev_s += e0.elapsed_time(e1) / 1e3
            done += n
            if self.fixed:
                gsvr.gsvr_sync_status(self.ctx.ctx)
                ensure_room(self.ctx)
            loss = self.ctx.loss()
            p = probe.psnr(self.ctx.theta, self.ctx.N) if probe is not None else None
            hist.append((done, dev_s, loss, p))
            if t_hit is None and target_psnr is not None and p is not None and p >= target_psnr:
                t_hit = dev_s
        gsvr.gsvr_sync_status(self.ctx.ctx)
        return {"history": hist, "time_to_target": t_hit}

    def close(self):
        self.ctx.close()


class BatchedReconstruction:
    """Several subjects in one context (the batched form): one set of launches
    per iteration serves every subject -- per-subject samplers, loss weights,
    losses and Adam bias corrections, Gaussians meeting only their subject's
    slices -- and the whole iteration (sample, forward, backward, Adam with
    StepLR, step counter) is one CUDA graph replayed `n` times per `advance`.
    Subject k's reference slice is frozen."""

    def __init__(self, cases, device=0, n_sample=1 << 18, lr=None, step_every=PLAIN_STEP_EVERY, gamma=0.5,
                 tune=True, graph=True, margin=2.0):
        self.cases = cases
        self.b = inputs.concat_cases(cases)
        self.n_subj = len(cases)
        self.stream = torch.cuda.Stream(device=device)
        self.n_sample = n_sample
        self.lr = dict(PLAIN_LR, **(lr or {}))
        self.step_every, self.gamma = step_every, gamma
        self.ctx, self.shape = make_context(self.b, device, self.stream, n_sample,
                                            subjects=(self.b["stack_subject"], self.b["gauss_count"]), tune=tune,
                                            margin=margin)
        M = self.ctx.M
        f = np.zeros(M, np.uint8)
        base = 0
        self.slice_first = []
        for c in cases:
            self.slice_first.append(base)
            if c.get("ref_slice") is not None:
                f[base + int(c["ref_slice"])] = 1
            base += inputs.n_slices_total(c["stacks"])
        gsvr.gsvr_set_frozen(self.ctx.ctx, f)
        self.graph = graph
        self.t = 0
        gsvr.gsvr_set_step(self.ctx.ctx, 0)
        if graph:
            self._capture()
        g = np.concatenate([[0], np.cumsum(self.b["gauss_count"])]).astype(np.int64)
        N = int(g[-1])
        dev = self.ctx.theta.device
        self.gauss_index = [torch.from_numpy(np.concatenate([c * N + np.arange(g[k], g[k + 1]) for c in range(11)]))
                            .to(dev) for k in range(self.n_subj)]

    def _capture(self):
        # the capture needs a forward at the current capacities first
        gsvr.gsvr_sample_pixels_subjects(self.ctx.ctx, self.n_sample, self.t)
        gsvr.gsvr_forward(self.ctx.ctx)
        gsvr.gsvr_sync_status(self.ctx.ctx)
        gsvr.gsvr_set_step(self.ctx.ctx, self.t)
        gsvr.gsvr_graph_capture(self.ctx.ctx, self.n_sample, lr=self.lr, step_every=self.step_every or 0,
                                gamma=self.gamma)

    def advance(self, n):
        if self.graph:
            gsvr.gsvr_graph_launch(self.ctx.ctx, n)
        else:
            for _ in range(n):
                gsvr.gsvr_sample_pixels_subjects(self.ctx.ctx, self.n_sample, self.t)
                gsvr.gsvr_forward(self.ctx.ctx)
                gsvr.gsvr_backward(self.ctx.ctx)
                self.t += 1
                gsvr.gsvr_adam_step(self.ctx.ctx, self.t, self.lr, step_every=self.step_every or 0, gamma=self.gamma)
            return
        self.t += n

    def subject_theta(self, k):
        return self.ctx.theta.index_select(0, self.gauss_index[k])

    def run(self, iters, probes=None, eval_every=25, targets=None, retire=False):
        """Returns {"history": [(iteration, device_seconds, [loss per subject], [psnr per subject])],
        "time_to_target": [s or None per subject], "iters_to_target": [...]}.  With
        `retire`, a subject that reaches its target leaves the batch
        (gsvr_set_subject_active: no more pixels, parameters kept) and the run
        ends once every subject has reached its target."""
        hist = []
        dev_s = 0.0
        hit_t = [None] * self.n_subj
        hit_i = [None] * self.n_subj
        active = np.ones(self.n_subj, np.uint8)

        def evaluate():
            return [p.psnr(self.subject_theta(k)) for k, p in enumerate(probes)] if probes else None

        hist.append((0, 0.0, None, evaluate()))
        done = 0
        while done < iters:
            n = min(eval_every, iters - done)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(self.stream)
            self.advance(n)
            e1.record(self.stream)
            e1.synchronize()
            dev_s += e0.elapsed_time(e1) / 1e3
            done += n
            gsvr.gsvr_sync_status(self.ctx.ctx)
            if ensure_room(self.ctx) and self.graph:
                self._capture()
            losses = gsvr.gsvr_get_subject_losses(self.ctx.ctx, self.n_subj).tolist()
            ps = evaluate()
            hist.append((done, dev_s, losses, ps))
            if targets is not None and ps is not None:
                for k in range(self.n_subj):
                    if hit_t[k] is None and targets[k] is not None and ps[k] >= targets[k]:
                        hit_t[k], hit_i[k] = dev_s, done
                if retire:
                    if all(h is not None for h in hit_t):
                        break
                    newly = [k for k in range(self.n_subj) if hit_t[k] is not None and active[k]]
                    if newly:
                        active[newly] = 0
                        gsvr.gsvr_set_subject_active(self.ctx.ctx, active)
                        if self.graph:
                            self._capture()
        return {"history": hist, "time_to_target": hit_t, "iters_to_target": hit_i}

    def close(self):
        self.ctx.close()
