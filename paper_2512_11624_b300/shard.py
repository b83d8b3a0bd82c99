"""Data-parallel split of one reconstruction across ranks.

The loss of Sec. 2.5 is a sum over slice pixels, so one reconstruction splits
by slices: each rank owns a contiguous range of the global slice order (whole
stacks where that balances, else sub-stacks of contiguous slices), holds
every Gaussian (replicated) and the poses of its own slices.  One step:

  1. sample the rank's pixels; every rank weights its pixels by
     1 / (global sample size) (gsvr_set_sample_total), so its loss and
     gradient are its exact share of the global ones;
  2. forward and backward on the rank's slices (the library's kernels);
  3. one all-reduce (sum) of the contiguous 11 N Gaussian gradient and one of
     the scalar loss -- the only exchange the split needs; the pose gradients
     stay with the slices' owner;
  4. Adam on the rank's parameter vector: the Gaussian part sees the same
     reduced gradient on every rank, so the replicas stay identical.

The scale regulariser of the paper's loss acts on the replicated Gaussians,
so only rank 0 adds it.  The engine is a gsvr.Context on the rank's GPU by
default; any object with the same methods (``set_pixel_sample``,
``set_sample_total``, ``forward``, ``backward``, ``grad``, ``loss``,
``adam_step``, ``set_objective``) can stand in for it.
"""
import numpy as np

from . import inputs


def _pixel_counts(stacks):
    return np.array([int(s["H"]) * int(s["W"]) for s in stacks for _ in range(int(s["n_slices"]))], np.int64)


def split_slices(stacks, world, stack_tolerance=0.05):
    """Global slice boundaries [b_0 = 0, ..., b_world = M] of the ranks.  Each
    boundary is the stack boundary nearest the balanced pixel share when it is
    within `stack_tolerance` of the total pixel count of it, else the nearest
    slice boundary."""
    px = _pixel_counts(stacks)
    cum = np.concatenate([[0], np.cumsum(px)])
    total = int(cum[-1])
    stack_b = np.cumsum([0] + [int(s["n_slices"]) for s in stacks])
    bounds = [0]
    for r in range(1, world):
        target = r * total / world
        sb = stack_b[np.argmin(np.abs(cum[stack_b] - target))]
        if abs(cum[sb] - target) <= stack_tolerance * total:
            b = int(sb)
        else:
            b = int(np.argmin(np.abs(cum - target)))
        bounds.append(max(b, bounds[-1]))
    bounds.append(len(px))
    return bounds


def sub_stack(st, k0, k1):
    """Slices [k0, k1) of a stack as a stack of their own: slice k of a stack
    of n is centred at origin + (k - (n - 1)/2) thickness n_hat, so the
    sub-stack's origin moves by (k0 + (n' - 1)/2 - (n - 1)/2) thickness n_hat."""
    n, n2 = int(st["n_slices"]), k1 - k0
    R = np.asarray(st["R"], np.float64)
    shift = (k0 + 0.5 * (n2 - 1) - 0.5 * (n - 1)) * float(st["thickness"])
    out = dict(st)
    out["n_slices"] = n2
    out["origin"] = np.asarray(st["origin"], np.float64) + shift * R[:, 2]
    return out


def shard_case(case, rank, world, bounds=None):
    """The rank's part of a case dictionary: its sub-stacks, the observations
    and mask of its pixels, every Gaussian and its slices' poses; plus
    ``slice_range`` and ``pixel_range`` (global, half-open)."""
    stacks = case["stacks"]
    bounds = split_slices(stacks, world) if bounds is None else bounds
    s0, s1 = bounds[rank], bounds[rank + 1]
    px = _pixel_counts(stacks)
    cum = np.concatenate([[0], np.cumsum(px)])
    p0, p1 = int(cum[s0]), int(cum[s1])
    part_stacks, first = [], 0
    for st in stacks:
        n = int(st["n_slices"])
        lo, hi = max(s0 - first, 0), min(s1 - first, n)
        if lo < hi:
            part_stacks.append(st if (lo, hi) == (0, n) else sub_stack(st, lo, hi))
        first += n
    N = int(case["N"])
    th = np.asarray(case["theta"])
    theta = np.concatenate([th[:11 * N], th[11 * N + 6 * s0:11 * N + 6 * s1]]).astype(np.float32)
    out = {"name": case.get("name", "case") + "/rank%d" % rank, "N": N, "stacks": part_stacks, "theta": theta,
           "I": np.asarray(case["I"])[p0:p1], "mask": np.asarray(case["mask"])[p0:p1],
           "slice_range": (s0, s1), "pixel_range": (p0, p1)}
    if "n_sample" in case:
        out["n_sample"] = case["n_sample"]
    return out


class ContextEngine:
    """gsvr.Context of one rank's part (the GPU engine)."""

    def __init__(self, part, device=0, **cfg):
        from . import gsvr
        self.g = gsvr
        self.ctx = gsvr.Context(part, device=device, **cfg)

    def set_pixel_sample(self, idx):
        self.g.gsvr_set_pixel_sample(self.ctx.ctx, np.asarray(idx, np.int32))

    def set_sample_total(self, n):
        self.g.gsvr_set_sample_total(self.ctx.ctx, int(n))

    def set_objective(self, loss_kind, lambda_reg, s_target):
        self.g.gsvr_set_objective(self.ctx.ctx, loss_kind, lambda_reg, s_target)

    def forward(self):
        self.ctx.forward()

    def backward(self):
        self.ctx.backward()
        self.g.gsvr_sync_status(self.ctx.ctx)

    def grad(self):
        return self.ctx.grad

    def theta(self):
        return self.ctx.theta

    def loss(self):
        return self.ctx.loss()

    def adam_step(self, t, **kw):
        self.g.gsvr_adam_step(self.ctx.ctx, t, **kw)
        self.g.gsvr_sync_status(self.ctx.ctx)

    def close(self):
        self.ctx.close()


class ShardedReconstruction:
    """One reconstruction split by slices over the ranks of the default
    process group (or a single rank without one)."""

    def __init__(self, case, engine=None, bounds=None, **engine_kw):
        import torch.distributed as dist
        self.dist = dist if dist.is_available() and dist.is_initialized() else None
        self.rank = self.dist.get_rank() if self.dist else 0
        self.world = self.dist.get_world_size() if self.dist else 1
        self.N = int(case["N"])
        self.bounds = split_slices(case["stacks"], self.world) if bounds is None else bounds
        self.part = shard_case(case, self.rank, self.world, self.bounds)
        self.engine = engine(self.part) if engine else ContextEngine(self.part, **engine_kw)

    def set_objective(self, loss_kind=0, lambda_reg=0.0, s_target=1.6):
        """The paper's objective; the regulariser on the replicated Gaussians counts once (rank 0)."""
        self.engine.set_objective(loss_kind, lambda_reg if self.rank == 0 else 0.0, s_target)

    def local_indices(self, idx_global):
        """The rank's pixels of a global pixel list, as indices into its part."""
        p0, p1 = self.part["pixel_range"]
        idx = np.asarray(idx_global, np.int64)
        return (idx[(idx >= p0) & (idx < p1)] - p0).astype(np.int32)

    def _all_reduce(self, t):
        if self.dist is not None:
            self.dist.all_reduce(t)

    def gradient(self, idx_global):
        """Forward + backward over the global pixel list; returns the global
        loss.  Afterwards the engine's gradient holds the global Gaussian
        gradient and the poses' gradients of this rank's slices."""
        import torch
        self.engine.set_pixel_sample(self.local_indices(idx_global))
        self.engine.set_sample_total(len(idx_global))
        self.engine.forward()
        self.engine.backward()
        g = self.engine.grad()
        self._all_reduce(g[:11 * self.N])
        loss = torch.tensor([self.engine.loss()], dtype=torch.float64)
        self._all_reduce(loss)
        if g.is_cuda:
            torch.cuda.synchronize(g.device)
        return float(loss.item())

    def step(self, t, idx_global, **adam_kw):
        """One optimisation step (Adam step number t >= 1); returns the global loss."""
        loss = self.gradient(idx_global)
        self.engine.adam_step(t, **adam_kw)
        return loss

    def close(self):
        self.engine.close()
