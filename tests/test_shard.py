"""The data-parallel split of one reconstruction (paper_2512_11624_b300.shard)
on CPU: two gloo ranks (world size 2, 127.0.0.1) against one rank.  Each rank's
engine here is the float64 oracle over the rank's part (sub-stacks,
observations, replicated Gaussians, its poses), so what is checked is the
split itself: the sub-stack geometry, the 1 / (global sample) pixel weights,
the all-reduce of the loss and of the 11 N Gaussian gradient, the poses kept
by their owner, and Adam keeping the replicated Gaussians identical.
Checked for a split at stack boundaries and for one inside a stack."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

from paper_2512_11624_b300 import inputs, shard


class OracleEngine:
    """The engine interface of shard.ShardedReconstruction, computed by the
    float64 oracle (test stand-in for the GPU context)."""

    LR = np.array([2e-3, 2e-3, 1e-3, 2e-3, 1e-3, 1e-2])

    def __init__(self, part):
        from oracle import oracle
        self.o = oracle
        self.stacks = part["stacks"]
        self.N = int(part["N"])
        self.M = inputs.n_slices_total(self.stacks)
        self.theta = np.asarray(part["theta"], np.float64).copy()
        self.I = np.asarray(part["I"], np.float64)
        self.m = np.zeros_like(self.theta)
        self.v = np.zeros_like(self.theta)
        self.n_total = 0
        self.idx = None

    def set_pixel_sample(self, idx):
        self.idx = np.asarray(idx, np.int64)

    def set_sample_total(self, n):
        self.n_total = int(n)

    def set_objective(self, loss_kind, lambda_reg, s_target):
        self.obj = (loss_kind, lambda_reg, s_target)

    def forward(self):
        pass

    def backward(self):
        _, self._loss, g, _ = self.o.forward_backward(self.stacks, self.theta, self.N, self.idx, self.I[self.idx],
                                                     1.0 / self.n_total, want_abs=False)
        self._grad = torch.from_numpy(g)

    def grad(self):
        return self._grad

    def loss(self):
        return self._loss

    def adam_step(self, t, **kw):
        self.theta, self.m, self.v = self.o.adam(self.N, self.M, self.theta, self._grad.numpy(), self.m, self.v,
                                                 self.LR, 0.9, 0.999, 1e-8, t)

    def close(self):
        pass


def _case():
    return inputs.random_case(5, 80, [(3, 12, 10), (4, 9, 11), (2, 13, 12), (3, 10, 10)], n_stacks=4,
                              motion_deg=6.0, motion_mm=3.0)


def _samples(case):
    P = inputs.n_pixels_total(case["stacks"])
    rng = np.random.default_rng(2)
    return [np.sort(rng.choice(P, P // 2, replace=False)) for _ in range(2)]


def _run(case, bounds=None):
    rec = shard.ShardedReconstruction(case, engine=OracleEngine, bounds=bounds)
    out = {"loss": [], "grad0": None}
    for t, idx in enumerate(_samples(case), start=1):
        if t == 1:
            out["loss"].append(rec.gradient(idx))
            out["grad0"] = rec.engine.grad().numpy().copy()
            rec.engine.adam_step(t)
        else:
            out["loss"].append(rec.step(t, idx))
    out["theta"] = rec.engine.theta.copy()
    out["slice_range"] = rec.part["slice_range"]
    return out


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, port, bounds, out):
    os.environ.update({"WORLD_SIZE": "2", "RANK": str(rank), "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=2)
    try:
        out[rank] = _run(_case(), bounds)
    finally:
        dist.barrier()
        dist.destroy_process_group()


def test_split_geometry_matches_whole_stacks():
    """Sub-stacks put every slice where the whole stack puts it."""
    from oracle import oracle
    case = _case()
    M = inputs.n_slices_total(case["stacks"])
    R, t = oracle.slice_frames(case["stacks"], case["theta"][11 * case["N"]:])
    for bounds in ([0, 5, M], [0, 2, 7, 9, M], shard.split_slices(case["stacks"], 3)):
        for r in range(len(bounds) - 1):
            part = shard.shard_case(case, r, len(bounds) - 1, bounds)
            s0, s1 = part["slice_range"]
            Rp, tp = oracle.slice_frames(part["stacks"], part["theta"][11 * case["N"]:])
            assert np.allclose(Rp, R[s0:s1], atol=1e-14) and np.allclose(tp, t[s0:s1], atol=1e-12)
            p0, p1 = part["pixel_range"]
            assert p1 - p0 == inputs.n_pixels_total(part["stacks"])
    # pixels per stack 360, 396, 312, 300: the stack boundary nearest the half (756 of 1368) is 5.3 % off,
    # so the split falls inside the second stack at 5 % tolerance and on its end at 10 %
    assert shard.split_slices(case["stacks"], 2) == [0, 6, M]
    assert shard.split_slices(case["stacks"], 2, stack_tolerance=0.1) == [0, 7, M]


@pytest.mark.timeout(600)
@pytest.mark.parametrize("bounds", [None, [0, 5, 12]])
def test_two_gloo_ranks_equal_one_rank(bounds):
    single = _run(_case(), [0, 12])
    port = _free_port()
    with mp.Manager() as man:
        out = man.dict()
        mp.spawn(_worker, args=(port, bounds, out), nprocs=2, join=True)
        res = dict(out)
    N = _case()["N"]
    for r in (0, 1):
        # global loss and global Gaussian gradient on every rank
        assert np.allclose(res[r]["loss"], single["loss"], rtol=1e-12, atol=0)
        assert np.allclose(res[r]["grad0"][:11 * N], single["grad0"][:11 * N], rtol=1e-10,
                           atol=1e-13 * np.abs(single["grad0"]).max())
        # the poses of the rank's own slices
        s0, s1 = res[r]["slice_range"]
        assert np.allclose(res[r]["grad0"][11 * N:], single["grad0"][11 * N + 6 * s0:11 * N + 6 * s1], rtol=1e-12,
                           atol=1e-15)
        assert np.allclose(res[r]["theta"][11 * N:], single["theta"][11 * N + 6 * s0:11 * N + 6 * s1], rtol=1e-9,
                           atol=1e-12)
        assert np.allclose(res[r]["theta"][:11 * N], single["theta"][:11 * N], rtol=1e-9, atol=1e-12)
    # the replicated Gaussians stay bitwise identical across the ranks
    assert np.array_equal(res[0]["theta"][:11 * N], res[1]["theta"][:11 * N])
    assert res[0]["slice_range"][1] == res[1]["slice_range"][0]
