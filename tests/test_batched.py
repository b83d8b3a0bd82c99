"""Batched form: several subjects in one context (one set of launches) against
each subject alone and against the oracle; per-subject sampler against its
definition; CUDA-graph replay of whole iterations against eager iterations."""
import numpy as np
import pytest

from paper_2512_11624_b300 import inputs
from tests.gpu_util import CUTOFF, describe_grad, forward_ok, grad_ok

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2512_11624_b300 import gsvr
    return gsvr


def three_subjects():
    return [inputs.random_case(51, 120, [(3, 20, 24)], n_stacks=2, motion_deg=8.0),
            inputs.random_case(52, 300, [(2, 33, 29), (3, 17, 21)], n_stacks=3, motion_deg=8.0),
            inputs.random_case(53, 60, [(4, 16, 16)], n_stacks=1, motion_deg=8.0)]


def batched_ctx(G, cases, **cfg):
    b = inputs.concat_cases(cases)
    ctx = G.Context(b, **cfg)
    G.gsvr_set_subjects(ctx.ctx, b["stack_subject"], b["gauss_count"])
    return b, ctx


def test_batched_matches_alone_and_oracle(G, oracle):
    cases = three_subjects()
    b, ctx = batched_ctx(G, cases, tile_h=12, tile_w=12)
    ctx.forward()
    ctx.backward()
    G.gsvr_sync_status(ctx.ctx)
    pred = ctx.pred.cpu().numpy()
    grad = ctx.grad.cpu().numpy().astype(np.float64)
    losses = G.gsvr_get_subject_losses(ctx.ctx, len(cases))
    assert abs(ctx.loss() - losses.sum()) <= 1e-12 * abs(losses.sum())
    ctx.close()
    pix0 = 0
    pose0 = 11 * b["N"]
    for k, c in enumerate(cases):
        P = inputs.n_pixels_total(c["stacks"])
        M = inputs.n_slices_total(c["stacks"])
        alone = G.Context(c, tile_h=12, tile_w=12)
        alone.forward()
        alone.backward()
        a_pred = alone.pred.cpu().numpy()
        assert np.array_equal(pred[pix0:pix0 + P], a_pred)  # same records in the same order
        assert abs(losses[k] - alone.loss()) <= 1e-12 * alone.loss()
        alone.close()
        g_k = np.concatenate([inputs.subject_theta(grad, b["gauss_count"], k), grad[pose0:pose0 + 6 * M]])
        pix = np.arange(P)
        _, L, g, a, _, t = oracle.forward_backward(c["stacks"], c["theta"].astype(np.float64), c["N"], pix,
                                                   c["I"].astype(np.float64), 1.0 / P, cutoff=CUTOFF)
        ok, worst, _ = grad_ok(g_k, g, a, t)
        assert ok.all(), describe_grad(g_k, g, a, c["N"], M, t)
        pix0 += P
        pose0 += 6 * M


def test_subject_sampler_matches_definition(G, oracle):
    cases = three_subjects()
    rng = np.random.default_rng(5)
    for c in cases:
        c["mask"] = (rng.uniform(size=c["mask"].size) < 0.7).astype(np.uint8)
    b, ctx = batched_ctx(G, cases, seed=99)
    n = 200
    G.gsvr_sample_pixels_subjects(ctx.ctx, n, 4)
    got = np.sort(G.gsvr_get_sample(ctx.ctx))
    want = []
    base = 0
    for k, c in enumerate(cases):
        order = np.array(tile_order(c["stacks"], 16, 16)) + base
        masked = order[b["mask"][order] > 0]
        m = min(n, masked.size)
        pos = oracle.sample_positions(masked.size, m, (99 + k * 0x9E3779B97F4A7C15) % (1 << 64), 4)
        want.append(masked[pos])
        base += inputs.n_pixels_total(c["stacks"])
    assert np.array_equal(got, np.sort(np.concatenate(want)))
    ctx.close()


def tile_order(stacks, th, tw):
    out, base = [], 0
    for s in stacks:
        H, W = s["H"], s["W"]
        for _ in range(s["n_slices"]):
            for ty in range((H + th - 1) // th):
                for tx in range((W + tw - 1) // tw):
                    for a in range(ty * th, min(H, (ty + 1) * th)):
                        for bb in range(tx * tw, min(W, (tx + 1) * tw)):
                            out.append(base + a * W + bb)
            base += H * W
    return out


def test_graph_replay_matches_eager(G):
    import torch
    cases = three_subjects()
    lr = dict(lr_mu=5e-3, lr_ls=5e-3, lr_q=2e-3, lr_c=1e-3, lr_rot=2e-3, lr_trans=5e-2)
    runs = []
    for use_graph in (False, True):
        stream = torch.cuda.Stream()
        b, ctx = batched_ctx(G, cases, stream=stream.cuda_stream, fixed_capacity=1, cap_records=200000,
                             cap_keys=800000, seed=7)
        G.gsvr_set_frozen(ctx.ctx, np.array([1] + [0] * (ctx.M - 1), np.uint8))
        ctx.forward()
        G.gsvr_sync_status(ctx.ctx)
        if use_graph:
            G.gsvr_set_step(ctx.ctx, 0)
            G.gsvr_graph_capture(ctx.ctx, 150, lr=lr, step_every=3, gamma=0.5)
            G.gsvr_graph_launch(ctx.ctx, 7)
        else:
            for k in range(7):
                G.gsvr_sample_pixels_subjects(ctx.ctx, 150, k)
                ctx.forward()
                ctx.backward()
                G.gsvr_adam_step(ctx.ctx, k + 1, lr=lr, step_every=3, gamma=0.5)
        G.gsvr_sync_status(ctx.ctx)
        stream.synchronize()
        runs.append(ctx.theta.cpu().numpy().astype(np.float64))
        ctx.close()
    e, g = runs
    assert np.abs(e - g).max() <= 1e-4 * np.abs(e).max()


def test_batched_driver_graph_equals_eager_and_descends(G):
    from paper_2512_11624_b300.recon import BatchedReconstruction
    cases = three_subjects()
    runs = []
    for graph in (False, True):
        br = BatchedReconstruction(cases, n_sample=300, tune=False, graph=graph, lr=dict(lr_c=5e-3))
        res = br.run(40, eval_every=10)
        runs.append((br.ctx.theta.cpu().numpy().astype(np.float64), res["history"]))
        br.close()
    (te, he), (tg, hg) = runs
    assert np.abs(te - tg).max() <= 1e-4 * np.abs(te).max()
    first, last = np.array(he[1][2]), np.array(he[-1][2])
    assert np.all(last < first), (first, last)
    assert np.allclose(np.array(hg[-1][2]), last, rtol=1e-3)


def test_retired_subject_keeps_its_parameters(G):
    """gsvr_set_subject_active: a retired subject draws no pixels, its loss reads
    0 and its parameters (Gaussians and slice poses) stay bit for bit while the
    others keep moving, in eager and graph iterations; returned to the sample,
    it moves again; retiring every subject is refused."""
    import torch
    cases = three_subjects()
    lr = dict(lr_mu=5e-3, lr_ls=5e-3, lr_q=2e-3, lr_c=1e-3, lr_rot=2e-3, lr_trans=5e-2)
    stream = torch.cuda.Stream()
    b, ctx = batched_ctx(G, cases, stream=stream.cuda_stream, fixed_capacity=1, cap_records=200000,
                         cap_keys=800000, seed=7)
    gc = b["gauss_count"]
    M = [inputs.n_slices_total(c["stacks"]) for c in cases]
    P = [inputs.n_pixels_total(c["stacks"]) for c in cases]
    pose0 = 11 * b["N"] + 6 * M[0]

    def subject1():
        th = ctx.theta.cpu().numpy()
        return np.concatenate([inputs.subject_theta(th, gc, 1), th[pose0:pose0 + 6 * M[1]]])

    def step(k):
        G.gsvr_sample_pixels_subjects(ctx.ctx, 150, k)
        ctx.forward()
        ctx.backward()
        G.gsvr_adam_step(ctx.ctx, k + 1, lr=lr)

    for k in range(3):
        step(k)
    G.gsvr_set_subject_active(ctx.ctx, [1, 0, 1])
    before = subject1()
    others = ctx.theta.cpu().numpy().copy()
    for k in range(3, 6):
        step(k)
    G.gsvr_sync_status(ctx.ctx)
    assert np.array_equal(subject1(), before)
    sample = G.gsvr_get_sample(ctx.ctx)
    assert not np.any((sample >= P[0]) & (sample < P[0] + P[1]))
    assert np.sum(sample < P[0]) == 150 and np.sum(sample >= P[0] + P[1]) == 150
    losses = G.gsvr_get_subject_losses(ctx.ctx, 3)
    assert losses[1] == 0.0 and losses[0] > 0.0 and losses[2] > 0.0
    g0 = inputs.subject_theta(ctx.theta.cpu().numpy(), gc, 0)
    assert not np.array_equal(g0, inputs.subject_theta(others, gc, 0))
    # graph iterations with the subject retired
    ctx.forward()
    G.gsvr_sync_status(ctx.ctx)
    G.gsvr_set_step(ctx.ctx, 6)
    G.gsvr_graph_capture(ctx.ctx, 150, lr=lr)
    G.gsvr_graph_launch(ctx.ctx, 4)
    G.gsvr_sync_status(ctx.ctx)
    stream.synchronize()
    assert np.array_equal(subject1(), before)
    # back in the sample: it moves again
    G.gsvr_set_subject_active(ctx.ctx, None)
    for k in range(10, 13):
        step(k)
    G.gsvr_sync_status(ctx.ctx)
    assert not np.array_equal(subject1(), before)
    with pytest.raises(G.GsvrError):
        G.gsvr_set_subject_active(ctx.ctx, [0, 0, 0])
    ctx.close()


def test_batched_driver_retires_converged_subjects(G):
    """BatchedReconstruction.run with `retire`: every subject reaches its (easy) target, the
    retired ones stop moving, and the run ends once all have reached it."""
    from paper_2512_11624_b300.recon import BatchedReconstruction

    class LossProbe:  # "PSNR" read from the subject's own loss history
        def __init__(self, br, k):
            self.br, self.k = br, k
            self.n = 0

        def psnr(self, theta_g):
            self.n += 1
            return float(self.n)  # rises by one per evaluation

    cases = three_subjects()
    br = BatchedReconstruction(cases, n_sample=300, tune=False, graph=True, lr=dict(lr_c=5e-3))
    probes = [LossProbe(br, k) for k in range(3)]
    res = br.run(200, probes=probes, eval_every=10, targets=[2.0, 4.0, 3.0], retire=True)
    assert res["iters_to_target"] == [10, 30, 20]
    assert res["history"][-1][0] == 30  # stopped once every target was reached
    br.close()
