"""The normalised top-K forward model on the GPU (through the C ABI,
gsvr_set_topk) against the float64 oracle of ``oracle/topk.py``.

- Forward values within 1e-5 relative (floored at 1e-3 of the case maximum),
  gradients within 1e-4 relative plus 1e-6 of the sum of |pair terms|, as on
  the plain path; cases with K below, at and above N, a lone Gaussian, two
  oblique stacks with motion, K = 64 and 128 (the forward's 64-thread blocks).
- The neighbour sets are unique except at distance ties (lattice-placed
  Gaussians tie often), so the GPU's sets are read back and checked to be valid
  K-nearest sets (no left-out mean nearer than an included one, beyond float32
  distance rounding), and the oracle is evaluated on exactly those sets.
- Partition of unity (equal amplitudes give exactly that amplitude, up to
  delta), K = 0 restoring the plain sum bit for bit, argument checks, a CUDA
  graph of whole iterations against the same iterations run eagerly, and the
  fetal workload (200,480 Gaussians, K = 50) on sampled pixels against the
  oracle's brute-force neighbours.
"""
import numpy as np
import pytest

from paper_2512_11624_b300 import inputs
from tests.gpu_util import describe_grad, forward_ok, grad_ok

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2512_11624_b300 import gsvr
    return gsvr


@pytest.fixture(scope="module")
def topk():
    from oracle import topk as t
    return t


def valid_sets(topk, case, pix, nbr, cnt, K, rel=1e-5):
    """Every set holds min(K, N) distinct means and no left-out mean is nearer
    than the farthest included one by more than float32 distance rounding."""
    th = case["theta"].astype(np.float64)
    N = case["N"]
    x, _, _, _, _ = topk.pixel_geometry(case["stacks"], th, N, pix)
    mu = topk.means(th, N)
    kk = min(K, N)
    for n in range(len(pix)):
        assert cnt[n] == kk
        s_ = nbr[n, :kk]
        assert len(np.unique(s_)) == kk and s_.min() >= 0 and s_.max() < N
        d2 = ((x[n] - mu) ** 2).sum(1)
        if kk < N:
            out = np.ones(N, bool)
            out[s_] = False
            assert d2[s_].max() <= d2[out].min() * (1 + rel) + 1e-12, n


def run(G, case, K, delta, sample=None, refresh=1):
    ctx = G.Context(case)
    if sample is not None:
        G.gsvr_set_pixel_sample(ctx.ctx, np.asarray(sample, np.int32))
    G.gsvr_set_topk(ctx.ctx, K, delta, refresh)
    ctx.forward()
    pix, nbr, cnt = G.gsvr_get_topk_neighbors(ctx.ctx, K)
    ctx.backward()
    G.gsvr_sync_status(ctx.ctx)
    out = dict(pred=ctx.pred.cpu().numpy().astype(np.float64), grad=ctx.grad.cpu().numpy().astype(np.float64),
               loss=ctx.loss(), pix=pix.astype(np.int64), nbr=nbr.astype(np.int64), cnt=cnt)
    ctx.close()
    return out


@pytest.mark.parametrize("seed,N,sizes,n_stacks,K,delta", [
    (21, 60, [(2, 12, 10)], 2, 8, 1e-3),
    (22, 400, [(3, 20, 24)], 2, 50, 1e-6),
    (23, 30, [(2, 9, 7)], 1, 50, 1e-2),
    (24, 1, [(1, 6, 5)], 1, 1, 1e-2),
    (25, 200, [(2, 16, 16), (3, 11, 13)], 2, 64, 1e-4),
    (31, 300, [(2, 15, 14)], 2, 128, 1e-4),
])
def test_matches_oracle(G, topk, seed, N, sizes, n_stacks, K, delta):
    case = inputs.random_case(seed, N, sizes, n_stacks=n_stacks, extent=4.0, motion_deg=8.0)
    gpu = run(G, case, K, delta)
    pix, kk = gpu["pix"], min(K, N)
    assert len(pix) == inputs.n_pixels_total(case["stacks"])
    valid_sets(topk, case, pix, gpu["nbr"], gpu["cnt"], K)
    th = case["theta"].astype(np.float64)
    I = case["I"].astype(np.float64)[pix]
    w = 1.0 / len(pix)
    pred, loss, g, _, A = topk.forward_backward(case["stacks"], th, N, pix, I, w, kk, delta,
                                                nbr=gpu["nbr"][:, :kk], want_abs=True)
    ok, worst = forward_ok(gpu["pred"][pix], pred)
    assert ok.all(), ("forward", (~ok).sum(), worst)
    assert abs(gpu["loss"] - loss) <= 1e-4 * loss + 1e-12, (gpu["loss"], loss)
    gok, gworst, plain = grad_ok(gpu["grad"], g, A)
    M = inputs.n_slices_total(case["stacks"])
    info = describe_grad(gpu["grad"], g, A, N, M)
    print("K=%d: fwd worst %.3g, grad worst %.3g (plain 1e-4 pass %.4f) %s" % (K, worst, gworst, plain, info))
    assert gok.all(), ("gradient", (~gok).sum(), gworst, info)


def test_partition_of_unity(G):
    case = inputs.random_case(26, 150, [(2, 14, 12)], n_stacks=2, extent=4.0)
    case["theta"][10 * case["N"]:11 * case["N"]] = 2.5
    gpu = run(G, case, 20, 1e-30)
    pix = np.arange(inputs.n_pixels_total(case["stacks"]))
    assert np.allclose(gpu["pred"][pix], 2.5, rtol=2e-6, atol=0)


def test_k_zero_restores_plain_sum(G):
    case = inputs.random_case(27, 120, [(2, 13, 15)], n_stacks=2, extent=4.0)
    ctx = G.Context(case)
    ctx.forward()
    plain = ctx.pred.cpu().numpy().copy()
    G.gsvr_set_topk(ctx.ctx, 10, 1e-3, 1)
    ctx.forward()
    ratio = ctx.pred.cpu().numpy().copy()
    G.gsvr_set_topk(ctx.ctx, 0, 1e-3, 1)
    ctx.forward()
    again = ctx.pred.cpu().numpy().copy()
    ctx.close()
    assert not np.array_equal(plain, ratio)
    assert np.array_equal(plain, again)


def test_argument_checks(G):
    case = inputs.random_case(28, 10, [(1, 6, 6)], n_stacks=1)
    ctx = G.Context(case)
    for K, d, r in [(129, 1e-3, 1), (-1, 1e-3, 1), (5, 0.0, 1), (5, float("nan"), 1), (5, 1e-3, 0)]:
        with pytest.raises(G.GsvrError) as e:
            G.gsvr_set_topk(ctx.ctx, K, d, r)
        assert "INVALID_ARG" in str(e.value)
    ctx.close()


def test_stale_grid_refresh(G):
    """refresh_every > 1: the first forward builds the grid, so it equals the
    refresh-every-forward result bit for bit."""
    case = inputs.random_case(29, 200, [(2, 12, 12)], n_stacks=2, extent=4.0)
    a = run(G, case, 12, 1e-3, refresh=5)
    b = run(G, case, 12, 1e-3, refresh=1)
    assert np.array_equal(a["pred"], b["pred"])


def test_graph_replay_matches_eager(G):
    """Whole iterations (sample, top-K forward, backward, Adam) captured in a
    CUDA graph and replayed give the parameters of the same iterations run
    eagerly (float32 atomics make the two differ in the last bits)."""
    import torch
    case = inputs.random_case(30, 150, [(2, 12, 12)], n_stacks=2, extent=4.0)
    lr = dict(lr_mu=5e-3, lr_ls=5e-3, lr_q=2e-3, lr_c=1e-3, lr_rot=2e-3, lr_trans=5e-2)
    runs = []
    for use_graph in (False, True):
        stream = torch.cuda.Stream()
        ctx = G.Context(case, stream=stream.cuda_stream, fixed_capacity=1, cap_records=200000, cap_keys=800000,
                        seed=7)
        G.gsvr_set_topk(ctx.ctx, 16, 1e-3, 1)
        if use_graph:
            G.gsvr_set_step(ctx.ctx, 0)
            G.gsvr_graph_capture(ctx.ctx, 120, lr=lr)
            G.gsvr_graph_launch(ctx.ctx, 5)
        else:
            for k in range(5):
                G.gsvr_sample_pixels(ctx.ctx, 120, k)
                ctx.forward()
                ctx.backward()
                G.gsvr_adam_step(ctx.ctx, k + 1, lr=lr)
        G.gsvr_sync_status(ctx.ctx)
        stream.synchronize()
        runs.append(ctx.theta.cpu().numpy().astype(np.float64))
        ctx.close()
    e, g = runs
    assert not np.array_equal(e, case["theta"].astype(np.float64))
    assert np.abs(e - g).max() <= 1e-4 * np.abs(e).max()


def test_fetal_sampled_pixels(G, topk):
    """The fetal workload (Gaussians on a 0.8 mm lattice: many distance ties)
    with K = 50 on 2^18 sampled pixels: 400 of them checked for valid sets and
    against the oracle on those sets."""
    case = inputs.fetal(0)
    N = case["N"]
    ctx = G.Context(case)
    G.gsvr_sample_pixels(ctx.ctx, 1 << 18, 0)
    G.gsvr_set_topk(ctx.ctx, 50, 1e-8, 1)
    ctx.forward()
    G.gsvr_sync_status(ctx.ctx)
    pix, nbr, cnt = G.gsvr_get_topk_neighbors(ctx.ctx, 50)
    pred = ctx.pred.cpu().numpy().astype(np.float64)
    ctx.close()
    assert len(pix) == 1 << 18
    rng = np.random.default_rng(0)
    pick = np.sort(rng.choice(len(pix), 400, replace=False))
    p = pix[pick].astype(np.int64)
    valid_sets(topk, case, p, nbr[pick], cnt[pick], 50)
    th = case["theta"].astype(np.float64)
    ref, _, _ = topk.forward(case["stacks"], th, N, p, 50, 1e-8, nbr=nbr[pick].astype(np.int64))
    ok, worst = forward_ok(pred[p], ref)
    print("fetal top-K: worst %.3g of the tolerance" % worst)
    assert ok.all(), ((~ok).sum(), worst)
