"""Densification on the GPU (gsvr_densify_accumulate / gsvr_densify_stats /
gsvr_densify: split, clone, prune) against the oracle of oracle/densify.py.

Decisions are float32 comparisons both sides take identically, so the kinds,
the new count and the output layout (which parent fills which slot) must
match exactly; kept Gaussians, their Adam moments and the slice poses are
copies (bit-exact); children are float32 arithmetic against the oracle's
float64 (means within 2e-6 (|mu| + step) + 1e-7 mm, log-scales within 1e-6,
amplitudes within 1e-6 relative, moments exactly 0).  The statistics step is
bit-exact against the oracle's float32 accumulation of the same gradients.
After a densification the forward model runs on the new Gaussians and matches
the plain-sum oracle on the oracle's own densified parameters."""
import numpy as np
import pytest

from paper_2512_11624_b300 import inputs
from gpu_util import forward_ok

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2512_11624_b300 import gsvr
    return gsvr


@pytest.fixture(scope="module")
def dens():
    from oracle import densify
    return densify


def small_case(seed=61, N=400):
    case = inputs.random_case(seed, N, [(3, 14, 17), (2, 12, 13)], n_stacks=2, motion_deg=6.0)
    th = case["theta"].copy()
    rng = np.random.default_rng(seed)
    th[3 * N:6 * N] = rng.uniform(-1.2, 0.6, 3 * N)  # scales 0.3 .. 1.8 mm
    th[10 * N:10 * N + 7] = 1e-5  # prunable amplitudes
    case["theta"] = th
    return case


def moments(seed, n):
    rng = np.random.default_rng(seed)
    return rng.normal(0, 1, n).astype(np.float32), rng.uniform(0, 1, n).astype(np.float32)


def run_densify(G, dens, case, acc, count, cfg, m=None, v=None):
    import torch
    N, M = case["N"], inputs.n_slices_total(case["stacks"])
    ctx = G.Context(case)
    if m is not None:
        ctx.adam_m.copy_(torch.from_numpy(m))
        ctx.adam_v.copy_(torch.from_numpy(v))
    G.gsvr_densify_stats(ctx.ctx, N, acc, count)
    out = ctx.densify(**cfg)
    got = (ctx.theta.cpu().numpy(), ctx.adam_m.cpu().numpy(), ctx.adam_v.cpu().numpy())
    z = np.zeros_like(case["theta"]) if m is None else None
    ref = dens.densify(case["theta"], m if m is not None else z, v if v is not None else z, N, M, acc, count,
                       cfg["grad_threshold"], cfg["log_scale_threshold"], cfg.get("prune_amplitude", 0.0),
                       cfg.get("split_factor", 1.6), cfg.get("clone_offset", 0.5), cfg.get("mass_preserving", 1))
    return ctx, out, got, ref


def check_layout(case, out, got, ref, dens, m, v):
    N, M = case["N"], inputs.n_slices_total(case["stacks"])
    th2, m2, v2, N2, kind, parent = ref
    assert out == (N2, int((kind == dens.SPLIT).sum()), int((kind == dens.CLONE).sum()),
                   int((kind == dens.PRUNE).sum()))
    gt, gm, gv = got
    assert gt.size == 11 * N2 + 6 * M
    A, R = gt[:11 * N2].reshape(11, N2), th2[:11 * N2].reshape(11, N2)
    src = case["theta"][:11 * N].reshape(11, N)
    keep = kind[parent] == dens.KEEP
    # kept Gaussians: bit-exact copies (parameters and moments)
    assert np.array_equal(A[:, keep], src[:, parent[keep]])
    assert np.array_equal(gm[:11 * N2].reshape(11, N2)[:, keep], m[:11 * N].reshape(11, N)[:, parent[keep]])
    assert np.array_equal(gv[:11 * N2].reshape(11, N2)[:, keep], v[:11 * N].reshape(11, N)[:, parent[keep]])
    ch = ~keep
    assert np.all(gm[:11 * N2].reshape(11, N2)[:, ch] == 0) and np.all(gv[:11 * N2].reshape(11, N2)[:, ch] == 0)
    step = np.abs(R[0:3, ch] - src[0:3, parent[ch]])
    assert np.all(np.abs(A[0:3, ch] - R[0:3, ch]) <= 2e-6 * (np.abs(R[0:3, ch]) + step) + 1e-7)
    assert np.all(np.abs(A[3:6, ch] - R[3:6, ch]) <= 1e-6)
    assert np.array_equal(A[6:10, ch], src[6:10, parent[ch]])
    assert np.all(np.abs(A[10, ch] - R[10, ch]) <= 1e-6 * np.abs(R[10, ch]))
    # poses and their moments
    assert np.array_equal(gt[11 * N2:], case["theta"][11 * N:])
    assert np.array_equal(gm[11 * N2:], m[11 * N:]) and np.array_equal(gv[11 * N2:], v[11 * N:])


CFG = dict(grad_threshold=1.5, log_scale_threshold=0.0, prune_amplitude=1e-4, split_factor=1.6, clone_offset=0.5)


@pytest.mark.parametrize("mass", [1, 0])
def test_split_clone_prune(G, dens, mass):
    case = small_case()
    N = case["N"]
    acc, count = inputs.densify_stats(5, N, count=3)
    m, v = moments(6, case["theta"].size)
    cfg = dict(CFG, mass_preserving=mass)
    ctx, out, got, ref = run_densify(G, dens, case, acc, count, cfg, m, v)
    assert out[1] > 20 and out[2] > 20 and out[3] == 7
    check_layout(case, out, got, ref, dens, m, v)
    a, c = G.gsvr_densify_stats(ctx.ctx, out[0])
    assert c == 0 and not a.any()
    ctx.close()


def test_accumulate_bit_exact(G, dens):
    import torch
    case = small_case(62, 300)
    N = case["N"]
    ctx = G.Context(case)
    rng = np.random.default_rng(7)
    acc = np.zeros((N, 4), np.float32)
    cnt = 0
    for k in range(3):
        g = rng.normal(0, 10.0 ** (k - 1), ctx.grad.numel()).astype(np.float32)
        ctx.grad.copy_(torch.from_numpy(g))
        G.gsvr_densify_accumulate(ctx.ctx)
        acc, cnt = dens.accumulate(acc, cnt, g, N)
    got, c = G.gsvr_densify_stats(ctx.ctx, N)
    assert c == cnt == 3
    assert np.array_equal(got, acc)
    ctx.close()


def test_forward_after_densify(G, dens):
    """The plain sum on the densified Gaussians against the oracle's forward on
    the oracle's densified parameters (every pixel)."""
    from oracle import oracle
    case = small_case(63, 120)
    N, M = case["N"], inputs.n_slices_total(case["stacks"])
    acc, count = inputs.densify_stats(8, N, count=2)
    z = np.zeros_like(case["theta"])
    ctx, out, got, ref = run_densify(G, dens, case, acc, count, CFG, z, z)
    ctx.forward()
    pred = ctx.pred.cpu().numpy().astype(np.float64)
    th2 = ref[0].astype(np.float32).astype(np.float64)
    pix = np.arange(inputs.n_pixels_total(case["stacks"]))
    I = case["I"].astype(np.float64)
    want, _, _, _, t_pred, _ = oracle.forward_backward(case["stacks"], th2, ref[3], pix, I, 1.0 / len(pix),
                                                       sel=np.zeros(ref[3], np.uint8), cutoff=1e-7)
    # children differ from the oracle's by float32 rounding of their means
    # (about 1e-7 mm), which moves a prediction by ~1e-6 of itself: 2e-5
    ok, worst = forward_ok(pred, want, t_pred, rtol=2e-5)
    assert ok.all(), worst
    ctx.backward()
    G.gsvr_adam_step(ctx.ctx, 1, {})
    G.gsvr_sync_status(ctx.ctx)
    assert np.all(np.isfinite(ctx.theta.cpu().numpy()))
    ctx.close()


def test_nothing_to_do_and_refusals(G, dens):
    case = small_case(64, 200)
    N = case["N"]
    acc, count = inputs.densify_stats(9, N, count=2)
    ctx = G.Context(case)
    G.gsvr_densify_stats(ctx.ctx, N, acc, count)
    before = ctx.theta.cpu().numpy()
    # a cap below the would-be count: refused, nothing changed (statistics kept)
    with pytest.raises(G.GsvrError) as e:
        ctx.densify(1.0, -5.0, max_gaussians=N)
    assert e.value.status == G.GSVR_ERR_CAPACITY
    assert np.array_equal(ctx.theta.cpu().numpy(), before)
    a, c = G.gsvr_densify_stats(ctx.ctx, N)
    assert c == count and np.array_equal(a, acc)
    # thresholds nobody passes: same Gaussians, statistics restart
    assert ctx.densify(1e30, 1e30) == (N, 0, 0, 0)
    assert np.array_equal(ctx.theta.cpu().numpy(), before)
    assert G.gsvr_densify_stats(ctx.ctx, N)[1] == 0
    with pytest.raises(G.GsvrError):
        ctx.densify(1.0, 0.0, split_factor=1.0)
    with pytest.raises(G.GsvrError):
        ctx.densify(1.0, 0.0, clone_offset=-1.0)
    # prune everything
    assert ctx.densify(1e30, 1e30, prune_amplitude=1e30)[0] == 0
    ctx.close()


def test_topk_context(G, dens):
    """The normalised top-K model after a densification (colours kept): the
    neighbour grid is rebuilt for the new count and forward / backward run."""
    case = small_case(65, 300)
    N = case["N"]
    th = case["theta"].copy()
    th[10 * N:11 * N] = np.abs(th[10 * N:11 * N]) + 0.1
    case["theta"] = th
    ctx = G.Context(case)
    G.gsvr_set_topk(ctx.ctx, 8, 1e-6, 1)
    ctx.forward()
    ctx.backward()
    G.gsvr_densify_accumulate(ctx.ctx)
    acc, c = G.gsvr_densify_stats(ctx.ctx, N)
    thr = float(np.quantile(acc[:, 0], 0.8))
    out = ctx.densify(thr, 0.0, mass_preserving=0)
    assert out[1] + out[2] > 0 and out[0] == N + out[1] + out[2]
    ctx.forward()
    ctx.backward()
    G.gsvr_sync_status(ctx.ctx)
    assert np.isfinite(ctx.loss())
    ctx.close()


def test_batched_context_refused(G):
    cases = [inputs.random_case(70 + k, 50, [(2, 8, 9)], n_stacks=1) for k in range(2)]
    b = inputs.concat_cases(cases)
    ctx = G.Context(b)
    G.gsvr_set_subjects(ctx.ctx, b["stack_subject"], b["gauss_count"])
    with pytest.raises(G.GsvrError) as e:
        ctx.densify(1.0, 0.0)
    assert e.value.status == G.GSVR_ERR_STATE
    ctx.close()


def test_fetal_workload(G, dens):
    """200,480 Gaussians of the fetal workload with heavy-tailed statistics:
    the new count and the whole layout exactly, values on every child."""
    case = inputs.fetal(0)
    N = case["N"]
    acc, count = inputs.densify_stats(11, N, count=5, scale=1e-4)
    thr = float(np.quantile(acc[:, 0] / count, 0.95))
    cfg = dict(grad_threshold=thr, log_scale_threshold=float(np.log(0.79)), prune_amplitude=0.0)
    z = np.zeros_like(case["theta"])
    ctx, out, got, ref = run_densify(G, dens, case, acc, count, cfg, z, z)
    assert out[1] > 1000 or out[2] > 1000
    check_layout(case, out, got, ref, dens, z, z)
    ctx.close()
