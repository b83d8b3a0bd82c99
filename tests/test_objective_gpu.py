"""The paper's objective options on the GPU (gsvr_set_objective, Sec. 2.5):
the L1 data term and the scale regulariser, on the plain path and on the
top-K path, against the float64 oracles with the tolerances of the plain
parity tests (forward 1e-5 relative, gradients 1e-4 relative plus a float32
floor in the sum of |terms|, plus the cutoff truncation bound on the plain
path)."""
import numpy as np
import pytest

from paper_2512_11624_b300 import inputs
from tests.gpu_util import CUTOFF, describe_grad, forward_ok, grad_ok

pytestmark = pytest.mark.gpu

LAM, S_T = 2.5e-3, 1.6


@pytest.fixture(scope="module")
def G():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2512_11624_b300 import gsvr
    return gsvr


def case_with_offset(seed):
    case = inputs.random_case(seed, 250, [(3, 21, 19), (2, 16, 23)], n_stacks=2, extent=4.0, motion_deg=8.0)
    case["I"] = (case["I"] + 0.02).astype(np.float32)  # keeps residuals off the L1 kink
    return case


@pytest.mark.parametrize("loss_kind,lam", [(1, 0.0), (0, LAM), (1, LAM)])
def test_plain_path(G, oracle, loss_kind, lam):
    case = case_with_offset(41)
    ctx = G.Context(case)
    G.gsvr_set_objective(ctx.ctx, loss_kind, lam, S_T)
    ctx.forward()
    ctx.backward()
    G.gsvr_sync_status(ctx.ctx)
    pred = ctx.pred.cpu().numpy().astype(np.float64)
    grad = ctx.grad.cpu().numpy().astype(np.float64)
    loss = ctx.loss()
    ctx.close()
    st, N = case["stacks"], case["N"]
    pix = np.arange(inputs.n_pixels_total(st))
    th = case["theta"].astype(np.float64)
    I = case["I"].astype(np.float64)[pix]
    p_ref, L_ref, g_ref, a_ref, t_pred, t_grad = oracle.forward_backward(
        st, th, N, pix, I, 1.0 / len(pix), cutoff=CUTOFF, loss_kind=loss_kind, lambda_reg=lam, s_target=S_T)
    assert np.abs(p_ref - I).min() > 1e-4
    ok, worst = forward_ok(pred[pix], p_ref, t_pred)
    assert ok.all(), worst
    assert abs(loss - L_ref) <= 1e-4 * L_ref, (loss, L_ref)
    gok, gworst, _ = grad_ok(grad, g_ref, a_ref, t_grad)
    M = inputs.n_slices_total(st)
    assert gok.all(), (gworst, describe_grad(grad, g_ref, a_ref, N, M, t_grad))


def test_topk_path(G):
    from oracle import topk
    case = case_with_offset(42)
    K, delta = 24, 1e-4
    ctx = G.Context(case)
    G.gsvr_set_objective(ctx.ctx, 1, LAM, S_T)
    G.gsvr_set_topk(ctx.ctx, K, delta, 1)
    ctx.forward()
    pix, nbr, _ = G.gsvr_get_topk_neighbors(ctx.ctx, K)
    ctx.backward()
    G.gsvr_sync_status(ctx.ctx)
    pred = ctx.pred.cpu().numpy().astype(np.float64)
    grad = ctx.grad.cpu().numpy().astype(np.float64)
    loss = ctx.loss()
    ctx.close()
    st, N = case["stacks"], case["N"]
    pix = pix.astype(np.int64)
    th = case["theta"].astype(np.float64)
    I = case["I"].astype(np.float64)[pix]
    p_ref, L_ref, g_ref, _, A = topk.forward_backward(st, th, N, pix, I, 1.0 / len(pix), K, delta,
                                                     nbr=nbr.astype(np.int64), want_abs=True, loss_kind=1,
                                                     lambda_reg=LAM, s_target=S_T)
    ok, worst = forward_ok(pred[pix], p_ref)
    assert ok.all(), worst
    assert abs(loss - L_ref) <= 1e-4 * L_ref, (loss, L_ref)
    gok, gworst, _ = grad_ok(grad, g_ref, A)
    M = inputs.n_slices_total(st)
    assert gok.all(), (gworst, describe_grad(grad, g_ref, A, N, M))


def test_argument_checks(G):
    case = inputs.random_case(43, 10, [(1, 6, 6)], n_stacks=1)
    ctx = G.Context(case)
    for lk, lam, s in [(2, 0.0, 1.6), (-1, 0.0, 1.6), (0, -1.0, 1.6), (0, float("inf"), 1.6), (0, 0.1, 0.0),
                       (0, 0.1, float("nan"))]:
        with pytest.raises(G.GsvrError) as e:
            G.gsvr_set_objective(ctx.ctx, lk, lam, s)
        assert "INVALID_ARG" in str(e.value)
    ctx.close()


@pytest.mark.parametrize("topk_K", [0, 16])
def test_slice_weights(G, oracle, topk_K):
    """Per-slice log sigma_i and log omega_i (gsvr_set_slice_weights) with the
    L1 term and the regulariser, on the plain path (topk_K = 0) and the top-K
    path: predictions, loss, parameter gradients and the per-slice gradients
    against the oracles; one Adam step of the per-slice terms against the
    textbook update (the frozen slice keeping its sigma)."""
    from oracle import topk
    case = case_with_offset(44)
    st, N = case["stacks"], case["N"]
    M = inputs.n_slices_total(st)
    rng = np.random.default_rng(5)
    slw = np.concatenate([rng.normal(0, 0.1, M), rng.normal(0, 0.3, M)]).astype(np.float32)
    ctx = G.Context(case)
    G.gsvr_set_objective(ctx.ctx, 1, LAM, S_T)
    if topk_K:
        G.gsvr_set_topk(ctx.ctx, topk_K, 1e-4, 1)
    G.gsvr_set_slice_weights(ctx.ctx, 1, 2e-3, 3e-3)
    G.gsvr_set_frozen(ctx.ctx, np.array([1] + [0] * (M - 1), np.uint8))
    params, grads = G.gsvr_slice_weight_views(ctx.ctx)
    params.copy_(__import__("torch").from_numpy(slw).cuda())
    ctx.forward()
    pix_t = None
    if topk_K:
        pix_t, nbr, _ = G.gsvr_get_topk_neighbors(ctx.ctx, topk_K)
    ctx.backward()
    G.gsvr_sync_status(ctx.ctx)
    pred = ctx.pred.cpu().numpy().astype(np.float64)
    grad = ctx.grad.cpu().numpy().astype(np.float64)
    gsl = grads.cpu().numpy().astype(np.float64)
    loss = ctx.loss()
    G.gsvr_adam_step(ctx.ctx, 1, lr=dict(lr_mu=0, lr_ls=0, lr_q=0, lr_c=0, lr_rot=0, lr_trans=0))
    after = params.cpu().numpy().astype(np.float64)
    ctx.close()
    pix = np.arange(inputs.n_pixels_total(st)) if not topk_K else pix_t.astype(np.int64)
    th = case["theta"].astype(np.float64)
    I = case["I"].astype(np.float64)[pix]
    ref_gs = np.zeros(2 * M)
    if topk_K:
        p_ref, L_ref, g_ref, _, A = topk.forward_backward(st, th, N, pix, I, 1.0 / len(pix), topk_K, 1e-4,
                                                         nbr=nbr.astype(np.int64), want_abs=True, loss_kind=1,
                                                         lambda_reg=LAM, s_target=S_T, slw=slw.astype(np.float64),
                                                         slw_grad=ref_gs)
        t_pred, t_grad = None, None
    else:
        p_ref, L_ref, g_ref, A, t_pred, t_grad = oracle.forward_backward(
            st, th, N, pix, I, 1.0 / len(pix), cutoff=CUTOFF, loss_kind=1, lambda_reg=LAM, s_target=S_T,
            slw=slw.astype(np.float64), slw_grad=ref_gs)
    ok, worst = forward_ok(pred[pix], p_ref, t_pred)
    assert ok.all(), worst
    assert abs(loss - L_ref) <= 1e-4 * abs(L_ref) + 1e-6, (loss, L_ref)
    gok, gworst, _ = grad_ok(grad, g_ref, A, t_grad)
    assert gok.all(), (gworst, describe_grad(grad, g_ref, A, N, M, t_grad))
    # per-slice gradients: float64 sums of float32 pixel terms
    assert np.allclose(gsl, ref_gs, rtol=1e-4, atol=1e-5 * np.abs(ref_gs).max()), np.abs(gsl - ref_gs).max()
    # Adam, step 1: p - lr sign(g) (bias-corrected first step), sigma of the frozen slice unchanged
    lr = np.concatenate([np.full(M, 2e-3), np.full(M, 3e-3)])
    want = slw.astype(np.float64) - lr * gsl / (np.abs(gsl) + 1e-8)
    want[0] = slw[0]
    assert np.allclose(after, want, rtol=1e-5, atol=1e-7)
