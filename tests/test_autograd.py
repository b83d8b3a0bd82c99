"""The adjoint behind torch.autograd.Function (loss output and prediction
output with an arbitrary downstream loss) against the FP64 oracle."""
import numpy as np
import pytest

from paper_2512_11624_b300 import inputs
from tests.gpu_util import CUTOFF, describe_grad, grad_ok

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2512_11624_b300 import autograd, gsvr
    return torch, gsvr, autograd


def test_loss_function_gradient_matches_oracle(mods, oracle):
    torch, gsvr, autograd = mods
    case = inputs.random_case(41, 400, [(3, 30, 36), (2, 27, 25)], n_stacks=2, motion_deg=8.0)
    gs = gsvr.Context(case, tile_h=12, tile_w=12)
    theta = torch.from_numpy(case["theta"].astype(np.float32)).cuda().requires_grad_(True)
    loss = autograd.SliceLoss.apply(theta, gs)
    (3.0 * loss).backward()
    pix = np.arange(inputs.n_pixels_total(case["stacks"]))
    _, L, g, a, _, t = oracle.forward_backward(case["stacks"], case["theta"].astype(np.float64), case["N"], pix,
                                               case["I"].astype(np.float64), 1.0 / len(pix), cutoff=CUTOFF)
    assert abs(float(loss) - L) <= 1e-5 * L
    ok, worst, _ = grad_ok(theta.grad.cpu().numpy().astype(np.float64), 3.0 * g, 3.0 * a, 3.0 * t)
    assert ok.all(), describe_grad(theta.grad.cpu().numpy(), 3.0 * g, 3.0 * a, case["N"],
                                   inputs.n_slices_total(case["stacks"]), 3.0 * t)
    rep = autograd.recompute_vs_store_bytes(gs)
    assert rep["store_per_pair_bytes"] == 4 * rep["pairs_evaluated"] and rep["recompute_bytes"] > 0
    gs.close()


def test_prediction_function_with_linear_downstream_loss(mods, oracle):
    """d(sum_p a_p I_hat_p)/dtheta equals the oracle's MSE gradient for the
    observations I' = I_hat_ref - a / (2 w) (whose residual weights are exactly a)."""
    torch, gsvr, autograd = mods
    case = inputs.random_case(42, 300, [(3, 26, 31)], n_stacks=2, motion_deg=8.0)
    P = inputs.n_pixels_total(case["stacks"])
    rng = np.random.default_rng(42)
    sub = rng.choice(P, P // 2, replace=False).astype(np.int32)
    gs = gsvr.Context(case, tile_h=16, tile_w=8)
    gsvr.gsvr_set_pixel_sample(gs.ctx, sub)
    theta = torch.from_numpy(case["theta"].astype(np.float32)).cuda().requires_grad_(True)
    pred = autograd.SlicePredict.apply(theta, gs)
    order = gs.sample_index().cpu().numpy()
    a_w = rng.normal(size=order.size)
    (pred * torch.from_numpy(a_w.astype(np.float32)).cuda()).sum().backward()
    th = case["theta"].astype(np.float64)
    pred_ref, _ = oracle.forward(case["stacks"], th, case["N"], order)
    assert np.allclose(pred.detach().cpu().numpy(), pred_ref, rtol=1e-4, atol=1e-5 * np.abs(pred_ref).max())
    w = 1.0 / order.size
    I_prime = pred_ref - a_w / (2 * w)
    _, _, g, a, _, t = oracle.forward_backward(case["stacks"], th, case["N"], order, I_prime, w, cutoff=CUTOFF)
    ok, worst, _ = grad_ok(theta.grad.cpu().numpy().astype(np.float64), g, a, t)
    assert ok.all(), describe_grad(theta.grad.cpu().numpy(), g, a, case["N"], inputs.n_slices_total(case["stacks"]),
                                   t)
    gs.close()
