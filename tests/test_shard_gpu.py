"""The data-parallel split of one reconstruction through the CUDA path, its
ranks emulated one after another on one GPU (each rank's part is a context of
its own; the test adds up what the all-reduce would).  Each part weights its
pixels by 1 / (global sample size) (gsvr_set_sample_total), so the parts'
losses and Gaussian gradients must add up to the whole case's, and each
part's pose gradients must be the whole case's for its slices: all checked
against the float64 all-pairs oracle of the whole case at the parity
tolerances, for a split at a stack boundary and one inside a stack."""
import numpy as np
import pytest

from paper_2512_11624_b300 import inputs, shard
from tests.gpu_util import CUTOFF, forward_ok, grad_ok

pytestmark = pytest.mark.gpu


def test_two_shards_on_one_gpu_add_up_to_the_whole(oracle):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2512_11624_b300 import gsvr
    case = inputs.random_case(21, 1200, [(4, 30, 28), (3, 26, 33), (5, 22, 24), (3, 31, 25)], n_stacks=4,
                              motion_deg=6.0, motion_mm=3.0)
    N = case["N"]
    M = inputs.n_slices_total(case["stacks"])
    P = inputs.n_pixels_total(case["stacks"])
    idx = np.sort(np.random.default_rng(3).choice(P, (2 * P) // 3, replace=False))
    pred_ref, L_ref, g_ref, a_ref, tp, tg = oracle.forward_backward(
        case["stacks"], case["theta"].astype(np.float64), N, idx, case["I"].astype(np.float64)[idx],
        1.0 / idx.size, cutoff=CUTOFF)
    for bounds in ([0, 7, M], [0, 9, M]):  # 7: stack boundary; 9: inside the third stack
        g_sum = np.zeros(11 * N)
        L = 0.0
        pred = np.zeros(P)
        for r in range(2):
            part = shard.shard_case(case, r, 2, bounds)
            p0, p1 = part["pixel_range"]
            s0, s1 = part["slice_range"]
            ctx = gsvr.Context(part)
            sel = idx[(idx >= p0) & (idx < p1)]
            gsvr.gsvr_set_pixel_sample(ctx.ctx, (sel - p0).astype(np.int32))
            gsvr.gsvr_set_sample_total(ctx.ctx, idx.size)
            ctx.forward()
            ctx.backward()
            gsvr.gsvr_sync_status(ctx.ctx)
            g = ctx.grad.cpu().numpy().astype(np.float64)
            pred[p0:p1] = ctx.pred.cpu().numpy()
            L += ctx.loss()
            g_sum += g[:11 * N]
            pose = slice(11 * N + 6 * s0, 11 * N + 6 * s1)
            ok, worst, _ = grad_ok(g[11 * N:], g_ref[pose], a_ref[pose], tg[pose])
            assert ok.all(), ("pose", bounds, r, worst)
            ctx.close()
        ok, worst = forward_ok(pred[idx], pred_ref, tp)
        assert ok.all(), ("forward", bounds, worst)
        assert abs(L - L_ref) <= 1e-5 * L_ref, (bounds, L, L_ref)
        ok, worst, plain = grad_ok(g_sum, g_ref[:11 * N], a_ref[:11 * N], tg[:11 * N])
        assert ok.all(), ("gaussians", bounds, worst)
