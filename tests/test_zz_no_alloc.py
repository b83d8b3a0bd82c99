"""gsvr_forward_noalloc -- the forward for callers that cannot allocate device
memory (its scratch is a fixed device array inside the library) -- against the
context-based gsvr_forward on the same inputs, on two calls in a row with
different pixel samples (the second call must not see the first call's
leftovers in the shared scratch).  Collected last so a failure here stops a
-x run only after every other test has run."""
import numpy as np
import pytest

from paper_2512_11624_b300 import inputs
from tests.gpu_util import forward_ok

pytestmark = pytest.mark.gpu


def test_forward_noalloc_matches_context_forward():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2512_11624_b300 import gsvr
    case = inputs.random_case(31, 700, [(4, 37, 45), (3, 29, 33)], n_stacks=2, motion_deg=8.0, motion_mm=3.0)
    N = case["N"]
    P = inputs.n_pixels_total(case["stacks"])
    rng = np.random.default_rng(31)
    samples = [rng.choice(P, P // 2, replace=False).astype(np.int32),
               rng.choice(P, P // 3, replace=True).astype(np.int32)]
    theta_d = torch.from_numpy(case["theta"].astype(np.float32)).cuda()
    I_d = torch.from_numpy(case["I"].astype(np.float32)).cuda()
    for call, idx in enumerate(samples):
        ctx = gsvr.Context(case)
        gsvr.gsvr_set_pixel_sample(ctx.ctx, idx)
        ctx.forward()
        ref_pred = ctx.pred.cpu().numpy().astype(np.float64)
        ref_loss = ctx.loss()
        ctx.close()
        pred_d = torch.full((P,), -1.0, dtype=torch.float32, device="cuda")
        loss_d = torch.zeros(1, dtype=torch.float64, device="cuda")
        gsvr.gsvr_forward_noalloc(case["stacks"], N, theta_d, I_d, torch.from_numpy(idx).cuda(), pred_d, loss_d)
        got = pred_d.cpu().numpy().astype(np.float64)
        pix = np.unique(idx)
        ok, worst = forward_ok(got[pix], ref_pred[pix])
        assert ok.all(), (call, worst)
        untouched = np.setdiff1d(np.arange(P), pix)
        assert np.all(got[untouched] == -1.0)
        assert abs(float(loss_d.item()) - ref_loss) <= 1e-6 * ref_loss, (call, float(loss_d.item()), ref_loss)


def test_forward_noalloc_rejects_oversize():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2512_11624_b300 import gsvr
    big = [inputs.stack(200, 1024, 1024, 1.0, 1.0, 3.0)]
    t = torch.zeros(11 + 6 * 200, dtype=torch.float32, device="cuda")
    I = torch.zeros(16, dtype=torch.float32, device="cuda")
    with pytest.raises(gsvr.GsvrError) as ei:
        gsvr.gsvr_forward_noalloc(big, 1, t, I, None, I, torch.zeros(1, dtype=torch.float64, device="cuda"))
    assert ei.value.status == 1 and "32 MiB" in str(ei.value)
