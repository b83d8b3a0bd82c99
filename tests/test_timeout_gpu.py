"""Failure detection without a GPU fault: a bounded device-side wait that runs
out.  The test hook gsvr_test_wait_timeout makes every block of the next
forward wait, for its first work item with records, on a shared-memory
barrier that nothing completes (bounded at 2 ms); the wait runs out, the
block drains the copies it started (normal 1 s bound) and stops.  The host reads GSVR_ERR_TIMEOUT at
gsvr_sync_status, and the context stays usable: the next forward is normal
and gives bitwise the predictions of the forward before the hook."""
import numpy as np
import pytest

from paper_2512_11624_b300 import inputs

pytestmark = pytest.mark.gpu


def test_bounded_wait_runs_out_and_context_recovers():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2512_11624_b300 import gsvr
    case = inputs.random_case(3, 1500, [(4, 48, 40), (3, 36, 44)], n_stacks=2, motion_deg=6.0, motion_mm=3.0)
    ctx = gsvr.Context(case)
    ctx.forward()
    assert gsvr.gsvr_sync_status(ctx.ctx) == gsvr.GSVR_OK
    ref = ctx.pred.cpu().numpy().copy()
    ref_loss = ctx.loss()
    with pytest.raises(gsvr.GsvrError):
        gsvr.gsvr_test_wait_timeout(ctx.ctx, 1, 10)  # limit below 1 us is refused
    gsvr.gsvr_test_wait_timeout(ctx.ctx, 1, 2_000_000)
    ctx.forward()
    with pytest.raises(gsvr.GsvrError) as ei:
        gsvr.gsvr_sync_status(ctx.ctx)
    assert ei.value.status == gsvr.GSVR_ERR_TIMEOUT, str(ei.value)
    # the status word was cleared by the read; the next forward is normal
    ctx.forward()
    assert gsvr.gsvr_sync_status(ctx.ctx) == gsvr.GSVR_OK
    assert np.array_equal(ctx.pred.cpu().numpy(), ref)
    assert ctx.loss() == ref_loss
    ctx.backward()
    assert gsvr.gsvr_sync_status(ctx.ctx) == gsvr.GSVR_OK
    ctx.close()
