"""gsvr_forward_noalloc -- the forward for callers that cannot allocate device
memory (its scratch is a fixed device array inside the library) -- against the
context-based gsvr_forward on the same inputs.  Checked:
- two calls in a row with different pixel samples: the second call must not
  see the first call's leftovers in the shared scratch;
- the every-pixel branch (idx = None);
- a sample drawn with replacement that is longer than the pixel count;
- a problem whose (slice, Gaussian) records overflow the scratch on the device
  (GSVR_ERR_CAPACITY), followed by a normal call that still matches;
- a problem whose pixel arrays alone exceed the scratch (rejected up front).
Collected last so a failure here stops a -x run only after every other test
has run."""
import numpy as np
import pytest

from paper_2512_11624_b300 import inputs
from tests.gpu_util import forward_ok

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2512_11624_b300 import gsvr
    return gsvr


def _case():
    return inputs.random_case(31, 700, [(4, 37, 45), (3, 29, 33)], n_stacks=2, motion_deg=8.0, motion_mm=3.0)


def _context_forward(G, case, idx):
    ctx = G.Context(case)
    G.gsvr_set_pixel_sample(ctx.ctx, idx)
    ctx.forward()
    pred = ctx.pred.cpu().numpy().astype(np.float64)
    loss = ctx.loss()
    ctx.close()
    return pred, loss


def _noalloc(G, case, idx):
    import torch
    P = inputs.n_pixels_total(case["stacks"])
    theta_d = torch.from_numpy(case["theta"].astype(np.float32)).cuda()
    I_d = torch.from_numpy(case["I"].astype(np.float32)).cuda()
    pred_d = torch.full((P,), -1.0, dtype=torch.float32, device="cuda")
    loss_d = torch.zeros(1, dtype=torch.float64, device="cuda")
    idx_d = torch.from_numpy(idx).cuda() if idx is not None else None
    G.gsvr_forward_noalloc(case["stacks"], case["N"], theta_d, I_d, idx_d, pred_d, loss_d)
    return pred_d.cpu().numpy().astype(np.float64), float(loss_d.item())


def _check(got, loss, ref_pred, ref_loss, pix, P, what):
    ok, worst = forward_ok(got[pix], ref_pred[pix])
    assert ok.all(), (what, worst)
    untouched = np.setdiff1d(np.arange(P), pix)
    assert np.all(got[untouched] == -1.0), what
    assert abs(loss - ref_loss) <= 1e-6 * ref_loss, (what, loss, ref_loss)


def test_forward_noalloc_matches_context_forward(G):
    case = _case()
    P = inputs.n_pixels_total(case["stacks"])
    rng = np.random.default_rng(31)
    samples = [rng.choice(P, P // 2, replace=False).astype(np.int32),
               rng.choice(P, P // 3, replace=True).astype(np.int32),
               rng.choice(P, 2 * P, replace=True).astype(np.int32),  # longer than P, duplicates count once
               None]                                                 # every pixel
    for call, idx in enumerate(samples):
        ref_pred, ref_loss = _context_forward(G, case, idx)
        got, loss = _noalloc(G, case, idx)
        pix = np.unique(idx) if idx is not None else np.arange(P)
        _check(got, loss, ref_pred, ref_loss, pix, P, call)


def test_forward_noalloc_capacity_overflow_then_recovers(G):
    import torch
    # 5,000 wide Gaussians (s = 20 mm) over 60 thin slices of 8 x 8 px: every
    # Gaussian meets every slice, 300,000 records, about twice the scratch's room
    rng = np.random.default_rng(5)
    st = [inputs.stack(60, 8, 8, 1.0, 1.0, 1.0)]
    N, M = 5000, 60
    th = np.zeros(11 * N + 6 * M, np.float32)
    th[0:N] = rng.uniform(-4, 4, N)
    th[N:2 * N] = rng.uniform(-4, 4, N)
    th[2 * N:3 * N] = rng.uniform(-30, 30, N)
    th[3 * N:6 * N] = np.log(20.0)
    th[6 * N:7 * N] = 1.0
    th[10 * N:11 * N] = rng.uniform(0, 1, N)
    P = 60 * 64
    t_d = torch.from_numpy(th).cuda()
    I_d = torch.zeros(P, dtype=torch.float32, device="cuda")
    pred_d = torch.zeros(P, dtype=torch.float32, device="cuda")
    loss_d = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(G.GsvrError) as ei:
        G.gsvr_forward_noalloc(st, N, t_d, I_d, None, pred_d, loss_d)
    assert ei.value.status == G.GSVR_ERR_CAPACITY, str(ei.value)
    # the next call on a problem that fits is unaffected by the overflowed one
    case = _case()
    P2 = inputs.n_pixels_total(case["stacks"])
    idx = np.random.default_rng(9).choice(P2, P2 // 2, replace=False).astype(np.int32)
    ref_pred, ref_loss = _context_forward(G, case, idx)
    got, loss = _noalloc(G, case, idx)
    _check(got, loss, ref_pred, ref_loss, np.unique(idx), P2, "after overflow")


def test_forward_noalloc_rejects_oversize(G):
    import torch
    big = [inputs.stack(200, 1024, 1024, 1.0, 1.0, 3.0)]
    t = torch.zeros(11 + 6 * 200, dtype=torch.float32, device="cuda")
    I = torch.zeros(16, dtype=torch.float32, device="cuda")
    with pytest.raises(G.GsvrError) as ei:
        G.gsvr_forward_noalloc(big, 1, t, I, None, I, torch.zeros(1, dtype=torch.float64, device="cuda"))
    assert ei.value.status == G.GSVR_ERR_INVALID_ARG and "32 MiB" in str(ei.value)
