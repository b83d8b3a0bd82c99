"""Gradient parity at the fetal size against the analytic float64 oracle.

The fetal workload (200,480 Gaussians; three orthogonal stacks of
40 x 192 x 192 px; 2^18 pixels drawn by the device sampler), its amplitudes
30 % off the fit and every primitive turned and stretched at random so that
every gradient group is nonzero, through the CUDA path in the bench's usual
launch shape (8 x 16 pixel tiles) and in the default 12 x 12.  The oracle is
the grid-pruned analytic gradient (oracle.local_grad: the per-pair
expressions of the all-pairs oracle, pairs below 1e-12 dropped, pinned against
the all-pairs oracle in test_oracle_local.py) over the same 2^18 pixels.
Compared element by element: every slice-pose entry (720) and every component
of 150 random Gaussians (1,650 entries), within
1e-4 |g| + 1e-6 (sum|terms| + B) + (sum of |terms| below the 1e-7 cut) + Bt,
B and Bt the prediction- and truncation-scale sums of tests/gpu_util.py."""
import numpy as np
import pytest

from paper_2512_11624_b300 import inputs
from tests.gpu_util import forward_ok, large_grad_check

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def G():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2512_11624_b300 import gsvr
    return gsvr


@pytest.fixture(scope="module")
def fetal_case():
    return inputs.fetal(0, amplitude_jitter=0.3, shape_jitter=0.2)


@pytest.mark.parametrize("tile", [(8, 16), (12, 12)])
def test_fetal_gradient_matches_oracle(G, oracle, fetal_case, tile):
    case = fetal_case
    N = case["N"]
    M = inputs.n_slices_total(case["stacks"])
    ctx = G.Context(case, tile_h=tile[0], tile_w=tile[1])
    G.gsvr_sample_pixels(ctx.ctx, case["n_sample"], 3)
    ctx.forward()
    ctx.backward()
    G.gsvr_sync_status(ctx.ctx)
    pix = np.sort(G.gsvr_get_sample(ctx.ctx).astype(np.int64))
    assert pix.size == case["n_sample"]
    g = ctx.grad.cpu().numpy().astype(np.float64)
    pred = ctx.pred.cpu().numpy().astype(np.float64)[pix]
    loss = ctx.loss()
    ctx.close()
    sel = np.sort(np.random.default_rng(11).choice(N, 150, replace=False))
    ref = oracle.local_grad(case["stacks"], case["theta"].astype(np.float64), N, pix,
                            case["I"].astype(np.float64)[pix], 1.0 / pix.size, sel)
    ok, worst = forward_ok(pred, ref["pred"], ref["trunc_pred"])
    assert ok.all(), ("forward", worst)
    assert abs(loss - ref["loss"]) <= 1e-5 * ref["loss"], (loss, ref["loss"])
    comp, pose = oracle.select_entries(N, M, sel)
    names = ["mu", "ls", "q", "c"]
    rows = [slice(0, 3), slice(3, 6), slice(6, 10), slice(10, 11)]
    worst = []
    for nm, rw in zip(names, rows):
        worst.append(large_grad_check(g[comp[rw]].ravel(), ref["g_sel"][rw].ravel(), ref["a_sel"][rw].ravel(),
                                      ref["b_sel"][rw].ravel(), ref["t_sel"][rw].ravel(), ref["bt_sel"][rw].ravel(),
                                      nm))
    gp = g[pose].reshape(M, 6)
    for nm, cols in (("rotation", slice(0, 3)), ("translation", slice(3, 6))):
        worst.append(large_grad_check(gp[:, cols].ravel(), *[ref[k].reshape(M, 6)[:, cols].ravel() for k in (
            "g_pose", "a_pose", "b_pose", "t_pose", "bt_pose")], nm))
    assert max(worst) <= 1.0, worst
