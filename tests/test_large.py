"""The large workload (1,000,372 Gaussians, six stacks of 48 x 256^2 px, 7.1M
masked pixels; primitives turned and stretched at random) through the CUDA
path at its full size, checked on sampled outputs the float64 oracle can
compute one by one.  The loss is taken over 20,000 random masked pixels.
- predictions of those pixels against the oracle's grid-searched float64 sums
  (which the small-case pins tie to the all-pairs oracle);
- the analytic gradient: every slice-pose entry (1,728) and all 11 components
  of the Gaussians of 700 random Gaussian parameters against the grid-pruned
  analytic oracle (oracle.local_grad), within 1e-4 |g| + 1e-6 (sum|terms| +
  B) + (sum of |terms| below the 1e-7 cut) + Bt, B and Bt the prediction- and
  truncation-scale sums of tests/gpu_util.py;
- as a second check, the gradient against float64 central differences of the
  same loss for 1,000 random parameters (700 Gaussian components, 300 slice
  poses), beyond the truncation terms T + Bt of the analytic reference (the
  differences take the untruncated model).
Amplitudes start 30 % off the fit so that residuals, and so the gradients,
are far from zero.  One forward + backward over every masked pixel is timed
and printed."""
import time

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
def run(G):
    case = inputs.large(0, amplitude_jitter=0.3, shape_jitter=0.2)
    N = case["N"]
    M = inputs.n_slices_total(case["stacks"])
    rng = np.random.default_rng(5)
    masked = np.nonzero(case["mask"])[0]
    pix = np.sort(rng.choice(masked, size=20000, replace=False))
    ctx = G.Context(case, tile_h=12, tile_w=12)
    G.gsvr_set_pixel_sample(ctx.ctx, pix.astype(np.int32))
    ctx.forward()
    ctx.backward()
    G.gsvr_sync_status(ctx.ctx)
    pred = ctx.pred.cpu().numpy().astype(np.float64)[pix]
    g = ctx.grad.cpu().numpy().astype(np.float64)
    loss = ctx.loss()
    # one full iteration over every masked pixel, timed (printed)
    G.gsvr_set_pixel_sample(ctx.ctx, None)
    ctx.forward()
    ctx.backward()
    G.gsvr_sync_status(ctx.ctx)
    t0 = time.perf_counter()
    for _ in range(3):
        ctx.forward()
        ctx.backward()
    G.gsvr_sync_status(ctx.ctx)
    st = ctx.stats()
    print("large: %.1f ms per forward + backward over %d pixels (%d records, %d keys)" %
          ((time.perf_counter() - t0) / 3 * 1e3, st["n_sampled"], st["n_records"], st["n_keys"]))
    ctx.close()
    params = np.concatenate([rng.choice(11 * N, 700, replace=False), 11 * N + rng.choice(6 * M, 300, replace=False)])
    return {"case": case, "N": N, "M": M, "pix": pix, "pred": pred, "g": g, "loss": loss, "params": params}


@pytest.fixture(scope="module")
def ref(run, oracle):
    """The analytic float64 reference for the Gaussians of the sampled parameters and every pose."""
    case, N, pix = run["case"], run["N"], run["pix"]
    sel = np.unique(run["params"][run["params"] < 11 * N] % N)
    out = oracle.local_grad(case["stacks"], case["theta"].astype(np.float64), N, pix,
                            case["I"].astype(np.float64)[pix], 1.0 / pix.size, sel)
    out["sel"] = sel
    return out


def test_large_case_analytic_gradient(run, ref, oracle):
    N, M, g = run["N"], run["M"], run["g"]
    ok, worst = forward_ok(run["pred"], ref["pred"], ref["trunc_pred"])
    assert ok.all(), ("forward", (~ok).sum(), worst)
    assert abs(run["loss"] - ref["loss"]) <= 1e-5 * ref["loss"], (run["loss"], ref["loss"])
    comp, pose = oracle.select_entries(N, M, ref["sel"])
    worst = []
    for nm, rw in zip(["mu", "ls", "q", "c"], [slice(0, 3), slice(3, 6), slice(6, 10), slice(10, 11)]):
        worst.append(large_grad_check(g[comp[rw]].ravel(), *[ref[k][rw].ravel() for k in (
            "g_sel", "a_sel", "b_sel", "t_sel", "bt_sel")], nm))
    gp = g[pose].reshape(M, 6)
    for nm, cols in (("rotation", slice(0, 3)), ("translation", slice(3, 6))):
        worst.append(large_grad_check(gp[:, cols].ravel(), *[ref[k].reshape(M, 6)[:, cols].ravel() for k in (
            "g_pose", "a_pose", "b_pose", "t_pose", "bt_pose")], nm))
    assert max(worst) <= 1.0, worst


def test_large_case_predictions_and_fd(run, ref, oracle):
    case, N, M, pix, g, params = run["case"], run["N"], run["M"], run["pix"], run["g"], run["params"]
    th = case["theta"].astype(np.float64)
    scale = np.ones(params.size)
    amp = (params >= 10 * N) & (params < 11 * N)
    scale[amp] = np.abs(th[params[amp]])
    h = 1e-4 * scale
    fd, pred_ref, trunc = oracle.local_fd(case["stacks"], th, N, pix, case["I"].astype(np.float64)[pix],
                                          1.0 / pix.size, params, h, cut=1e-12, trunc_cut=1e-7)
    ok, worst = forward_ok(run["pred"], pred_ref, trunc)
    assert ok.all(), ("forward", (~ok).sum(), worst)
    # the CUDA path differentiates the model with the pairs below the 1e-7 cut dropped; the
    # differences take the full model: they may differ by the dropped terms (T) and by their
    # effect on the residuals (Bt), both from the analytic reference
    slack = np.zeros(params.size)
    where = {int(j): k for k, j in enumerate(ref["sel"])}
    for k, q in enumerate(params):
        if q < 11 * N:
            row, col = q // N, where[int(q % N)]
            slack[k] = ref["t_sel"][row, col] + ref["bt_sel"][row, col]
        else:
            slack[k] = ref["t_pose"][q - 11 * N] + ref["bt_pose"][q - 11 * N]
    gp = g[params]
    err = np.abs(gp - fd)
    groups = {"mu": params < 3 * N, "ls": (params >= 3 * N) & (params < 6 * N),
              "q": (params >= 6 * N) & (params < 10 * N), "c": amp,
              "rot": (params >= 11 * N) & ((params - 11 * N) % 6 < 3),
              "trans": (params >= 11 * N) & ((params - 11 * N) % 6 >= 3)}
    top = np.abs(fd).max()
    for name, sel in groups.items():
        if not sel.any():
            continue
        # floor: 1e-3 of the group's largest entry, and 1e-6 of the largest overall (the quaternion
        # gradient of an isotropic Gaussian is exactly zero)
        floor = max(1e-3 * np.abs(fd[sel]).max(), 1e-6 * top)
        rel = np.maximum(err[sel] - slack[sel], 0.0) / np.maximum(np.abs(fd[sel]), floor)
        print("%-5s n=%3d  median rel %.2e  99%% %.2e  max %.2e" % (name, sel.sum(), np.median(rel),
                                                                   np.quantile(rel, 0.99), rel.max()))
        # float32 accumulation over ~10^3 terms per entry: 1e-3 relative to the floored magnitude
        assert np.all(rel <= 1e-3), (name, rel.max())
