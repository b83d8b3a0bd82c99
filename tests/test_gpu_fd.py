"""GPU gradients against central finite differences of the GPU's own loss
(float32 forward, float64 loss sum), on the parameters with the largest
gradient x scale: every group (mu, log-scales, quaternion, amplitude, slice
rotation, slice translation) is represented.  Step h = 1e-3 x the parameter's
scale; tolerance 1e-2 relative (the FD truncation error is O(h^2) and the
float32 forward is deterministic, so its rounding enters as ~1e-7 L / h)."""
import numpy as np
import pytest

from paper_2512_11624_b300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2512_11624_b300 import gsvr
    return gsvr


GROUPS = [("mu", 0, 3), ("ls", 3, 6), ("q", 6, 10), ("c", 10, 11)]


@pytest.mark.parametrize("seed", [21, 22])
def test_gradient_matches_central_differences(G, seed):
    import torch
    case = inputs.random_case(seed, 120, [(3, 26, 30), (2, 22, 18)], n_stacks=2, motion_deg=8.0, motion_mm=3.0)
    ctx = G.Context(case, tile_h=12, tile_w=12)
    N, M = case["N"], ctx.M
    theta0 = ctx.theta.clone()
    ctx.forward()
    ctx.backward()
    L0 = ctx.loss()
    g = ctx.grad.cpu().numpy().astype(np.float64)
    th = theta0.cpu().numpy().astype(np.float64)
    # scale per parameter: mm for mu and translation, 1 for log-scales, quaternions, rotations; |c| for amplitudes
    scale = np.ones_like(th)
    scale[:3 * N] = 1.0
    scale[10 * N:11 * N] = np.maximum(np.abs(th[10 * N:11 * N]), 1e-2)
    pose = np.arange(11 * N, 11 * N + 6 * M)
    scale[pose[(pose - 11 * N) % 6 >= 3]] = 1.0
    score = np.abs(g) * scale
    picks = []
    groups = [(a * N, b * N) for _, a, b in GROUPS] + [(11 * N + k, 11 * N + 6 * M) for k in (0, 3)]
    for lo, hi in groups:  # the strongest 20 of every group, then the strongest overall
        idx = np.arange(lo, hi) if lo < 11 * N else np.arange(lo, hi, 6)
        if lo >= 11 * N:
            idx = np.concatenate([idx + d for d in range(3)])
        picks += list(idx[np.argsort(-score[idx])[:20]])
    rest = np.setdiff1d(np.argsort(-score)[:200], picks)
    picks = np.array(picks + list(rest[:max(0, 200 - len(picks))]))
    worst = 0.0
    for k in picks:
        h = 1e-3 * scale[k]
        Ls = []
        for sgn in (1.0, -1.0):
            t = theta0.clone()
            t[k] += sgn * h
            ctx.theta.copy_(t)
            ctx.forward()
            Ls.append(ctx.loss())
        fd = (Ls[0] - Ls[1]) / (2 * h)
        lim = 1e-2 * abs(g[k]) + 2e-6 * L0 / h
        worst = max(worst, abs(fd - g[k]) / lim)
        assert abs(fd - g[k]) <= lim, (k, fd, g[k], lim)
    print("worst |fd - g| / limit over %d parameters: %.3f" % (len(picks), worst))
    ctx.theta.copy_(theta0)
    ctx.close()
