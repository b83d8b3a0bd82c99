"""Content-adaptive initialisation of the means on the GPU (gsvr_init_means,
Sec. 2.5) against the oracle of oracle/init.py: the drawn pixels bit for bit
(the draw is an integer decision both sides take in the same arithmetic), the
total weight exactly, the means within float32 rounding of the slice frames
(2e-5 mm + 1e-6 relative); on a small moving case and on the fetal workload
(200,000 draws, 1,000 means checked); argument and empty-weight checks."""
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


@pytest.fixture(scope="module")
def ini():
    from oracle import init
    return init


def check(G, ini, case, n, lam, seed, sub=None):
    st = case["stacks"]
    M = inputs.n_slices_total(st)
    pose = case["theta"][11 * case["N"]:].astype(np.float32).reshape(M, 6)
    ctx = G.Context(case)
    mu, pix, T = G.gsvr_init_means(ctx.ctx, n, lam, seed, pose=pose)
    mu, pix = mu.cpu().numpy().astype(np.float64), pix.cpu().numpy().astype(np.int64)
    ctx.close()
    W = ini.weights(st, case["I"], case["mask"], lam)
    assert T == int(W.sum())
    ks = np.arange(n) if sub is None else sub
    assert np.array_equal(pix[ks], ini.draw_pixels(W, ks, seed))
    ref, rpix = ini.init_means(st, case["I"], case["mask"], pose.astype(np.float64), n, lam, seed, ks=ks)
    assert np.array_equal(rpix, pix[ks])
    err = np.abs(mu[:, ks].T - ref)
    assert np.all(err <= 2e-5 + 1e-6 * np.abs(ref)), err.max()
    return pix


@pytest.mark.parametrize("lam", [0.0, 0.3, 1.0])
def test_small_case(G, ini, lam):
    case = inputs.random_case(51, 40, [(3, 17, 21), (2, 13, 11)], n_stacks=2, motion_deg=8.0)
    pix = check(G, ini, case, 5000, lam, 11)
    if lam == 1.0:  # every masked pixel equally likely
        m = np.flatnonzero(case["mask"])
        counts = np.bincount(pix, minlength=len(case["mask"]))[m]
        assert counts.std() < 4 * np.sqrt(5000 / len(m))


def test_fetal_workload(G, ini):
    case = inputs.fetal(0)
    rng = np.random.default_rng(2)
    check(G, ini, case, 200000, 0.0, 5, sub=np.sort(rng.choice(200000, 1000, replace=False)))


def test_errors(G):
    case = inputs.random_case(52, 10, [(1, 6, 6)], n_stacks=1)
    ctx = G.Context(case)
    for n, lam in [(-1, 0.0), (10, -0.1), (10, 1.5)]:
        with pytest.raises(G.GsvrError) as e:
            G.gsvr_init_means(ctx.ctx, n, lam, 0)
        assert "INVALID_ARG" in str(e.value)
    ctx.close()
    flat = dict(case)
    flat["I"] = np.zeros_like(case["I"])
    ctx = G.Context(flat)
    with pytest.raises(G.GsvrError) as e:
        G.gsvr_init_means(ctx.ctx, 10, 0.0, 0)
    assert "INVALID_ARG" in str(e.value)
    mu, pix, T = G.gsvr_init_means(ctx.ctx, 10, 0.5, 0)  # the uniform part still draws
    assert T > 0
    ctx.close()
