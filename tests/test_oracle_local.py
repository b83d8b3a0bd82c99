"""Pins of the oracle's large-case path (grid neighbour search, local central
differences) against its brute-force all-pairs path on small random cases:
predictions equal the all-pairs sum up to the terms below the 1e-12 cut, and
the local differences equal the analytic all-pairs gradient for every kind of
parameter (mu, log-scales, quaternion, amplitude, slice rotation, slice
translation)."""
import numpy as np

from paper_2512_11624_b300 import inputs


def test_local_fd_matches_all_pairs(oracle):
    case = inputs.random_case(31, 60, [(3, 14, 12), (2, 11, 13)], n_stacks=2, motion_deg=8.0, motion_mm=3.0)
    N = case["N"]
    M = inputs.n_slices_total(case["stacks"])
    th = case["theta"].astype(np.float64)
    P = inputs.n_pixels_total(case["stacks"])
    rng = np.random.default_rng(1)
    pix = np.sort(rng.choice(P, size=P // 2, replace=False))
    I = case["I"].astype(np.float64)[pix]
    w = 1.0 / pix.size
    pred_ref, L, g, a, tp, tg = oracle.forward_backward(case["stacks"], th, N, pix, I, w, cutoff=1e-12)
    params = np.concatenate([rng.choice(11 * N, 60, replace=False), 11 * N + rng.choice(6 * M, 24, replace=False)])
    scale = np.where(params >= 10 * N, np.maximum(np.abs(th[params]), 1e-2), 1.0)
    scale[params >= 11 * N] = 1.0
    h = 1e-5 * scale
    fd, pred, trunc = oracle.local_fd(case["stacks"], th, N, pix, I, w, params, h, cut=1e-12, trunc_cut=1e-7)
    assert np.allclose(pred, pred_ref, rtol=1e-10, atol=1e-12 * np.abs(pred_ref).max())
    assert np.all(trunc >= 0) and np.all(trunc <= np.abs(pred_ref).max())
    err = np.abs(fd - g[params])
    assert np.all(err <= 1e-6 * np.abs(g[params]) + 1e-9 * np.abs(g).max()), (err.max(), np.abs(g[params]).max())


def _check_local_grad(oracle, case, pix, sel):
    N = case["N"]
    M = inputs.n_slices_total(case["stacks"])
    th = case["theta"].astype(np.float64)
    I = case["I"].astype(np.float64)[pix]
    w = 1.0 / pix.size
    pred_ref, L, g, a, tp, tg = oracle.forward_backward(case["stacks"], th, N, pix, I, w, cutoff=1e-7)
    # what the grid path drops: every pair below 1e-12 (per output, sum of |terms|)
    _, _, _, _, tp12, tg12 = oracle.forward_backward(case["stacks"], th, N, pix, I, w, cutoff=1e-12)
    out = oracle.local_grad(case["stacks"], th, N, pix, I, w, sel, cut=1e-12, trunc_cut=1e-7)
    comp, pose = oracle.select_entries(N, M, sel)
    assert np.all(np.abs(out["pred"] - pred_ref) <= 1e-12 * np.abs(pred_ref) + tp12 + 1e-300)
    assert np.allclose(out["trunc_pred"], tp - tp12, rtol=1e-9, atol=1e-300)
    assert abs(out["loss"] - L) <= 1e-10 * L
    # gradient and |terms|: equal up to the pairs below 1e-12 (and float64 rounding)
    for got, ref, A, T in ((out["g_sel"], g[comp], a[comp], tg12[comp]), (out["g_pose"], g[pose], a[pose], tg12[pose])):
        err = np.abs(got - ref)
        assert np.all(err <= 1e-9 * np.abs(ref) + 1e-13 * A + T + 1e-300), err.max()
    for got, ref, T in ((out["a_sel"], a[comp], tg12[comp]), (out["a_pose"], a[pose], tg12[pose])):
        assert np.all(np.abs(got - (ref - T)) <= 1e-9 * ref + 1e-300)
    # the sums below the 1e-7 cut: the all-pairs sums at 1e-7 minus those at 1e-12
    for got, ref, T in ((out["t_sel"], tg[comp], tg12[comp]), (out["t_pose"], tg[pose], tg12[pose])):
        assert np.all(np.abs(got - (ref - T)) <= 1e-9 * ref + 1e-300)
    assert np.all(out["t_sel"] <= out["a_sel"]) and np.all(out["t_pose"] <= out["a_pose"])
    return out


def test_local_grad_matches_all_pairs_random(oracle):
    """The grid-pruned analytic gradient (every pose entry, every component of
    selected Gaussians) equals the all-pairs analytic gradient, including the
    |term| scales and the sums below the 1e-7 cut, on two random geometries
    with oblique stacks and motion (exact normalisation)."""
    for seed, N, sizes in ((31, 60, [(3, 14, 12), (2, 11, 13)]), (7, 150, [(4, 17, 9), (3, 10, 21)])):
        case = inputs.random_case(seed, N, sizes, n_stacks=2, motion_deg=8.0, motion_mm=3.0)
        P = inputs.n_pixels_total(case["stacks"])
        rng = np.random.default_rng(seed)
        pix = np.sort(rng.choice(P, size=(2 * P) // 3, replace=False))
        sel = np.sort(rng.choice(N, size=N // 2, replace=False))
        out = _check_local_grad(oracle, case, pix, sel)
        assert np.abs(out["g_pose"]).max() > 0 and np.abs(out["g_sel"]).max() > 0


def test_local_grad_matches_all_pairs_tiny(oracle):
    """The same on the 2,000-Gaussian tiny workload, every pixel, 300 selected
    Gaussians."""
    case = inputs.tiny(0)
    P = inputs.n_pixels_total(case["stacks"])
    sel = np.sort(np.random.default_rng(3).choice(case["N"], size=300, replace=False))
    _check_local_grad(oracle, case, np.arange(P), sel)


def test_local_grad_prediction_scale_sums(oracle):
    """b_sel / b_pose are the |term| sums taken with each residual weight
    replaced by 2 w sum_j |c_j g_pj|.  With positive amplitudes that is
    2 w I_hat_p, the residual weight of zero observations, so they equal the
    all-pairs oracle's |term| sums at I = 0 (up to the pairs below 1e-12)."""
    case = inputs.random_case(12, 90, [(3, 13, 15), (2, 12, 11)], n_stacks=2, motion_deg=8.0, motion_mm=3.0)
    N = case["N"]
    M = inputs.n_slices_total(case["stacks"])
    th = case["theta"].astype(np.float64)
    assert np.all(th[10 * N:11 * N] > 0)
    P = inputs.n_pixels_total(case["stacks"])
    rng = np.random.default_rng(4)
    pix = np.sort(rng.choice(P, size=P // 2, replace=False))
    sel = np.sort(rng.choice(N, size=40, replace=False))
    w = 1.0 / pix.size
    I = case["I"].astype(np.float64)[pix]
    out = oracle.local_grad(case["stacks"], th, N, pix, I, w, sel, cut=1e-12, trunc_cut=1e-7)
    zero = np.zeros(pix.size)
    _, _, _, a0, _, t12 = oracle.forward_backward(case["stacks"], th, N, pix, zero, w, cutoff=1e-12)
    comp, pose = oracle.select_entries(N, M, sel)
    for got, ref, T in ((out["b_sel"], a0[comp], t12[comp]), (out["b_pose"], a0[pose], t12[pose])):
        assert np.all(np.abs(got - ref) <= 1e-9 * ref + 2 * T + 1e-300), np.abs(got - ref).max()
    # and they do not depend on the observations (float64 sums in a thread-dependent order)
    out0 = oracle.local_grad(case["stacks"], th, N, pix, zero, w, sel, cut=1e-12, trunc_cut=1e-7)
    assert np.allclose(out0["b_sel"], out["b_sel"], rtol=1e-12) and np.allclose(out0["b_pose"], out["b_pose"],
                                                                                 rtol=1e-12)
    assert np.allclose(out0["a_sel"], out["b_sel"], rtol=1e-12) and np.allclose(out0["a_pose"], out["b_pose"],
                                                                                rtol=1e-12)


def test_local_grad_truncation_scale_sums(oracle):
    """bt_sel / bt_pose are the |term| sums with each residual weight replaced
    by 2 w trunc_pred_p; with observations I_p = I_hat_p - trunc_pred_p that is
    the residual weight itself, so they equal that call's a_sel / a_pose."""
    case = inputs.random_case(13, 120, [(3, 14, 13), (2, 12, 12)], n_stacks=2, motion_deg=8.0, motion_mm=3.0,
                              s_hi=3.0)
    N = case["N"]
    th = case["theta"].astype(np.float64)
    P = inputs.n_pixels_total(case["stacks"])
    rng = np.random.default_rng(6)
    pix = np.sort(rng.choice(P, size=P // 2, replace=False))
    sel = np.sort(rng.choice(N, size=50, replace=False))
    w = 1.0 / pix.size
    out = oracle.local_grad(case["stacks"], th, N, pix, case["I"].astype(np.float64)[pix], w, sel, cut=1e-12,
                            trunc_cut=1e-4)
    assert out["trunc_pred"].max() > 0 and out["bt_sel"].max() > 0
    out2 = oracle.local_grad(case["stacks"], th, N, pix, out["pred"] - out["trunc_pred"], w, sel, cut=1e-12,
                             trunc_cut=1e-4)
    assert np.allclose(out2["a_sel"], out["bt_sel"], rtol=1e-9, atol=1e-300)
    assert np.allclose(out2["a_pose"], out["bt_pose"], rtol=1e-9, atol=1e-300)
