"""Pins for the FP64 oracle against facts fixed by the paper and by mathematics,
not against the oracle's own formulas.

- Conventions against library routines: quaternion -> rotation and
  axis-angle -> rotation against scipy's Rotation; Adam against torch.optim.Adam.
- Eq. 1 / Eq. 3 (the PSF integral) against dense numerical quadrature of the
  convolution; this pins Eq. 4 and the normalisation of the closed form.
- Closed forms: a lone isotropic Gaussian read at its mean; an axis-aligned
  Gaussian as a product of 1-D convolutions (variances add); Sigma_PSF -> 0
  reduces to the volume value of Eq. 2's numerator.
- Invariants: mass conservation of the blurred field (true only with the exact
  normalisation), linearity in the amplitudes, and joint rigid motion of volume
  and slices (Sec. 2.4) leaving every prediction unchanged.
- Gradients against float64 central finite differences of the loss.
- The sampler's counter generator against SplitMix64's published first output,
  and its permutation property by brute force.
"""
import numpy as np
import pytest
from scipy.spatial.transform import Rotation

from paper_2512_11624_b300 import inputs

SIG = 1.0 / 2.355


def wxyz_to_scipy(q):
    return np.array([q[1], q[2], q[3], q[0]])


def scipy_cov(q, ls):
    R = Rotation.from_quat(wxyz_to_scipy(q)).as_matrix()
    return R @ np.diag(np.exp(2 * np.asarray(ls))) @ R.T


def theta_of(mu, ls, q, c, pose):
    mu, ls, q = np.atleast_2d(mu), np.atleast_2d(ls), np.atleast_2d(q)
    return np.concatenate([mu.T.reshape(-1), ls.T.reshape(-1), q.T.reshape(-1), np.atleast_1d(c),
                           np.asarray(pose, np.float64).reshape(-1)])


def sim_frames(stacks, pose):
    """Slice frames built here with scipy (stack convention: slice k centred at
    origin + (k - (n-1)/2) * thickness * normal; R_i = Rot(r) R_stack)."""
    Rs, ts = [], []
    i = 0
    for s in stacks:
        for k in range(s["n_slices"]):
            c0 = s["origin"] + (k - 0.5 * (s["n_slices"] - 1)) * s["thickness"] * s["R"][:, 2]
            Q = Rotation.from_rotvec(pose[i, :3]).as_matrix()
            Rs.append(Q @ s["R"])
            ts.append(Q @ c0 + pose[i, 3:])
            i += 1
    return np.array(Rs), np.array(ts)


def pixel_world(stacks, pose, pix):
    Rs, ts = sim_frames(stacks, pose)
    out, sl = [], []
    base, i = 0, 0
    starts = []
    for s in stacks:
        for k in range(s["n_slices"]):
            starts.append((base, i, s))
            base += s["H"] * s["W"]
            i += 1
    for p in pix:
        for b0, i0, s in reversed(starts):
            if p >= b0:
                loc = p - b0
                a, b = divmod(loc, s["W"])
                u = np.array([(b - 0.5 * (s["W"] - 1)) * s["dx"], (a - 0.5 * (s["H"] - 1)) * s["dy"], 0.0])
                out.append(Rs[i0] @ u + ts[i0])
                sl.append(i0)
                break
    return np.array(out), np.array(sl), Rs


# ----------------------------------------------------------------------- conventions
def test_quaternion_matches_scipy(oracle):
    rng = np.random.default_rng(1)
    for _ in range(20):
        q = rng.normal(size=4) * rng.uniform(0.2, 3.0)
        R = oracle.quat_to_rot(q)
        ref = Rotation.from_quat(wxyz_to_scipy(q / np.linalg.norm(q))).as_matrix()
        assert np.abs(R - ref).max() < 1e-14


@pytest.mark.parametrize("scale", [0.0, 1e-9, 1e-5, 3e-3, 0.2, 1.5, 3.0])
def test_rodrigues_matches_scipy(oracle, scale):
    rng = np.random.default_rng(2)
    for _ in range(5):
        r = rng.normal(size=3)
        r = r / np.linalg.norm(r) * scale
        assert np.abs(oracle.rodrigues(r) - Rotation.from_rotvec(r).as_matrix()).max() < 1e-14


def test_covariance_is_R_S_St_Rt(oracle):
    """Sec. 2.2: Sigma = R S S^T R^T with log-space scales."""
    rng = np.random.default_rng(3)
    N = 7
    th = inputs.random_gaussians(rng, N)
    S = oracle.gauss_cov(th, N)
    for j in range(N):
        q = th[6 * N + j:10 * N:N]
        ls = th[3 * N + j:6 * N:N]
        assert np.abs(S[j] - scipy_cov(q, ls)).max() < 1e-13


def test_slice_frames_vs_scipy(oracle):
    rng = np.random.default_rng(4)
    case = inputs.random_case(4, 3, [(3, 5, 7), (2, 4, 6)], n_stacks=2)
    M = inputs.n_slices_total(case["stacks"])
    pose = inputs.random_motion(rng, M, 20.0, 5.0)
    R, t = oracle.slice_frames(case["stacks"], pose)
    Rs, ts = sim_frames(case["stacks"], pose)
    assert np.abs(R - Rs).max() < 1e-13 and np.abs(t - ts).max() < 1e-12


def test_parameter_count(oracle):
    """11 parameters per primitive (Sec. 2.2; ~550k for N = 50k)."""
    rng = np.random.default_rng(0)
    assert inputs.random_gaussians(rng, 50_000).size == 550_000


# --------------------------------------------------------------- PSF integral (Eq. 1/3)
def quadrature_value(x_p, R_i, var, gauss, h=0.1, lim=8.0):
    """(V * phi)(x_p) by the trapezoid rule in PSF-whitened coordinates:
    E_z[V(x_p + R_i diag(sigma) z)], z ~ N(0, I), on [-lim, lim]^3."""
    z1 = np.arange(-lim, lim + 0.5 * h, h)
    w1 = np.exp(-0.5 * z1 ** 2) / np.sqrt(2 * np.pi) * h
    Z = np.stack(np.meshgrid(z1, z1, z1, indexing="ij"), -1).reshape(-1, 3)
    W = (w1[:, None, None] * w1[None, :, None] * w1[None, None, :]).reshape(-1)
    X = x_p[None, :] + (Z * np.sqrt(var)[None, :]) @ R_i.T
    V = np.zeros(X.shape[0])
    for mu, Sg, c in gauss:
        d = X - mu
        Pi = np.linalg.inv(Sg)
        V += c * np.exp(-0.5 * np.einsum("ni,ij,nj->n", d, Pi, d))
    return float((V * W).sum())


def test_closed_form_matches_quadrature(oracle):
    rng = np.random.default_rng(5)
    st = [inputs.stack(2, 5, 5, 1.0, 1.0, 3.0), inputs.stack(1, 5, 5, 0.8, 0.8, 2.5,
                                                               Rotation.random(random_state=9).as_matrix())]
    M = 3
    pose = inputs.random_motion(rng, M, 8.0, 2.0)
    N = 3
    pix = np.array([3, 12, 27, 61])
    xw, sl, Rs = pixel_world(st, pose, pix)
    mu = xw[[0, 1, 3]] + rng.normal(0.0, 0.7, size=(3, 3))
    ls = rng.uniform(np.log(0.5), np.log(2.0), size=(3, 3))
    q = rng.normal(size=(3, 4))
    c = rng.uniform(0.2, 1.0, 3)
    th = theta_of(mu, ls, q, c, pose)
    pred, _ = oracle.forward(st, th, N, pix)
    gauss = [(mu[j], scipy_cov(q[j], ls[j]), c[j]) for j in range(N)]
    vars_ = [np.array([1.2 * 1.0 * SIG, 1.2 * 1.0 * SIG, 3.0 * SIG]) ** 2] * 2 + \
            [np.array([1.2 * 0.8 * SIG, 1.2 * 0.8 * SIG, 2.5 * SIG]) ** 2]
    for k, p in enumerate(pix):
        ref = quadrature_value(xw[k], Rs[sl[k]], vars_[sl[k]], gauss)
        assert abs(pred[k] - ref) <= 1e-9 * abs(ref), (k, pred[k], ref)


def test_lone_gaussian_at_its_mean(oracle):
    """Isotropic s^2 I under PSF diag(a^2, a^2, b^2): c s^3 / ((s^2 + a^2) sqrt(s^2 + b^2));
    the literal substitution gives c; with no PSF both give c."""
    s, c = 1.3, 0.77
    st = [inputs.stack(1, 5, 5, 1.0, 1.0, 3.0, origin=(2.0, -1.0, 0.5))]
    th = theta_of([2.0, -1.0, 0.5], [np.log(s)] * 3, [0.3, -0.2, 0.5, 0.1], c, np.zeros(6))
    pix = np.array([12])  # centre pixel of a 5 x 5 slice sits at the origin of the stack
    a, b = 1.2 * SIG, 3.0 * SIG
    v, _ = oracle.forward(st, th, 1, pix)
    assert abs(v[0] - c * s ** 3 / ((s * s + a * a) * np.sqrt(s * s + b * b))) < 1e-15
    v, _ = oracle.forward(st, th, 1, pix, norm_mode=1)
    assert abs(v[0] - c) < 1e-15
    st[0]["fwhm"] = np.zeros(3)
    for mode in (0, 1):
        v, _ = oracle.forward(st, th, 1, pix, norm_mode=mode)
        assert abs(v[0] - c) < 1e-15


def test_axis_aligned_is_product_of_1d_convolutions(oracle):
    """q = identity, slice normal along z: each axis convolves independently
    (1-D Gaussian convolution: variances add, mass is kept)."""
    rng = np.random.default_rng(6)
    st = [inputs.stack(3, 6, 7, 0.9, 1.1, 2.8, origin=(0.3, -0.2, 0.1))]
    s = np.array([0.7, 1.6, 1.1])
    mu = np.array([0.9, -1.4, 1.3])
    c = 0.6
    th = theta_of(mu, np.log(s), [1.0, 0.0, 0.0, 0.0], c, np.zeros(18))
    pix = rng.choice(3 * 42, 12, replace=False)
    pred, _ = oracle.forward(st, th, 1, pix)
    var = (np.array([1.2 * 0.9, 1.2 * 1.1, 2.8]) * SIG) ** 2
    for k, p in enumerate(pix):
        sl, loc = divmod(p, 42)
        a, b = divmod(loc, 7)
        x = np.array([(b - 3.0) * 0.9 + 0.3, (a - 2.5) * 1.1 - 0.2, (sl - 1.0) * 2.8 + 0.1])
        ref = c
        for ax in range(3):
            tot = s[ax] ** 2 + var[ax]
            ref *= s[ax] / np.sqrt(tot) * np.exp(-0.5 * (x[ax] - mu[ax]) ** 2 / tot)
        assert abs(pred[k] - ref) <= 1e-13 * max(abs(ref), 1e-300) + 1e-300


def test_zero_psf_is_volume_value(oracle):
    """Sigma_PSF = 0: the pixel reads V(x) = sum_j c_j exp(-1/2 (x-mu)^T Sigma_j^-1 (x-mu))."""
    rng = np.random.default_rng(7)
    case = inputs.random_case(7, 25, [(2, 6, 5)], n_stacks=2)
    st = case["stacks"]
    for s in st:
        s["fwhm"] = np.zeros(3)
    N = case["N"]
    th = case["theta"].astype(np.float64)
    M = inputs.n_slices_total(st)
    pose = th[11 * N:].reshape(M, 6)
    pix = rng.choice(inputs.n_pixels_total(st), 15, replace=False)
    pred, _ = oracle.forward(st, th, N, pix)
    xw, _, _ = pixel_world(st, pose, pix)
    for k in range(len(pix)):
        ref = 0.0
        for j in range(N):
            q = th[6 * N + j:10 * N:N]
            ls = th[3 * N + j:6 * N:N]
            d = xw[k] - th[j:3 * N:N]
            ref += th[10 * N + j] * np.exp(-0.5 * d @ np.linalg.solve(scipy_cov(q, ls), d))
        assert abs(pred[k] - ref) <= 1e-12 * abs(ref) + 1e-300


@pytest.mark.slow
def test_mass_conservation(oracle):
    """Convolution with a unit-mass PSF keeps the mass c (2 pi)^(3/2) sqrt(det Sigma_j):
    sum of the blurred field over a fine 3D grid of pixels.  The literal
    substitution (no normalisation factor) gains mass sqrt(det Sigma_obs / det Sigma_j)."""
    h = 0.25
    n = 96
    st = [inputs.stack(n, n, n, h, h, h)]
    st[0]["fwhm"] = np.array([0.6, 0.4, 0.7])  # wider than a pixel, as a thick-slice PSF
    ls = np.log([1.0, 1.2, 0.8])
    q = np.array([0.9, 0.2, -0.3, 0.25])
    c = 0.7
    th = theta_of([0.05, -0.1, 0.07], ls, q, c, np.zeros(6 * n))
    pix = np.arange(n * n * n)
    pred, _ = oracle.forward(st, th, 1, pix)
    mass_ref = c * (2 * np.pi) ** 1.5 * np.exp(ls.sum())
    assert abs(pred.sum() * h ** 3 - mass_ref) <= 1e-6 * mass_ref
    pred1, _ = oracle.forward(st, th, 1, pix, norm_mode=1)
    So = scipy_cov(q, ls) + np.diag((st[0]["fwhm"] * SIG) ** 2)
    lit = c * (2 * np.pi) ** 1.5 * np.sqrt(np.linalg.det(So))
    assert abs(pred1.sum() * h ** 3 - lit) <= 1e-6 * lit
    assert lit > 1.01 * mass_ref


def test_linearity_in_amplitudes(oracle):
    case = inputs.random_case(8, 40, [(3, 7, 9)], n_stacks=2)
    N, st = case["N"], case["stacks"]
    th = case["theta"].astype(np.float64)
    rng = np.random.default_rng(8)
    c1 = rng.normal(size=N)
    c2 = rng.normal(size=N)
    pix = np.arange(inputs.n_pixels_total(st))
    preds = []
    for c in (c1, c2, 0.7 * c1 - 1.9 * c2):
        t = th.copy()
        t[10 * N:11 * N] = c
        preds.append(oracle.forward(st, t, N, pix)[0])
    lin = 0.7 * preds[0] - 1.9 * preds[1]
    assert np.abs(preds[2] - lin).max() <= 1e-12 * np.abs(lin).max()


def rigid_transform(th, N, M, Q, b):
    th = th.astype(np.float64).copy()
    mu = th[:3 * N].reshape(3, N).T
    th[:3 * N] = (mu @ Q.T + b).T.reshape(-1)
    q = th[6 * N:10 * N].reshape(4, N).T
    rq = Rotation.from_matrix(Q) * Rotation.from_quat(np.stack([q[:, 1], q[:, 2], q[:, 3], q[:, 0]], 1))
    qs = rq.as_quat()
    th[6 * N:10 * N] = np.stack([qs[:, 3], qs[:, 0], qs[:, 1], qs[:, 2]], 0).reshape(-1)
    pose = th[11 * N:].reshape(M, 6)
    for i in range(M):
        R = Q @ Rotation.from_rotvec(pose[i, :3]).as_matrix()
        pose[i, :3] = Rotation.from_matrix(R).as_rotvec()
        pose[i, 3:] = Q @ pose[i, 3:] + b
    th[11 * N:] = pose.reshape(-1)
    return th


def test_joint_rigid_motion_invariance(oracle):
    """Moving the volume and every slice by the same rigid map (Q, b) changes no
    prediction (Sec. 2.4: the PSF rotates with the slice)."""
    case = inputs.random_case(9, 60, [(3, 8, 9), (2, 7, 6)], n_stacks=2)
    N, st = case["N"], case["stacks"]
    M = inputs.n_slices_total(st)
    th = case["theta"].astype(np.float64)
    pix = np.arange(inputs.n_pixels_total(st))
    p0, _ = oracle.forward(st, th, N, pix)
    Q = Rotation.from_rotvec([0.3, -0.5, 0.2]).as_matrix()
    th2 = rigid_transform(th, N, M, Q, np.array([1.5, -2.0, 0.7]))
    p1, _ = oracle.forward(st, th2, N, pix)
    assert np.abs(p1 - p0).max() <= 1e-12 * np.abs(p0).max()


# -------------------------------------------------------------------- gradients
@pytest.mark.parametrize("norm_mode", [0, 1])
def test_gradient_matches_central_differences(oracle, norm_mode):
    case = inputs.random_case(10, 20, [(2, 6, 6), (1, 5, 7)], n_stacks=2, extent=3.0, motion_deg=10.0)
    N, st = case["N"], case["stacks"]
    th = case["theta"].astype(np.float64)
    pix = np.arange(inputs.n_pixels_total(st))
    I = case["I"].astype(np.float64)[pix]
    w = 1.0 / len(pix)
    _, L0, g, _ = oracle.forward_backward(st, th, N, pix, I, w, norm_mode=norm_mode)
    fd = np.zeros_like(g)
    for e in range(th.size):
        h = 1e-6 * max(1.0, abs(th[e]))
        tp, tm = th.copy(), th.copy()
        tp[e] += h
        tm[e] -= h
        fd[e] = (oracle.forward(st, tp, N, pix, I, w, norm_mode)[1] -
                 oracle.forward(st, tm, N, pix, I, w, norm_mode)[1]) / (2 * h)
    err = np.abs(g - fd)
    assert np.all(err <= 1e-6 * np.abs(g) + 1e-9 * np.abs(g).max()), (err.max(), np.argmax(err))


def test_absgrad_bounds_gradient(oracle):
    case = inputs.random_case(11, 30, [(2, 6, 6)], n_stacks=2, extent=4.0)
    N, st = case["N"], case["stacks"]
    th = case["theta"].astype(np.float64)
    pix = np.arange(inputs.n_pixels_total(st))
    _, _, g, a = oracle.forward_backward(st, th, N, pix, case["I"][pix], 1.0 / len(pix))
    assert np.all(np.abs(g) <= a * (1 + 1e-12) + 1e-300)


# ------------------------------------------------------------------------- Adam
def test_adam_matches_torch(oracle):
    import torch
    rng = np.random.default_rng(12)
    N, M = 5, 3
    n = 11 * N + 6 * M
    th = rng.normal(size=n)
    lr = np.array([2.5e-2, 2.5e-2, 1e-2, 1e-2, 2.5e-3, 1e-1])
    groups_idx = [np.arange(0, 3 * N), np.arange(3 * N, 6 * N), np.arange(6 * N, 10 * N), np.arange(10 * N, 11 * N)]
    pose_idx = np.arange(11 * N, n).reshape(M, 6)
    groups_idx += [pose_idx[:, :3].reshape(-1), pose_idx[:, 3:].reshape(-1)]
    params = [torch.tensor(th[ix], dtype=torch.float64, requires_grad=True) for ix in groups_idx]
    opt = torch.optim.Adam([{"params": [p], "lr": float(l)} for p, l in zip(params, lr)], betas=(0.9, 0.999),
                           eps=1e-8, weight_decay=0.0)
    m = np.zeros(n)
    v = np.zeros(n)
    cur = th.copy()
    for t in range(1, 4):
        g = rng.normal(size=n) * (10.0 ** rng.uniform(-3, 1, size=n))
        for p, ix in zip(params, groups_idx):
            p.grad = torch.tensor(g[ix], dtype=torch.float64)
        opt.step()
        cur, m, v = oracle.adam(N, M, cur, g, m, v, lr, 0.9, 0.999, 1e-8, t)
        ref = np.zeros(n)
        for p, ix in zip(params, groups_idx):
            ref[ix] = p.detach().numpy()
        assert np.abs(cur - ref).max() <= 1e-13 * np.abs(ref).max()


def test_adam_frozen_slice_keeps_pose(oracle):
    rng = np.random.default_rng(13)
    N, M = 2, 3
    n = 11 * N + 6 * M
    th = rng.normal(size=n)
    fz = np.array([0, 1, 0], np.uint8)
    out, _, _ = oracle.adam(N, M, th, rng.normal(size=n), np.zeros(n), np.zeros(n), np.full(6, 0.1), 0.9, 0.999,
                            1e-8, 1, fz)
    sl = slice(11 * N + 6, 11 * N + 12)
    assert np.array_equal(out[sl], th[sl])
    assert not np.array_equal(out[11 * N:11 * N + 6], th[11 * N:11 * N + 6])


# ---------------------------------------------------------------------- sampler
def test_splitmix64_published_first_output(oracle):
    """SplitMix64 from state 0: first output 0xE220A8397B1DCDAF (Steele et al. 2014)."""
    assert oracle.splitmix64(0, 0) == 0xE220A8397B1DCDAF


@pytest.mark.parametrize("n", [1, 2, 3, 5, 64, 100, 1000, 4097])
def test_sampler_is_a_permutation(oracle, n):
    for step in (0, 1, 7):
        pos = oracle.sample_positions(n, n, 1234, step)
        assert np.array_equal(np.sort(pos), np.arange(n))


def test_sampler_subset_uniform(oracle):
    n, k = 1000, 100
    counts = np.zeros(n)
    for step in range(400):
        pos = oracle.sample_positions(n, k, 99, step)
        assert len(np.unique(pos)) == k and pos.min() >= 0 and pos.max() < n
        counts[pos] += 1
    # each element is drawn with probability k/n = 0.1 per step: mean 40, sd ~6
    assert abs(counts.mean() - 40.0) < 1e-9
    assert counts.std() < 9.0 and counts.min() > 10 and counts.max() < 75


def test_truncation_sums(oracle):
    """Sums over pairs below a cutoff: 0 for a cutoff below every pair factor, equal
    to the full sums of |terms| for a cutoff above every factor (factor <= 1)."""
    case = inputs.random_case(21, 15, [(2, 7, 8)], n_stacks=2, extent=5.0)
    N, st = case["N"], case["stacks"]
    th = case["theta"].astype(np.float64)
    pix = np.arange(inputs.n_pixels_total(st))
    I = case["I"].astype(np.float64)
    r0 = oracle.forward_backward(st, th, N, pix, I, 1.0 / len(pix), cutoff=1e-300)
    assert np.all(r0[4] == 0.0) and np.all(r0[5] == 0.0)
    r1 = oracle.forward_backward(st, th, N, pix, I, 1.0 / len(pix), cutoff=1.5)
    assert np.allclose(r1[5], r1[3], rtol=1e-12, atol=0)
    assert np.allclose(r1[4], np.abs(r1[0]), rtol=1e-12)  # positive amplitudes
    r2 = oracle.forward_backward(st, th, N, pix, I, 1.0 / len(pix), cutoff=1e-3)
    assert np.all(r2[5] <= r2[3] * (1 + 1e-12)) and np.all(r2[4] <= np.abs(r2[0]) * (1 + 1e-12))


# ----------------------------------------------------- paper objective (L1 + scale regulariser)
def test_l1_and_scale_regulariser_match_central_differences(oracle):
    """The paper's loss (Sec. 2.5): sum of |I - I_hat| plus lambda_reg times
    sum_j |s_j - s_target|^2 (scales in mm).  Value against a direct numpy
    evaluation from the oracle's predictions; gradient against central
    differences (residuals away from the L1 kink)."""
    case = inputs.random_case(14, 10, [(2, 5, 6)], n_stacks=2, extent=3.0, motion_deg=10.0)
    N, st = case["N"], case["stacks"]
    th = case["theta"].astype(np.float64)
    pix = np.arange(inputs.n_pixels_total(st))
    I = case["I"].astype(np.float64)[pix] + 0.05
    w, lam, s_t = 1.0 / len(pix), 2.5e-3, 1.6
    pred, L = oracle.forward(st, th, N, pix, I, w, loss_kind=1, lambda_reg=lam, s_target=s_t)
    scales = np.exp(th[3 * N:6 * N])
    assert np.isclose(L, w * np.abs(pred - I).sum() + lam * ((scales - s_t) ** 2).sum(), rtol=1e-13)
    assert np.abs(pred - I).min() > 1e-4
    _, L0, g, _ = oracle.forward_backward(st, th, N, pix, I, w, loss_kind=1, lambda_reg=lam, s_target=s_t)
    assert np.isclose(L0, L, rtol=1e-13)
    fd = np.zeros_like(g)
    for e in range(th.size):
        h = 1e-6 * max(1.0, abs(th[e]))
        tp, tm = th.copy(), th.copy()
        tp[e] += h
        tm[e] -= h
        fd[e] = (oracle.forward(st, tp, N, pix, I, w, loss_kind=1, lambda_reg=lam, s_target=s_t)[1] -
                 oracle.forward(st, tm, N, pix, I, w, loss_kind=1, lambda_reg=lam, s_target=s_t)[1]) / (2 * h)
    err = np.abs(g - fd)
    assert np.all(err <= 1e-6 * np.abs(g) + 1e-9 * np.abs(g).max()), (err.max(), np.argmax(err))


@pytest.mark.parametrize("loss_kind", [0, 1])
def test_slice_scale_and_aleatoric_weight(oracle, loss_kind):
    """The per-slice outlier terms of Sec. 2.4 (log sigma_i, log omega_i): the
    prediction is exactly sigma_i times the plain one; the weight's gradient
    vanishes at omega_i = the slice's mean pixel loss (the minimiser of
    l / omega + log omega); all gradients against central differences."""
    case = inputs.random_case(16, 8, [(2, 5, 6), (1, 4, 5)], n_stacks=2, extent=3.0, motion_deg=10.0)
    N, st = case["N"], case["stacks"]
    M = inputs.n_slices_total(st)
    th = case["theta"].astype(np.float64)
    pix = np.arange(inputs.n_pixels_total(st))
    I = case["I"].astype(np.float64)[pix] + 0.05
    w = 1.0 / len(pix)
    rng = np.random.default_rng(3)
    slw = np.concatenate([rng.normal(0, 0.2, M), rng.normal(0, 0.5, M)])
    p0, _ = oracle.forward(st, th, N, pix, I, w, loss_kind=loss_kind)
    p1, _ = oracle.forward(st, th, N, pix, I, w, loss_kind=loss_kind, slw=slw)
    sl = np.searchsorted(np.cumsum([0] + [s["H"] * s["W"] for s in st for _ in range(s["n_slices"])])[1:], pix,
                         side="right")
    assert np.allclose(p1, np.exp(slw[sl]) * p0, rtol=1e-14, atol=0)
    # omega at the slice's mean loss: zero derivative
    r = np.exp(slw[sl]) * p0 - I
    l = w * (np.abs(r) if loss_kind else r * r)
    opt = slw.copy()
    opt[M:] = np.log(np.bincount(sl, l, M) / np.bincount(sl, np.full(len(pix), w), M))
    gs = np.zeros(2 * M)
    oracle.forward_backward(st, th, N, pix, I, w, loss_kind=loss_kind, slw=opt, slw_grad=gs)
    assert np.abs(gs[M:]).max() <= 1e-12
    # central differences in theta and in the slice terms
    gs = np.zeros(2 * M)
    _, L0, g, _ = oracle.forward_backward(st, th, N, pix, I, w, loss_kind=loss_kind, slw=slw, slw_grad=gs)
    full = np.concatenate([g, gs])
    x0 = np.concatenate([th, slw])
    n = th.size

    def L(x):
        return oracle.forward(st, x[:n], N, pix, I, w, loss_kind=loss_kind, slw=x[n:])[1]
    fd = np.zeros_like(full)
    for e in range(x0.size):
        h = 1e-6 * max(1.0, abs(x0[e]))
        xp, xm = x0.copy(), x0.copy()
        xp[e] += h
        xm[e] -= h
        fd[e] = (L(xp) - L(xm)) / (2 * h)
    err = np.abs(full - fd)
    assert np.all(err <= 1e-6 * np.abs(full) + 1e-9 * np.abs(full).max()), (err.max(), np.argmax(err))
