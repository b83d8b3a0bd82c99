"""Seeded synthetic input generators shared by the CUDA path's tests/benchmark and
the oracle's tests.

This module holds none of the method's arithmetic (no Gaussian evaluation, no
covariance addition, no gradient): it only draws parameters, builds stack
descriptions and simulates observations from an analytic phantom, on the CPU
with numpy.  It imports nothing else from this package, so importing it never
loads the CUDA library.

Workloads (shapes follow the paper's acquisitions: three orthogonal thick-slice
stacks, brain-sized field of view, motion of a few degrees / millimetres;
Sec. 3.2 "Data"):

- ``tiny``   2,000 Gaussians, 1 stack of 8 x 32 x 32 px (1 x 1 x 3 mm).
- ``fetal``  ~200k Gaussians on a 0.8 mm grid inside a brain-like phantom,
             3 orthogonal stacks of 40 x 192 x 192 px (1 x 1 x 3.5 mm),
             per-slice motion U(+-5 deg) / U(+-3 mm), Rician noise 2 %.
- ``random_case`` small random geometries for edge-case parity tests.

Stack dictionaries: ``n_slices, H, W, dx, dy, thickness`` (mm), ``R`` (3x3,
columns = slice x axis, slice y axis, slice normal in world coordinates),
``origin`` (3, world position of the stack centre), ``fwhm`` (3, PSF FWHM along
slice x, y and normal; in-plane 1.2 x pixel size, through-plane = thickness).
"""
from __future__ import annotations

import numpy as np
from scipy.spatial.transform import Rotation

FWHM_TO_SIGMA = 1.0 / 2.355


def stack(n_slices, H, W, dx, dy, thickness, R=None, origin=(0.0, 0.0, 0.0)):
    R = np.eye(3) if R is None else np.asarray(R, dtype=np.float64)
    return {"n_slices": int(n_slices), "H": int(H), "W": int(W), "dx": float(dx), "dy": float(dy),
            "thickness": float(thickness), "R": R.astype(np.float64),
            "origin": np.asarray(origin, np.float64),
            "fwhm": np.array([1.2 * dx, 1.2 * dy, thickness], np.float64)}


# Orthogonal stack orientations: columns = (slice x, slice y, normal).
AXIAL = np.eye(3)
CORONAL = np.array([[1.0, 0.0, 0.0], [0.0, 0.0, -1.0], [0.0, 1.0, 0.0]])   # normal = world y
SAGITTAL = np.array([[0.0, 0.0, 1.0], [1.0, 0.0, 0.0], [0.0, 1.0, 0.0]])   # normal = world x


def n_slices_total(stacks):
    return int(sum(s["n_slices"] for s in stacks))


def n_pixels_total(stacks):
    return int(sum(s["n_slices"] * s["H"] * s["W"] for s in stacks))


def random_gaussians(rng, N, lo=-16.0, hi=16.0, s_lo=0.5, s_hi=2.0):
    """Means U(lo, hi)^3, per-axis scales log-uniform [s_lo, s_hi], unit quaternions
    (normalised 4-D normal), amplitudes U(0, 1).  Returns the 11 N SoA vector."""
    mu = rng.uniform(lo, hi, size=(3, N))
    ls = rng.uniform(np.log(s_lo), np.log(s_hi), size=(3, N))
    q = rng.normal(size=(4, N))
    q /= np.linalg.norm(q, axis=0, keepdims=True)
    c = rng.uniform(0.0, 1.0, size=(1, N))
    return np.concatenate([mu, ls, q, c], axis=0).reshape(-1)


def random_motion(rng, M, max_deg, max_mm):
    """Per-slice motion (axis-angle r, translation tau): axis uniform on S^2,
    angle U(-max_deg, max_deg), tau ~ U(-max_mm, max_mm)^3.  Shape (M, 6)."""
    ax = rng.normal(size=(M, 3))
    ax /= np.linalg.norm(ax, axis=1, keepdims=True)
    ang = np.deg2rad(rng.uniform(-max_deg, max_deg, size=(M, 1)))
    tau = rng.uniform(-max_mm, max_mm, size=(M, 3))
    return np.concatenate([ax * ang, tau], axis=1)


def smooth_observations(rng, stacks, noise=0.01):
    """A smooth field over (slice, row, col) plus Gaussian noise, for the tiny and
    random cases (any values give a nonzero loss and gradient)."""
    out = []
    k0 = 0
    for s in stacks:
        n, H, W = s["n_slices"], s["H"], s["W"]
        k = np.arange(n)[:, None, None] + k0
        a = np.arange(H)[None, :, None]
        b = np.arange(W)[None, None, :]
        ph = rng.uniform(0, 2 * np.pi, 3)
        img = (0.45 + 0.2 * np.sin(0.31 * b + ph[0]) * np.cos(0.23 * a + ph[1])
               + 0.1 * np.sin(0.7 * k + ph[2]))
        out.append(img.reshape(-1))
        k0 += n
    I = np.concatenate(out)
    return (I + rng.normal(0.0, noise, size=I.shape)).astype(np.float32)


def tiny(seed=0):
    """The tiny plain case: 2,000 Gaussians, 1 axial stack of 8 x 32 x 32 px at
    1 x 1 mm, 3 mm thick (slice centres z = (k - 3.5) * 3), identity poses."""
    rng = np.random.default_rng(seed)
    N = 2000
    theta_g = random_gaussians(rng, N)
    stacks = [stack(8, 32, 32, 1.0, 1.0, 3.0)]
    M = n_slices_total(stacks)
    pose = np.zeros((M, 6))
    I = smooth_observations(rng, stacks)
    mask = np.ones(n_pixels_total(stacks), np.uint8)
    theta = np.concatenate([theta_g, pose.reshape(-1)]).astype(np.float32)
    return {"name": "tiny", "N": N, "stacks": stacks, "theta": theta, "I": I, "mask": mask,
            "n_sample": int(mask.sum())}


def random_case(seed, N, sizes, n_stacks=1, motion_deg=6.0, motion_mm=4.0, extent=None, s_lo=0.5, s_hi=2.0,
                thickness=3.0, dx=1.0):
    """Small random geometry: n_stacks stacks with random orientations (first
    axial), each of the given (n_slices, H, W); random Gaussians spread over the
    field of view; random per-slice motion; smooth observations."""
    rng = np.random.default_rng(seed)
    stacks = []
    for k in range(n_stacks):
        n, H, W = sizes[k % len(sizes)]
        R = np.eye(3) if k == 0 else Rotation.random(random_state=int(rng.integers(1 << 31))).as_matrix()
        origin = rng.uniform(-1.5, 1.5, 3)
        stacks.append(stack(n, H, W, dx, dx, thickness, R, origin))
    if extent is None:
        extent = 0.45 * min(min(s["H"], s["W"]) * s["dx"] for s in stacks)
    theta_g = random_gaussians(rng, N, -extent, extent, s_lo, s_hi)
    M = n_slices_total(stacks)
    pose = random_motion(rng, M, motion_deg, motion_mm)
    I = smooth_observations(rng, stacks)
    mask = np.ones(n_pixels_total(stacks), np.uint8)
    theta = np.concatenate([theta_g, pose.reshape(-1)]).astype(np.float32)
    return {"name": "random", "N": N, "stacks": stacks, "theta": theta, "I": I, "mask": mask,
            "n_sample": int(mask.sum())}


# --------------------------------------------------------------------------- phantom
class BrainPhantom:
    """Brain-like analytic phantom, intensities in [0, 1] (T2-like):
    background 0, CSF shell 0.95 between the outer ellipsoid and the cortex,
    folded cortex band 0.45 (2.5 mm thick), white matter 0.65, deep grey matter
    0.55, two ventricles 0.95.  Edges are logistic with a 0.3 mm width.
    Semi-axes (35, 28, 25) mm times ``scale``.  ``jitter`` > 0 draws a member
    of the same canonical-frame family: semi-axes times U(1 +- jitter), tissue
    levels times U(1 +- jitter / 1.5) (the fold pattern always varies with
    the seed)."""

    def __init__(self, seed=0, scale=1.0, jitter=0.0):
        rng = np.random.default_rng(seed + 7919)
        self.axes = np.array([35.0, 28.0, 25.0]) * scale
        self.scale = scale
        self.ka = rng.integers(2, 7, size=8).astype(np.float64)
        self.kb = rng.integers(1, 6, size=8).astype(np.float64)
        self.ph = rng.uniform(0, 2 * np.pi, size=8)
        self.width = 0.3
        # tissue levels: CSF, cortex, white matter, deep grey matter, ventricles
        self.levels = np.array([0.95, 0.45, 0.65, 0.55, 0.95])
        if jitter > 0:  # a member of the canonical-frame family: semi-axes and levels varied
            self.axes = self.axes * rng.uniform(1 - jitter, 1 + jitter, size=3)
            self.levels = self.levels * rng.uniform(1 - jitter / 1.5, 1 + jitter / 1.5, size=5)
        self.L = float(np.mean(self.axes))

    @staticmethod
    def _sig(z):
        return 0.5 * (1.0 + np.tanh(0.5 * z))

    def _ell(self, x, centre, axes):
        p = (x - np.asarray(centre)) / np.asarray(axes)
        rho = np.sqrt((p * p).sum(-1))
        return self._sig((1.0 - rho) * float(np.min(axes)) / self.width)

    def __call__(self, x):
        x = np.asarray(x, dtype=np.float64)
        p = x / self.axes
        rho = np.sqrt((p * p).sum(-1)) + 1e-12
        th = np.arccos(np.clip(p[..., 2] / rho, -1.0, 1.0))
        phi = np.arctan2(p[..., 1], p[..., 0])
        fold = np.ones_like(rho)
        for a, b, c in zip(self.ka, self.kb, self.ph):
            fold += 0.03 * np.sin(a * th + c) * np.cos(b * phi)
        rc_out = 0.93 * fold
        rc_in = rc_out - 2.5 / self.L
        k = self.L / self.width
        m_out = self._sig((1.0 - rho) * k)
        m_cx = self._sig((rc_out - rho) * k)
        m_wm = self._sig((rc_in - rho) * k)
        s = self.scale
        m_gm = self._ell(x, (0.0, 0.0, -2.0 * s), (12.0 * s, 8.0 * s, 6.0 * s))
        m_v = np.maximum(self._ell(x, (6.0 * s, 2.0 * s, 4.0 * s), (3.5 * s, 9.0 * s, 4.0 * s)),
                         self._ell(x, (-6.0 * s, 2.0 * s, 4.0 * s), (3.5 * s, 9.0 * s, 4.0 * s)))
        csf, ctx_, wm, dgm, ven = self.levels
        inner = wm * (1 - m_gm) + dgm * m_gm
        inner = inner * (1 - m_v) + ven * m_v
        cx = ctx_ * (1 - m_wm) + inner * m_wm
        brain = csf * (1 - m_cx) + cx * m_cx
        return m_out * brain

    def inside(self, x, dilate=0.0):
        p = np.asarray(x) / (self.axes + dilate)
        return (p * p).sum(-1) <= 1.0


def _slice_frames_sim(stacks, motion):
    """Simulator-side slice frames (its own geometry, written with scipy's
    Rotation): R_i = Rot(r_i) R_stack, centre = Rot(r_i) c0_i + tau_i."""
    Rs, ts = [], []
    i = 0
    for s in stacks:
        n = s["n_slices"]
        for k in range(n):
            c0 = s["origin"] + (k - 0.5 * (n - 1)) * s["thickness"] * s["R"][:, 2]
            Q = Rotation.from_rotvec(motion[i, :3]).as_matrix()
            Rs.append(Q @ s["R"])
            ts.append(Q @ c0 + motion[i, 3:])
            i += 1
    return np.array(Rs), np.array(ts)


def _pixel_grid(s):
    a = (np.arange(s["H"]) - 0.5 * (s["H"] - 1)) * s["dy"]
    b = (np.arange(s["W"]) - 0.5 * (s["W"] - 1)) * s["dx"]
    return a, b


def simulate_phantom_stacks(phantom, stacks, motion, mask_dilate_mm=15.0, noise_frac=0.02, seed=0,
                            nodes=(3, 3, 5)):
    """Observed slices: the phantom integrated over each pixel's PSF (separable
    Gauss-Hermite quadrature along the slice axes) at the moved pixel position,
    then Rician noise sqrt((I + n1)^2 + n2^2), n ~ N(0, (noise_frac * max)^2).
    Only pixels inside the nominal-geometry mask (phantom dilated by
    mask_dilate_mm) are simulated; the others read 0.  Returns (I, mask)."""
    rng = np.random.default_rng(seed + 104729)
    Rm, tm = _slice_frames_sim(stacks, motion)
    Rn, tn = _slice_frames_sim(stacks, np.zeros_like(motion))
    gh = [np.polynomial.hermite_e.hermegauss(n) for n in nodes]
    offs, wts = [], []
    for i0, w0 in zip(*gh[0]):
        for i1, w1 in zip(*gh[1]):
            for i2, w2 in zip(*gh[2]):
                offs.append((i0, i1, i2))
                wts.append(w0 * w1 * w2)
    offs = np.array(offs)
    wts = np.array(wts) / np.sum(wts)
    I_all, mask_all = [], []
    i = 0
    for s in stacks:
        a, b = _pixel_grid(s)
        A, B = np.meshgrid(a, b, indexing="ij")
        u = np.stack([B.reshape(-1), A.reshape(-1), np.zeros(A.size)], axis=1)
        sig = s["fwhm"] * FWHM_TO_SIGMA
        for k in range(s["n_slices"]):
            xn = u @ Rn[i].T + tn[i]
            msk = phantom.inside(xn, mask_dilate_mm)
            img = np.zeros(u.shape[0])
            idx = np.nonzero(msk)[0]
            for c0 in range(0, idx.size, 8192):
                sel = idx[c0:c0 + 8192]
                ul = u[sel][:, None, :] + offs[None, :, :] * sig[None, None, :]
                xw = ul @ Rm[i].T + tm[i]
                img[sel] = (phantom(xw) * wts[None, :]).sum(-1)
            I_all.append(img)
            mask_all.append(msk)
            i += 1
    I = np.concatenate(I_all)
    mask = np.concatenate(mask_all).astype(np.uint8)
    sd = noise_frac * max(1e-6, float(I.max()))
    n1 = rng.normal(0.0, sd, I.shape)
    n2 = rng.normal(0.0, sd, I.shape)
    I = np.sqrt((I + n1) ** 2 + n2 ** 2) * mask
    return I.astype(np.float32), mask


def grid_gaussians(phantom, h=0.8, s=0.8):
    """Gaussians on an h-mm grid inside the phantom's outer ellipsoid, isotropic
    scale s, identity quaternion, amplitude phantom(mu) h^3 / ((2 pi)^(3/2) s^3)
    (so that their sum approximates the phantom)."""
    ext = phantom.axes
    axes = [np.arange(-e + 0.5 * h, e, h) for e in ext]
    X, Y, Z = np.meshgrid(*axes, indexing="ij")
    P = np.stack([X.reshape(-1), Y.reshape(-1), Z.reshape(-1)], 1)
    P = P[phantom.inside(P)]
    N = P.shape[0]
    c = phantom(P) * h ** 3 / ((2 * np.pi) ** 1.5 * s ** 3)
    ls = np.full((3, N), np.log(s))
    q = np.zeros((4, N))
    q[0] = 1.0
    return np.concatenate([P.T, ls, q, c[None, :]], axis=0).reshape(-1), N


def background_gaussians(phantom, h=2.4, margin=15.0):
    """Zero-amplitude isotropic Gaussians (scale h) on an h-mm grid over the
    band within `margin` mm outside the phantom: the background a normalised
    (ratio) model must represent explicitly, since its prediction tends to the
    nearest Gaussians' amplitudes however far they are."""
    ext = np.asarray(phantom.axes) + margin
    axes = [np.arange(-e + 0.5 * h, e, h) for e in ext]
    X, Y, Z = np.meshgrid(*axes, indexing="ij")
    P = np.stack([X.reshape(-1), Y.reshape(-1), Z.reshape(-1)], 1)
    P = P[phantom.inside(P, margin) & ~phantom.inside(P)]
    N = P.shape[0]
    ls = np.full((3, N), np.log(h))
    q = np.zeros((4, N))
    q[0] = 1.0
    return np.concatenate([P.T, ls, q, np.zeros((1, N))], axis=0).reshape(-1), N


def with_gaussians(case, theta_g_extra, n_extra):
    """The case with n_extra more Gaussians appended (component-major layout)."""
    N = case["N"]
    g = case["theta"][:11 * N].reshape(11, N)
    e = np.asarray(theta_g_extra, np.float32).reshape(11, n_extra)
    out = dict(case)
    out["N"] = N + n_extra
    out["theta"] = np.concatenate([np.concatenate([g, e], axis=1).reshape(-1), case["theta"][11 * N:]]).astype(
        np.float32)
    return out


def jitter_gaussians(rng, theta_g, N, amplitude_jitter=0.0, shape_jitter=0.0):
    """A start away from the fit: amplitude_jitter > 0 multiplies the
    amplitudes by U(1 +- jitter); shape_jitter > 0 adds U(+-jitter) to every
    log-scale and turns every Gaussian by a random rotation (anisotropic,
    oriented primitives, so that every gradient group is nonzero)."""
    if not (amplitude_jitter > 0 or shape_jitter > 0):
        return theta_g
    th = theta_g.reshape(11, N).copy()
    if amplitude_jitter > 0:
        th[10] *= rng.uniform(1 - amplitude_jitter, 1 + amplitude_jitter, size=N)
    if shape_jitter > 0:
        th[3:6] += rng.uniform(-shape_jitter, shape_jitter, size=(3, N))
        q = rng.normal(size=(4, N))
        th[6:10] = q / np.linalg.norm(q, axis=0)
    return th.reshape(-1)


def fetal(seed=0, with_truth=False, init="phantom", ref_slice=20, motion_deg=5.0, motion_mm=3.0, jitter=0.0,
          amplitude_jitter=0.0, shape_jitter=0.0):
    """The fetal-scale plain case: ~200k Gaussians on a 0.8 mm grid inside the
    brain phantom; axial / coronal / sagittal stacks of 40 x 192 x 192 px at
    1 x 1 x 3.5 mm centred on the origin; per-slice motion U(+-5 deg) axis
    uniform on the sphere, U(+-3 mm); Rician noise 2 %; pixel mask = brain
    dilated by 15 mm; 2^18 pixels sampled per iteration.  Poses start at 0
    (the unknown motion is what the optimisation recovers).  motion_deg /
    motion_mm widen the motion range; jitter > 0 draws the phantom from the
    canonical-frame family (see BrainPhantom); amplitude_jitter and
    shape_jitter move the start away from the fit (jitter_gaussians)."""
    rng = np.random.default_rng(seed)
    ph = BrainPhantom(seed, jitter=jitter)
    stacks = [stack(40, 192, 192, 1.0, 1.0, 3.5, R) for R in (AXIAL, CORONAL, SAGITTAL)]
    M = n_slices_total(stacks)
    motion = random_motion(rng, M, motion_deg, motion_mm)
    if ref_slice is not None:
        motion[ref_slice] = 0.0  # the reference slice fixes the frame (its pose is frozen)
    I, mask = simulate_phantom_stacks(ph, stacks, motion, seed=seed)
    theta_g, N = grid_gaussians(ph)
    if init == "flat":
        # cold start: every amplitude from the mean observed intensity inside the brain
        h, s = 0.8, 0.8
        level = float(np.mean(I[mask > 0][I[mask > 0] > 0.2])) if np.any(I[mask > 0] > 0.2) else 0.5
        theta_g = theta_g.reshape(11, N)
        theta_g[10] = level * h ** 3 / ((2 * np.pi) ** 1.5 * s ** 3)
        theta_g = theta_g.reshape(-1)
    theta_g = jitter_gaussians(rng, theta_g, N, amplitude_jitter, shape_jitter)
    theta = np.concatenate([theta_g, np.zeros(6 * M)]).astype(np.float32)
    out = {"name": "fetal", "N": N, "stacks": stacks, "theta": theta, "I": I, "mask": mask,
           "n_sample": 1 << 18, "ref_slice": ref_slice, "phantom": ph}
    if with_truth:
        out["motion"] = motion
    return out


def first_stacks(case, n):
    """The same case restricted to its first n stacks (observations, mask, poses
    cut accordingly); the pixel sample shrinks with the pixel count."""
    stacks = case["stacks"][:n]
    P = n_pixels_total(stacks)
    M = n_slices_total(stacks)
    N = case["N"]
    out = dict(case)
    out["stacks"] = stacks
    out["I"] = case["I"][:P]
    out["mask"] = case["mask"][:P]
    out["theta"] = np.concatenate([case["theta"][:11 * N], case["theta"][11 * N:11 * N + 6 * M]])
    frac = P / n_pixels_total(case["stacks"])
    out["n_sample"] = min(int(out["mask"].sum()), int(case["n_sample"] * frac))
    return out


def grid_probe(phantom, h=0.8, margin=2.0):
    """An isotropic h-mm grid over the phantom's bounding box as one axial stack
    with a zero-width PSF (each pixel then reads the volume itself), the phantom
    value at every grid point, and the mask of points inside the phantom."""
    ext = phantom.axes + margin
    n = [int(np.ceil(2 * e / h)) for e in ext]
    st = stack(n[2], n[1], n[0], h, h, h)
    st["fwhm"] = np.zeros(3)
    xs = (np.arange(n[0]) - 0.5 * (n[0] - 1)) * h
    ys = (np.arange(n[1]) - 0.5 * (n[1] - 1)) * h
    zs = (np.arange(n[2]) - 0.5 * (n[2] - 1)) * h
    Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
    P = np.stack([X.reshape(-1), Y.reshape(-1), Z.reshape(-1)], 1)
    ref = phantom(P).astype(np.float32)
    inside = phantom.inside(P).astype(np.uint8)
    return st, ref, inside


def concat_cases(cases):
    """Several cases as one batched case: stacks, observations, masks and poses
    concatenated in subject order, Gaussian parameters concatenated per
    component (the parameter vector stays component-major over all Gaussians).
    Adds "stack_subject" (per stack) and "gauss_count" (per subject)."""
    Ns = [int(c["N"]) for c in cases]
    N = sum(Ns)
    comps = []
    for k in range(11):
        comps.append(np.concatenate([c["theta"][k * n:(k + 1) * n] for c, n in zip(cases, Ns)]))
    poses = np.concatenate([c["theta"][11 * n:] for c, n in zip(cases, Ns)])
    out = {"name": "batched", "N": N, "stacks": [s for c in cases for s in c["stacks"]],
           "theta": np.concatenate(comps + [poses]).astype(np.float32),
           "I": np.concatenate([c["I"] for c in cases]).astype(np.float32),
           "mask": np.concatenate([c["mask"] for c in cases]).astype(np.uint8),
           "stack_subject": np.array([k for k, c in enumerate(cases) for _ in c["stacks"]], np.int32),
           "gauss_count": np.array(Ns, np.int64), "n_sample": max(int(c.get("n_sample", 0)) for c in cases)}
    return out


def subject_theta(theta, gauss_count, k):
    """The 11 N_k Gaussian entries of subject k from a batched parameter vector."""
    g = np.concatenate([[0], np.cumsum(gauss_count)]).astype(np.int64)
    N = int(g[-1])
    return np.concatenate([theta[c * N + g[k]:c * N + g[k + 1]] for c in range(11)])


def batched(seed=1000, n_subjects=16, nodes=(1, 1, 3)):
    """The batched multi-subject workload: subjects of uneven size.  Subject k
    (seed + k): Gaussians N_k log-uniform in [50k, 500k] (brain phantom scaled so
    its 0.8 mm grid holds N_k), 3-9 stacks (three orthogonal first, then random
    oblique orientations), 24-60 slices of W x W px with W in {128, 160, 192,
    224, 256} at 160 mm / W in-plane, thickness U(2.5, 4.5) mm, per-slice motion
    U(+-15 deg) / U(+-8 mm) (the reference slice 0 of stack 0 unmoved), Rician
    noise 2 %, mask = phantom dilated by 15 mm x scale; flat-amplitude start."""
    cases = []
    for k in range(n_subjects):
        rng = np.random.default_rng(seed + k)
        Nk = float(np.exp(rng.uniform(np.log(5e4), np.log(5e5))))
        scale = (Nk / 200480.0) ** (1.0 / 3.0)
        ph = BrainPhantom(seed + k, scale=scale)
        n_st = int(rng.integers(3, 10))
        W = int(rng.choice([128, 160, 192, 224, 256]))
        dx = 160.0 / W
        thick = float(rng.uniform(2.5, 4.5))
        n_sl = int(rng.integers(24, 61))
        Rs = [AXIAL, CORONAL, SAGITTAL] + [Rotation.random(random_state=int(rng.integers(1 << 31))).as_matrix()
                                           for _ in range(n_st - 3)]
        stacks = [stack(n_sl, W, W, dx, dx, thick, R) for R in Rs]
        M = n_slices_total(stacks)
        motion = random_motion(rng, M, 15.0, 8.0)
        motion[n_sl // 2] = 0.0
        I, mask = simulate_phantom_stacks(ph, stacks, motion, mask_dilate_mm=15.0 * scale, seed=seed + k,
                                          nodes=nodes)
        theta_g, N = grid_gaussians(ph)
        level = float(np.mean(I[mask > 0][I[mask > 0] > 0.2])) if np.any(I[mask > 0] > 0.2) else 0.5
        th = theta_g.reshape(11, N)
        th[10] = level * 0.8 ** 3 / ((2 * np.pi) ** 1.5 * 0.8 ** 3)
        cases.append({"name": "subject%d" % k, "N": N, "stacks": stacks,
                      "theta": np.concatenate([th.reshape(-1), np.zeros(6 * M)]).astype(np.float32), "I": I,
                      "mask": mask, "n_sample": 1 << 18, "ref_slice": n_sl // 2, "phantom": ph})
    return cases


def large(seed=0, nodes=(1, 1, 3), amplitude_jitter=0.0, shape_jitter=0.0):
    """The large single-subject workload: the brain phantom scaled by 2.307
    (semi-axes 80.8 / 64.6 / 57.7 mm) so that its 1.08 mm grid holds ~1M
    Gaussians (s = 1.08 mm); six stacks of 48 x 256 x 256 px at
    0.8 x 0.8 x 3.0 mm (axial, coronal, sagittal, and the axial stack turned
    45 degrees about x, y and z); per-slice motion U(+-10 deg) / U(+-5 mm)
    (slice 24 of stack 0 unmoved); Rician noise 2 %; mask = phantom dilated by
    15 mm; every masked pixel each iteration.  amplitude_jitter > 0 multiplies
    the amplitudes by U(1 +- jitter) (a start away from the fit);
    shape_jitter > 0 adds U(+-jitter) to every log-scale and turns every
    Gaussian by a random rotation (anisotropic, oriented primitives)."""
    rng = np.random.default_rng(seed)
    ph = BrainPhantom(seed, scale=2.307)
    turned = [Rotation.from_euler(ax, 45.0, degrees=True).as_matrix() @ AXIAL for ax in ("x", "y", "z")]
    stacks = [stack(48, 256, 256, 0.8, 0.8, 3.0, R) for R in [AXIAL, CORONAL, SAGITTAL] + turned]
    M = n_slices_total(stacks)
    motion = random_motion(rng, M, 10.0, 5.0)
    motion[24] = 0.0
    I, mask = simulate_phantom_stacks(ph, stacks, motion, mask_dilate_mm=15.0, seed=seed, nodes=nodes)
    theta_g, N = grid_gaussians(ph, h=1.08, s=1.08)
    theta_g = jitter_gaussians(rng, theta_g, N, amplitude_jitter, shape_jitter)
    theta = np.concatenate([theta_g, np.zeros(6 * M)]).astype(np.float32)
    return {"name": "large", "N": N, "stacks": stacks, "theta": theta, "I": I, "mask": mask,
            "n_sample": int(mask.sum()), "ref_slice": 24, "phantom": ph, "motion": motion}


def metric_volumes(seed, shape, noise=0.05, blur=1.0):
    """A reference volume Y (smooth random field in [0, 1], with a sharp-edged
    ellipsoid for structure) and a degraded copy X (blurred by `blur` voxels,
    Gaussian noise of standard deviation `noise`, 3 % gain and 0.02 offset)
    on a grid of `shape` (D, H, W), float32, with the mask of the ellipsoid
    dilated by 2 voxels: the inputs of the image-quality metrics."""
    from scipy import ndimage
    rng = np.random.default_rng(seed)
    D, H, W = shape
    f = ndimage.gaussian_filter(rng.uniform(0, 1, shape), 2.0)
    f = (f - f.min()) / max(f.max() - f.min(), 1e-12)
    z, y, x = np.meshgrid(*[(np.arange(n) - 0.5 * (n - 1)) / max(0.5 * n, 1.0) for n in shape], indexing="ij")
    r = (x / 0.7) ** 2 + (y / 0.6) ** 2 + (z / 0.8) ** 2
    Y = np.clip(0.35 * f + 0.6 * (r < 1.0), 0.0, 1.0)
    X = 1.03 * ndimage.gaussian_filter(Y, blur) + 0.02 + noise * rng.normal(0, 1, shape)
    mask = ndimage.binary_dilation(r < 1.0, iterations=2)
    return X.astype(np.float32), Y.astype(np.float32), mask.astype(np.uint8)


def densify_stats(seed, N, count=4, scale=1.0):
    """Densification statistics of N Gaussians after `count` passes: summed
    gradient norms (log-normal, heavy-tailed like real mean-gradient norms,
    median `scale` per pass) and summed gradient vectors whose norm does not
    exceed that sum; float32 (N, 4)."""
    rng = np.random.default_rng(seed)
    n = scale * count * rng.lognormal(0.0, 1.0, N)
    d = rng.normal(0, 1, (N, 3))
    d /= np.maximum(np.linalg.norm(d, axis=1, keepdims=True), 1e-12)
    frac = rng.uniform(0.2, 1.0, (N, 1))
    acc = np.concatenate([n[:, None], d * frac * n[:, None]], axis=1)
    return acc.astype(np.float32), int(count)
