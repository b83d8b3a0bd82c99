"""Oracle of the content-adaptive initialisation of the Gaussian means
(Sec. 2.5, "Content-Adaptive Initialization"):

    P_init(T_i(u)) proportional to (1 - lambda_init) |grad I_i(u)| + lambda_init

over the masked slice pixels; every mean is drawn from P_init and placed at the
drawn pixel's world position T_i(u), jittered uniformly within the pixel's
voxel footprint (dx x dy x slice thickness) so that repeated draws of a pixel
give distinct means.

TEST INFRASTRUCTURE ONLY (same rules as oracle.py).

The draw turns floating point into an integer (which pixel), so both sides take
that decision in the same arithmetic, the kernel's: the gradient magnitude in
float32 with every operation rounded separately (no fused multiply-add), the
weight quantised to the integer floor(1024 w), an integer cumulative sum, and
for draw k the integer t = floor(x_k T / 2^64) (x_k the 64-bit SplitMix64
output for counter k, T the total weight) mapped to the first pixel whose
cumulative weight exceeds t.  Jitter uniforms are 24-bit fractions of further
SplitMix64 outputs.  Positions are then computed in float64.
"""
import numpy as np

from . import oracle as _o

QUANT = 1024.0
JITTER_CTR = 1 << 40


def _slices(stacks):
    out, base = [], 0
    for s in stacks:
        for k in range(int(s["n_slices"])):
            out.append((s, k, base))
            base += int(s["H"]) * int(s["W"])
    return out


def grad_magnitude(stacks, I):
    """|grad I| per pixel (float32, global pixel order): central differences
    over the neighbouring pixels (one-sided at the image border), divided by
    the pixel spacing times the span."""
    I = np.asarray(I, np.float32)
    out = np.zeros(I.shape, np.float32)
    for (s, _, b) in _slices(stacks):
        H, W = int(s["H"]), int(s["W"])
        img = I[b:b + H * W].reshape(H, W)
        cm = np.clip(np.arange(W) - 1, 0, W - 1)
        cp = np.clip(np.arange(W) + 1, 0, W - 1)
        rm = np.clip(np.arange(H) - 1, 0, H - 1)
        rp = np.clip(np.arange(H) + 1, 0, H - 1)
        dxs = np.float32(s["dx"]) * (cp - cm).astype(np.float32)
        dys = np.float32(s["dy"]) * (rp - rm).astype(np.float32)
        with np.errstate(divide="ignore", invalid="ignore"):
            gx = (img[:, cp] - img[:, cm]) / dxs[None, :]
            gy = (img[rp, :] - img[rm, :]) / dys[:, None]
        gx = np.where(np.isfinite(gx), gx, np.float32(0)).astype(np.float32)
        gy = np.where(np.isfinite(gy), gy, np.float32(0)).astype(np.float32)
        out[b:b + H * W] = np.sqrt(gx * gx + gy * gy).reshape(-1)
    return out


def weights(stacks, I, mask, lambda_init):
    """Integer draw weights floor(1024 ((1 - lambda) |grad I| + lambda)) of the
    masked pixels (0 elsewhere)."""
    g = grad_magnitude(stacks, I)
    lam = np.float32(lambda_init)
    w = (np.float32(1.0) - lam) * g + lam
    q = np.floor(w * np.float32(QUANT)).astype(np.int64)
    return np.where(np.asarray(mask) != 0, q, 0)


def draw_pixels(W, ks, seed):
    """Pixel of draws ks: the first index whose cumulative weight exceeds
    floor(x_k T / 2^64)."""
    C = np.cumsum(np.asarray(W, np.int64))
    T = int(C[-1])
    if T <= 0:
        raise ValueError("no weight to draw from")
    t = np.array([(_o.splitmix64(seed, int(k)) * T) >> 64 for k in ks], dtype=object)
    return np.searchsorted(C, t.astype(np.int64), side="right")


def jitter(ks, seed):
    """(len(ks), 3) uniforms in [-1/2, 1/2): 24-bit fractions of SplitMix64
    outputs at counters 2^40 + 3 k + a."""
    out = np.zeros((len(ks), 3))
    for n, k in enumerate(ks):
        for a in range(3):
            x = _o.splitmix64(seed, JITTER_CTR + 3 * int(k) + a)
            out[n, a] = (x >> 40) * 2.0 ** -24 - 0.5
    return out


def init_means(stacks, I, mask, theta_pose, n, lambda_init, seed, ks=None):
    """(mu (len, 3) float64, pixel index (len)) of draws ks (default 0 .. n-1)
    of the content-adaptive initialisation, with the slice frames of the given
    poses (M x 6)."""
    ks = np.arange(int(n)) if ks is None else np.asarray(ks)
    W = weights(stacks, I, mask, lambda_init)
    pix = draw_pixels(W, ks, seed)
    R, t = _o.slice_frames(stacks, np.asarray(theta_pose, np.float64))
    sl = _slices(stacks)
    firsts = np.array([b for (_, _, b) in sl], np.int64)
    j = jitter(ks, seed)
    mu = np.zeros((len(ks), 3))
    for k, p in enumerate(pix):
        i = int(np.searchsorted(firsts, p, side="right") - 1)
        s, _, b = sl[i]
        a, c = divmod(int(p - b), int(s["W"]))
        u = np.array([(c + j[k, 0] - 0.5 * (int(s["W"]) - 1)) * float(s["dx"]),
                      (a + j[k, 1] - 0.5 * (int(s["H"]) - 1)) * float(s["dy"]),
                      j[k, 2] * float(s["thickness"])])
        mu[k] = R[i] @ u + t[i]
    return mu, pix
