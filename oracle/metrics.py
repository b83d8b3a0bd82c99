"""Oracle of the image-quality metrics that score a reconstructed volume
against its ground truth (Sec. 3, Table 1: PSNR, SSIM, NCC).

TEST INFRASTRUCTURE ONLY (same rules as oracle.py): plain float64 numpy, the
definitions written out, no blocking or separable filtering.

The paper names the three metrics but not their parameters; the readings:

- the reconstruction X and the ground truth Y are sampled on the same D x H x W
  grid, and every metric is taken over the voxels of a mask (the brain);
- PSNR = 10 log10(L^2 / MSE), L the data range passed in;
- NCC = the Pearson correlation of X and Y over the masked voxels;
- SSIM (Wang, Bovik, Sheikh, Simoncelli 2004) with its usual constants
  K1 = 0.01, K2 = 0.03 (C1 = (K1 L)^2, C2 = (K2 L)^2) and its 11-tap Gaussian
  window of standard deviation 1.5 voxels, in 3D the product window
  11 x 11 x 11.  Near the grid border the window keeps the offsets that stay
  on the grid and is renormalised over them.  Local statistics are weighted
  population moments over every grid voxel of the window (masked or not):
      mu_X = sum_o w_o X(v + o),   s_X^2 = sum_o w_o X(v + o)^2 - mu_X^2,
      s_XY = sum_o w_o X(v + o) Y(v + o) - mu_X mu_Y,
  and the SSIM map
      ((2 mu_X mu_Y + C1)(2 s_XY + C2)) / ((mu_X^2 + mu_Y^2 + C1)(s_X^2 + s_Y^2 + C2))
  is averaged over the masked voxels.
"""
import numpy as np

K1 = 0.01
K2 = 0.03
SIGMA = 1.5
RADIUS = 5


def window_1d():
    """Unnormalised taps exp(-o^2 / (2 sigma^2)), o = -RADIUS .. RADIUS."""
    o = np.arange(-RADIUS, RADIUS + 1, dtype=np.float64)
    return np.exp(-0.5 * (o / SIGMA) ** 2)


def _window_3d():
    g = window_1d()
    return g[:, None, None] * g[None, :, None] * g[None, None, :]


def local_stats(X, Y, voxels=None):
    """(mu_X, mu_Y, s_X^2, s_Y^2, s_XY) at every voxel of the (D, H, W) grid, or
    at the flat voxel indices `voxels`, from the renormalised 3D window.  Every
    voxel by its own window sum: the whole grid only for small volumes."""
    X = np.asarray(X, np.float64)
    Y = np.asarray(Y, np.float64)
    D, H, W = X.shape
    w3 = _window_3d()
    if voxels is None:
        out = [np.zeros((D, H, W)) for _ in range(5)]
        norm = np.zeros((D, H, W))
        for dz in range(-RADIUS, RADIUS + 1):
            for dy in range(-RADIUS, RADIUS + 1):
                for dx in range(-RADIUS, RADIUS + 1):
                    if abs(dz) >= D or abs(dy) >= H or abs(dx) >= W:
                        continue  # the offset leaves the grid from every voxel
                    w = w3[dz + RADIUS, dy + RADIUS, dx + RADIUS]
                    # output voxels v whose neighbour v + o is on the grid
                    oz = slice(max(0, -dz), min(D, D - dz))
                    oy = slice(max(0, -dy), min(H, H - dy))
                    ox = slice(max(0, -dx), min(W, W - dx))
                    iz = slice(max(0, dz), min(D, D + dz))
                    iy = slice(max(0, dy), min(H, H + dy))
                    ix = slice(max(0, dx), min(W, W + dx))
                    x = X[iz, iy, ix]
                    y = Y[iz, iy, ix]
                    norm[oz, oy, ox] += w
                    out[0][oz, oy, ox] += w * x
                    out[1][oz, oy, ox] += w * y
                    out[2][oz, oy, ox] += w * x * x
                    out[3][oz, oy, ox] += w * y * y
                    out[4][oz, oy, ox] += w * x * y
        mx, my = out[0] / norm, out[1] / norm
        return (mx, my, out[2] / norm - mx * mx, out[3] / norm - my * my, out[4] / norm - mx * my)
    res = np.zeros((5, len(voxels)))
    for n, v in enumerate(np.asarray(voxels, np.int64)):
        z, r = divmod(int(v), H * W)
        y0, x0 = divmod(r, W)
        z0, z1 = max(0, z - RADIUS), min(D, z + RADIUS + 1)
        a0, a1 = max(0, y0 - RADIUS), min(H, y0 + RADIUS + 1)
        b0, b1 = max(0, x0 - RADIUS), min(W, x0 + RADIUS + 1)
        w = w3[z0 - z + RADIUS:z1 - z + RADIUS, a0 - y0 + RADIUS:a1 - y0 + RADIUS, b0 - x0 + RADIUS:b1 - x0 + RADIUS]
        w = w / w.sum()
        x = X[z0:z1, a0:a1, b0:b1]
        y = Y[z0:z1, a0:a1, b0:b1]
        mx, my = (w * x).sum(), (w * y).sum()
        res[:, n] = (mx, my, (w * x * x).sum() - mx * mx, (w * y * y).sum() - my * my, (w * x * y).sum() - mx * my)
    return tuple(res)


def ssim_from_stats(stats, L):
    mx, my, vx, vy, cxy = stats
    C1 = (K1 * L) ** 2
    C2 = (K2 * L) ** 2
    return ((2 * mx * my + C1) * (2 * cxy + C2)) / ((mx * mx + my * my + C1) * (vx + vy + C2))


def ssim_map(X, Y, L, voxels=None):
    """The SSIM map on the whole grid (small volumes), or at flat voxel
    indices `voxels`."""
    return ssim_from_stats(local_stats(X, Y, voxels), float(L))


def psnr(X, Y, mask, L):
    m = np.asarray(mask).reshape(-1) != 0
    d = np.asarray(X, np.float64).reshape(-1)[m] - np.asarray(Y, np.float64).reshape(-1)[m]
    return 10.0 * np.log10(float(L) ** 2 / np.mean(d * d))


def ncc(X, Y, mask):
    m = np.asarray(mask).reshape(-1) != 0
    x = np.asarray(X, np.float64).reshape(-1)[m]
    y = np.asarray(Y, np.float64).reshape(-1)[m]
    x = x - x.mean()
    y = y - y.mean()
    return float((x * y).sum() / np.sqrt((x * x).sum() * (y * y).sum()))


def ssim(X, Y, mask, L):
    """Mean SSIM over the masked voxels (whole-grid map: small volumes)."""
    S = ssim_map(X, Y, L)
    return float(S.reshape(-1)[np.asarray(mask).reshape(-1) != 0].mean())


def metrics(X, Y, mask, L):
    """(PSNR, SSIM, NCC) of the volumes X, Y (D, H, W) over `mask`."""
    return psnr(X, Y, mask, L), ssim(X, Y, mask, L), ncc(X, Y, mask)
