"""Oracle of coarse-to-fine densification: split, clone and prune of the
Gaussians (the progressive densification the paper names as future work,
"Limitations and Future Work", after Kerbl et al. 2023, 3D Gaussian
Splatting, adaptive density control).

TEST INFRASTRUCTURE ONLY (same rules as oracle.py).

The paper gives no rule; the one built here, in the notation of Sec. 2.2
(mean mu_j, log-scales ls_j, quaternion q_j = (w, x, y, z), amplitude c_j):

- statistic: per Gaussian the running sums of ||dL/dmu_j|| and of dL/dmu_j
  over the backward passes since the last densification, and the count of
  those passes; the mean norm is sum / count (0 when count = 0);
- decision (float32, so that both implementations take it identically):
  prune when |c_j| < prune_amplitude; otherwise, when the mean norm exceeds
  grad_threshold, split if the largest log-scale exceeds log_scale_threshold,
  else clone; otherwise keep;
- split: the two children sit at mu_j +- d a, a the principal axis (the
  rotation's column of the largest log-scale, first index on ties) and
  d = s sqrt(1 - 1/phi^2), s that scale; their principal scale is s / phi,
  the other scales and q unchanged.  The pair then has the parent's mean and
  covariance (s^2/phi^2 + d^2 = s^2 along a).  Amplitudes c phi / 2 keep the
  summed mass c (2 pi)^(3/2) s_0 s_1 s_2 (mass_preserving, the plain sum);
  the normalised ratio model keeps c;
- clone: the two copies sit at mu_j +- delta u, u the direction of the summed
  mean gradient (the principal axis if it is zero), delta = clone_offset times
  the smallest scale; scales and q unchanged; amplitudes c / 2 (mass
  preserving) or c;
- output order: the Gaussians in index order, a kept one once, a split or
  cloned one as its two children (+ first), a pruned one not at all; Adam
  moments are copied for kept Gaussians and zero for children; the slice
  poses (and their moments) follow unchanged; the statistics restart at 0.
"""
import numpy as np

KEEP, PRUNE, SPLIT, CLONE = 1, 0, 2, 3


def _f32(x):
    return np.float32(x)


def accumulate(acc, count, grad, N):
    """One accumulation step in float32: acc (N, 4) += (||g||, g), count + 1,
    g = (dL/dmu_x, dL/dmu_y, dL/dmu_z) from the component-major gradient; the
    norm as sqrt((gx gx + gy gy) + gz gz), every operation rounded to float32."""
    acc = np.asarray(acc, np.float32).copy()
    g = np.asarray(grad, np.float32)
    gx, gy, gz = g[0:N], g[N:2 * N], g[2 * N:3 * N]
    n = np.sqrt((gx * gx + gy * gy) + gz * gz)
    acc[:, 0] += n
    acc[:, 1] += gx
    acc[:, 2] += gy
    acc[:, 3] += gz
    return acc, int(count) + 1


def decide(theta, N, acc, count, grad_threshold, log_scale_threshold, prune_amplitude):
    """Per-Gaussian decision (KEEP, PRUNE, SPLIT, CLONE) in float32."""
    th = np.asarray(theta, np.float32)
    acc = np.asarray(acc, np.float32)
    c = th[10 * N:11 * N]
    ls = th[3 * N:6 * N].reshape(3, N)
    if count > 0:
        avg = acc[:, 0] / np.float32(count)
    else:
        avg = np.zeros(N, np.float32)
    kind = np.full(N, KEEP, np.int64)
    big = ls.max(axis=0) > _f32(log_scale_threshold)
    hot = avg > _f32(grad_threshold)
    kind[hot & big] = SPLIT
    kind[hot & ~big] = CLONE
    kind[np.abs(c) < _f32(prune_amplitude)] = PRUNE
    return kind


def _rotation(q):
    w, x, y, z = q / np.linalg.norm(q)
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def densify(theta, m, v, N, M, acc, count, grad_threshold, log_scale_threshold, prune_amplitude=0.0,
            split_factor=1.6, clone_offset=0.5, mass_preserving=True):
    """(theta', m', v', N', kind, parent) after one densification: float64
    parameter vectors of 11 N' + 6 M entries, the per-Gaussian decisions and,
    per output Gaussian, the index of its parent."""
    th = np.asarray(theta, np.float64)
    m = np.asarray(m, np.float64)
    v = np.asarray(v, np.float64)
    acc = np.asarray(acc, np.float32)
    kind = decide(theta, N, acc, count, grad_threshold, log_scale_threshold, prune_amplitude)
    nout = np.where(kind == PRUNE, 0, np.where(kind == KEEP, 1, 2))
    N2 = int(nout.sum())
    g = th[:11 * N].reshape(11, N)
    gm = m[:11 * N].reshape(11, N)
    gv = v[:11 * N].reshape(11, N)
    out = np.zeros((11, N2))
    om = np.zeros((11, N2))
    ov = np.zeros((11, N2))
    parent = np.zeros(N2, np.int64)
    phi = float(split_factor)
    o = 0
    for j in range(N):
        if kind[j] == PRUNE:
            continue
        if kind[j] == KEEP:
            out[:, o], om[:, o], ov[:, o] = g[:, j], gm[:, j], gv[:, j]
            parent[o] = j
            o += 1
            continue
        mu, ls, q, c = g[0:3, j], g[3:6, j].copy(), g[6:10, j], g[10, j]
        k = int(np.argmax(ls))
        a = _rotation(q)[:, k]
        if kind[j] == SPLIT:
            step = np.exp(ls[k]) * np.sqrt(1.0 - 1.0 / phi ** 2) * a
            ls[k] -= np.log(phi)
            c2 = c * phi / 2.0 if mass_preserving else c
        else:
            s = acc[j, 1:4].astype(np.float64)
            n = np.linalg.norm(s)
            u = s / n if n > 0 else a
            step = float(clone_offset) * np.exp(ls.min()) * u
            c2 = c / 2.0 if mass_preserving else c
        for sign in (1.0, -1.0):
            out[0:3, o] = mu + sign * step
            out[3:6, o] = ls
            out[6:10, o] = q
            out[10, o] = c2
            parent[o] = j
            o += 1
    poses = th[11 * N:11 * N + 6 * M]
    theta2 = np.concatenate([out.reshape(-1), poses])
    m2 = np.concatenate([om.reshape(-1), m[11 * N:11 * N + 6 * M]])
    v2 = np.concatenate([ov.reshape(-1), v[11 * N:11 * N + 6 * M]])
    return theta2, m2, v2, N2, kind, parent
