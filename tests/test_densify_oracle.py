"""Pins for the oracle of densification (split, clone, prune; the paper's
coarse-to-fine future work after 3D Gaussian Splatting's adaptive density
control), against facts fixed by the mathematics:

- a split pair has the parent's mass, mean and covariance (mixture moments
  from covariances built with scipy's rotation, not the oracle's);
- a clone pair has the parent's mass and mean, and covariance
  Sigma + delta^2 u u^T;
- with mass preservation the plain sum's integral over space (the summed
  masses, by a 3D grid quadrature) is unchanged;
- the decision table on crafted cases: strict thresholds, prune before the
  rest, first index on tied largest scales, count 0 meaning no split or clone;
- the output layout: N' = N - pruned + split + cloned, kept Gaussians and
  their Adam moments copied exactly, children with zero moments, poses and
  their moments unchanged, children of one parent adjacent and parents in
  index order;
- the float32 accumulation step against numpy's norm.
"""
import numpy as np
import pytest
from scipy.spatial.transform import Rotation


@pytest.fixture(scope="module")
def dens():
    from oracle import densify
    return densify


def _gauss(seed, N, M=2):
    rng = np.random.default_rng(seed)
    mu = rng.uniform(-5, 5, (3, N))
    ls = rng.normal(0.0, 0.4, (3, N))
    q = rng.normal(0, 1, (4, N))
    c = rng.uniform(0.2, 1.0, N)
    th = np.concatenate([mu.reshape(-1), ls.reshape(-1), q.reshape(-1), c, rng.normal(0, 0.05, 6 * M)])
    return th.astype(np.float32)


def _sigma(q, ls):
    R = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
    return R @ np.diag(np.exp(2 * ls)) @ R.T


def _mass(c, ls):
    return c * (2 * np.pi) ** 1.5 * np.exp(ls.sum())


def _children(dens, kind_want, mass=True):
    N = 1
    th = _gauss(3, N)
    th[3:6] = [0.9, 0.2, -0.3]  # principal axis 0
    acc = np.array([[5.0, 1.0, -2.0, 0.5]], np.float32)
    lst = 0.5 if kind_want == dens.SPLIT else 2.0
    out = dens.densify(th, np.zeros_like(th), np.zeros_like(th), N, 2, acc, 2, 1.0, lst, 0.0, 1.6, 0.5, mass)
    th2, _, _, N2, kind, _ = out
    assert kind[0] == kind_want and N2 == 2
    g = th.astype(np.float64)[:11].reshape(11, 1)[:, 0]
    ch = th2[:22].reshape(11, 2)
    return g, ch


def test_split_keeps_mass_mean_covariance(dens):
    g, ch = _children(dens, dens.SPLIT)
    S = _sigma(g[6:10], g[3:6])
    mean = ch[0:3].mean(axis=1)
    assert np.allclose(mean, g[0:3], atol=1e-12)
    cov = np.zeros((3, 3))
    for k in range(2):
        d = ch[0:3, k] - mean
        cov += 0.5 * (_sigma(ch[6:10, k], ch[3:6, k]) + np.outer(d, d))
    assert np.allclose(cov, S, rtol=1e-10, atol=1e-12)
    assert _mass(ch[10, 0], ch[3:6, 0]) + _mass(ch[10, 1], ch[3:6, 1]) == pytest.approx(_mass(g[10], g[3:6]), rel=1e-12)
    assert ch[3, 0] == pytest.approx(g[3] - np.log(1.6), abs=1e-12)


def test_clone_keeps_mass_mean(dens):
    g, ch = _children(dens, dens.CLONE)
    S = _sigma(g[6:10], g[3:6])
    mean = ch[0:3].mean(axis=1)
    assert np.allclose(mean, g[0:3], atol=1e-12)
    u = np.array([1.0, -2.0, 0.5]) / np.linalg.norm([1.0, -2.0, 0.5])
    delta = 0.5 * np.exp(g[3:6].min())
    cov = np.zeros((3, 3))
    for k in range(2):
        d = ch[0:3, k] - mean
        cov += 0.5 * (_sigma(ch[6:10, k], ch[3:6, k]) + np.outer(d, d))
    assert np.allclose(cov, S + delta ** 2 * np.outer(u, u), rtol=1e-10, atol=1e-12)
    assert ch[10].sum() == pytest.approx(g[10], rel=1e-12)


def test_ratio_model_keeps_colours(dens):
    g, ch = _children(dens, dens.SPLIT, mass=False)
    assert np.all(ch[10] == g[10])


def test_plain_sum_integral_unchanged(dens):
    """Quadrature of the plain sum over a box holding every Gaussian."""
    N, M = 12, 1
    th = _gauss(4, N, M)
    th[3 * N:6 * N] = np.random.default_rng(5).uniform(-0.6, 0.1, 3 * N)
    acc = np.zeros((N, 4), np.float32)
    acc[:, 0] = np.linspace(0.0, 3.0, N)
    acc[:, 1:] = 1.0
    th2, _, _, N2, kind, _ = dens.densify(th, np.zeros_like(th), np.zeros_like(th), N, M, acc, 1, 1.0, -0.2)
    assert set(kind) >= {dens.SPLIT, dens.CLONE, dens.KEEP}

    def integral(theta, n):
        g = np.asarray(theta, np.float64)[:11 * n].reshape(11, n)
        h = 0.25
        ax = np.arange(-12, 12, h) + 0.5 * h
        X, Y, Z = np.meshgrid(ax, ax, ax, indexing="ij")
        P = np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1)
        tot = 0.0
        for j in range(n):
            Sinv = np.linalg.inv(_sigma(g[6:10, j], g[3:6, j]))
            d = P - g[0:3, j]
            tot += g[10, j] * np.exp(-0.5 * np.einsum("pi,ij,pj->p", d, Sinv, d)).sum() * h ** 3
        return tot
    assert integral(th2, N2) == pytest.approx(integral(th, N), rel=1e-9)


def test_decision_table(dens):
    N = 6
    th = _gauss(6, N)
    ls = th[3 * N:6 * N].reshape(3, N)
    ls[:] = -1.0
    ls[1, 1] = 0.5          # large: split
    ls[0, 2] = ls[2, 2] = 0.5  # tie of the largest scale: axis 0
    th[10 * N + 3] = 1e-4   # pruned whatever its gradient
    th[3 * N:6 * N] = ls.reshape(-1)
    acc = np.zeros((N, 4), np.float32)
    acc[:, 0] = [4.0, 4.0, 4.0, 4.0, 2.0, 4.0]  # mean 2 (count 2) except index 4: mean 1 = threshold
    acc[:, 1] = 1.0
    kind = dens.decide(th, N, acc, 2, 1.0, 0.0, 1e-3)
    assert list(kind) == [dens.CLONE, dens.SPLIT, dens.SPLIT, dens.PRUNE, dens.KEEP, dens.CLONE]
    assert list(dens.decide(th, N, acc, 0, 1.0, 0.0, 1e-3)) == [1, 1, 1, 0, 1, 1]
    th2, _, _, _, _, parent = dens.densify(th, np.zeros_like(th), np.zeros_like(th), N, 2, acc, 2, 1.0, 0.0, 1e-3)
    g2 = th2[:11 * len(parent)].reshape(11, -1)
    # the tied Gaussian splits along axis 0 (its first largest log-scale)
    k = np.flatnonzero(parent == 2)
    assert np.allclose(g2[3, k], 0.5 - np.log(1.6)) and np.allclose(g2[5, k], 0.5)


def test_layout(dens):
    N, M = 40, 3
    th = _gauss(7, N, M)
    rng = np.random.default_rng(8)
    m = rng.normal(0, 1, th.size).astype(np.float32)
    v = rng.uniform(0, 1, th.size).astype(np.float32)
    acc = np.zeros((N, 4), np.float32)
    acc[:, 0] = rng.uniform(0, 3, N)
    acc[:, 1:] = rng.normal(0, 1, (N, 3))
    th[10 * N:10 * N + 5] = 0.0
    th2, m2, v2, N2, kind, parent = dens.densify(th, m, v, N, M, acc, 1, 1.5, 0.2, 0.05)
    ns, nc, npr = (kind == dens.SPLIT).sum(), (kind == dens.CLONE).sum(), (kind == dens.PRUNE).sum()
    assert ns > 0 and nc > 0 and npr == 5
    assert N2 == N - npr + ns + nc and len(th2) == 11 * N2 + 6 * M
    assert np.all(np.diff(parent) >= 0)
    g, g2 = th.reshape(-1)[:11 * N].reshape(11, N), th2[:11 * N2].reshape(11, N2)
    gm, gm2 = m[:11 * N].reshape(11, N), m2[:11 * N2].reshape(11, N2)
    for o, j in enumerate(parent):
        if kind[j] == dens.KEEP:
            assert np.array_equal(g2[:, o], g[:, j].astype(np.float64)) and np.array_equal(gm2[:, o], gm[:, j])
        else:
            assert np.all(gm2[:, o] == 0) and np.all(v2[:11 * N2].reshape(11, N2)[:, o] == 0)
            assert np.sum(parent == j) == 2
    assert np.array_equal(th2[11 * N2:], th[11 * N:].astype(np.float64))
    assert np.array_equal(m2[11 * N2:], m[11 * N:]) and np.array_equal(v2[11 * N2:], v[11 * N:])


def test_accumulate(dens):
    N = 50
    rng = np.random.default_rng(9)
    grad = rng.normal(0, 1, 11 * N + 12).astype(np.float32)
    acc, cnt = dens.accumulate(np.zeros((N, 4), np.float32), 0, grad, N)
    acc, cnt = dens.accumulate(acc, cnt, grad, N)
    g = grad[:3 * N].reshape(3, N).astype(np.float64)
    assert cnt == 2
    assert np.allclose(acc[:, 0], 2 * np.linalg.norm(g, axis=0), rtol=1e-6)
    assert np.allclose(acc[:, 1:], 2 * g.T, rtol=1e-6)
