"""Float64 oracle of the paper's normalised top-K forward model and of its
gradient.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference arm of ``bench.py`` import this module.  It does not
import the CUDA package and the CUDA package does not import it.

The model (Eq. 2 with the covariance of every primitive replaced by its
observed covariance, Eq. 5 with the slice intensity scale sigma_i = 1):

    I_hat_p = sum_{j in S} c_j E_pj / (sum_{j in S} E_pj + delta)
    E_pj    = exp(-1/2 v^T Sigma_obs,ij^-1 v),  v = T_i(u_p) - mu_j
    Sigma_obs,ij = Sigma_j + R_i Sigma_PSF R_i^T            (Eq. 4)
    S = S^K(T_i(u_p)): the K means nearest to the pixel's world position in
        Euclidean distance (Sec. 2.5, "Sparse Computation (Top-K)"); ties are
        broken by the smaller Gaussian index.

The loss is the MSE of the plain path, L = sum_p w_p (I_hat_p - I_p)^2.  The
gradient is the exact derivative of L for fixed neighbour sets (the top-K
selection is piecewise constant in the parameters).  Slice frames, rotations
and covariances come from ``oracle.py`` (the C oracle); everything else is
written out here in float64 numpy, one (pixel, Gaussian) pair at a time in
vectorised form.
"""
import numpy as np

from . import oracle as _o

FWHM_TO_SIGMA = 1.0 / 2.355


def _slices(stacks):
    """Per slice: (stack dict, slice index in stack, first global pixel)."""
    out, base = [], 0
    for s in stacks:
        for k in range(int(s["n_slices"])):
            out.append((s, k, base))
            base += int(s["H"]) * int(s["W"])
    return out


def pixel_geometry(stacks, theta, N, pix):
    """World position x (P,3), slice index (P), local coordinate u (P,3) of
    every listed pixel, and the slice frames R (M,3,3), t (M,3)."""
    N = int(N)
    sl_list = _slices(stacks)
    M = len(sl_list)
    pose = np.asarray(theta, np.float64)[11 * N:].reshape(M, 6)
    R, t = _o.slice_frames(stacks, pose)
    firsts = np.array([b for (_, _, b) in sl_list], np.int64)
    pix = np.asarray(pix, np.int64)
    sl = np.searchsorted(firsts, pix, side="right") - 1
    u = np.zeros((len(pix), 3), np.float64)
    for n, p in enumerate(pix):
        s, _, b = sl_list[sl[n]]
        a, col = divmod(int(p - b), int(s["W"]))
        u[n, 0] = (col - 0.5 * (int(s["W"]) - 1)) * float(s["dx"])
        u[n, 1] = (a - 0.5 * (int(s["H"]) - 1)) * float(s["dy"])
    x = np.einsum("pab,pb->pa", R[sl], u) + t[sl]
    return x, sl, u, R, t


def psf_var(stacks):
    """Sigma_PSF diagonal in slice axes (M,3): (FWHM / 2.355)^2."""
    out = []
    for (s, _, _) in _slices(stacks):
        out.append((np.asarray(s["fwhm"], np.float64) * FWHM_TO_SIGMA) ** 2)
    return np.array(out)


def means(theta, N):
    th = np.asarray(theta, np.float64)
    N = int(N)
    return np.stack([th[0:N], th[N:2 * N], th[2 * N:3 * N]], axis=1)


def knn(x, mu, K):
    """Indices (P,K) of the K means nearest each point, by squared Euclidean
    distance, ties to the smaller index, nearest first (brute force)."""
    d2 = ((x[:, None, :] - mu[None, :, :]) ** 2).sum(-1)
    order = np.argsort(d2, axis=1, kind="stable")
    return order[:, :int(K)]


def _pairs(stacks, theta, N, pix, K, nbr):
    x, sl, u, R, t = pixel_geometry(stacks, theta, N, pix)
    mu = means(theta, N)
    if nbr is None:
        nbr = knn(x, mu, K)
    nbr = np.asarray(nbr, np.int64)
    Sig = _o.gauss_cov(theta, N)                      # (N,3,3)
    var = psf_var(stacks)                             # (M,3)
    Rs = R[sl]                                        # (P,3,3)
    Spsf = np.einsum("pab,pb,pcb->pac", Rs, var[sl], Rs)  # R diag(var) R^T
    Sobs = Sig[nbr] + Spsf[:, None, :, :]             # (P,K,3,3)
    P = np.linalg.inv(Sobs)
    v = x[:, None, :] - mu[nbr]                       # (P,K,3)
    Pv = np.einsum("pkab,pkb->pka", P, v)
    E = np.exp(-0.5 * np.einsum("pka,pka->pk", v, Pv))
    return x, sl, u, R, nbr, Pv, E, var


def _slice_terms(slw, M, sl, model, I, w, loss_kind):
    """Per-slice outlier terms (Sec. 2.4): prediction sigma_i * model, pixel
    loss w (l(r) / omega_i + log omega_i) with log sigma_i = slw[i], log
    omega_i = slw[M + i] (slw None: sigma = omega = 1 without the log term).
    Returns (pred, per-pixel loss, dL/dmodel, per-pixel d/dlog sigma, d/dlog omega)."""
    w = np.broadcast_to(np.asarray(w, np.float64), model.shape)
    sig = np.exp(slw[sl]) if slw is not None else np.ones_like(model)
    lw = slw[M + sl] if slw is not None else np.zeros_like(model)
    iw = np.exp(-lw)
    pred = sig * model
    r = pred - I
    l = w * (np.abs(r) if loss_kind else r * r)
    dl = w * (np.sign(r) if loss_kind else 2.0 * r)
    loss_p = l * iw + (w * lw if slw is not None else 0.0)
    return pred, loss_p, sig * dl * iw, dl * iw * sig * model, w - l * iw


def forward(stacks, theta, N, pix, K, delta, nbr=None, I_obs=None, w_pix=1.0, loss_kind=0, lambda_reg=0.0,
            s_target=1.6, slw=None):
    """(pred, loss, nbr): predictions of the listed pixels, the loss when I_obs
    is given (data term MSE, loss_kind 0, or L1, 1, plus the scale regulariser
    of oracle.scale_reg and the per-slice terms of slw), and the neighbour sets."""
    th = np.asarray(theta, np.float64)
    c = th[10 * int(N):11 * int(N)]
    _, sl, _, R, nbr, _, E, _ = _pairs(stacks, th, N, pix, K, nbr)
    num = (c[nbr] * E).sum(1)
    den = E.sum(1) + float(delta)
    model = num / den
    sw = np.asarray(slw, np.float64) if slw is not None else None
    I = np.asarray(I_obs, np.float64) if I_obs is not None else np.zeros_like(model)
    pred, loss_p, _, _, _ = _slice_terms(sw, R.shape[0], sl, model, I, w_pix, loss_kind)
    loss = 0.0
    if I_obs is not None:
        loss = float(loss_p.sum())
        if lambda_reg:
            loss += _o.scale_reg(th, N, lambda_reg, s_target)[0]
    return pred, loss, nbr


def _drot_dquat(qh):
    """d R(q) / d q_k for a unit quaternion (w, x, y, z): four 3x3 matrices,
    from R = [[1-2(y^2+z^2), 2(xy-wz), 2(xz+wy)], [2(xy+wz), 1-2(x^2+z^2),
    2(yz-wx)], [2(xz-wy), 2(yz+wx), 1-2(x^2+y^2)]] differentiated entry by entry."""
    w, x, y, z = qh
    dw = np.array([[0, -2 * z, 2 * y], [2 * z, 0, -2 * x], [-2 * y, 2 * x, 0]], np.float64)
    dx = np.array([[0, 2 * y, 2 * z], [2 * y, -4 * x, -2 * w], [2 * z, 2 * w, -4 * x]], np.float64)
    dy = np.array([[-4 * y, 2 * x, 2 * w], [2 * x, 0, 2 * z], [-2 * w, 2 * z, -4 * y]], np.float64)
    dz = np.array([[-4 * z, -2 * w, 2 * x], [2 * w, -4 * z, 2 * y], [2 * x, 2 * y, 0]], np.float64)
    return [dw, dx, dy, dz]


def _skew(a):
    return np.array([[0.0, -a[2], a[1]], [a[2], 0.0, -a[0]], [-a[1], a[0], 0.0]])


def _drod_dr(r):
    """d Rod(r) / d r_k (three 3x3 matrices), Gallego & Yezzi (2015):
    dR/dr_k = ((r_k [r]x + [r x (I - R) e_k]x) / |r|^2) R, and [e_k]x at r = 0."""
    r = np.asarray(r, np.float64)
    th2 = float(r @ r)
    E = np.eye(3)
    if th2 < 1e-24:
        return [_skew(E[k]) for k in range(3)]
    Rr = _o.rodrigues(r)
    out = []
    for k in range(3):
        a = np.cross(r, (E - Rr) @ E[k])
        out.append(((r[k] * _skew(r) + _skew(a)) / th2) @ Rr)
    return out


def forward_backward(stacks, theta, N, pix, I_obs, w_pix, K, delta, nbr=None, want_abs=False, loss_kind=0,
                     lambda_reg=0.0, s_target=1.6, slw=None, slw_grad=None):
    """(pred, loss, grad, nbr) in float64; grad has the parameter-vector layout
    (11 N Gaussian entries component-major, then (r, tau) per slice).  With
    want_abs, also A (same layout): the sum of the absolute values of the
    products a float32 evaluation adds up for the entry, per (pixel,
    neighbour) pair: the pair's contribution for the means, amplitudes and
    poses; for the log-scales and the quaternion, every product of the chain
    through Sigma_j = R(q / |q|) diag(exp(2 ls)) R^T (whose terms cancel for
    near-isotropic Gaussians, where the exact entry is near 0)."""
    th = np.asarray(theta, np.float64)
    N = int(N)
    c = th[10 * N:11 * N]
    x, sl, u, R, nbr, Pv, E, var = _pairs(stacks, th, N, pix, K, nbr)
    num = (c[nbr] * E).sum(1)
    den = E.sum(1) + float(delta)
    model = num / den
    I = np.asarray(I_obs, np.float64)
    sw = np.asarray(slw, np.float64) if slw is not None else None
    pred, loss_p, gbar, gsig, gomg = _slice_terms(sw, R.shape[0], sl, model, I, w_pix, loss_kind)
    loss = float(loss_p.sum())
    if slw_grad is not None:
        Ms = R.shape[0]
        slw_grad[:] = 0.0
        np.add.at(slw_grad[:Ms], sl, gsig)
        np.add.at(slw_grad[Ms:], sl, gomg)
    pred_model = model                                            # the ratio before sigma_i
    gam = gbar[:, None] * (c[nbr] - pred_model[:, None]) / den[:, None] * E  # dL/dE times E
    dc_pair = gbar[:, None] * E / den[:, None]
    # per pair: dL/dmu = gam P v ; dL/dSigma_obs = 1/2 gam P v v^T P ; dL/dx = -gam P v
    g_mu = gam[:, :, None] * Pv
    G = 0.5 * gam[:, :, None, None] * np.einsum("pka,pkb->pkab", Pv, Pv)
    M = R.shape[0]
    grad = np.zeros(11 * N + 6 * M, np.float64)
    dmu = np.zeros((N, 3))
    dSig = np.zeros((N, 3, 3))
    dc = np.zeros(N)
    np.add.at(dmu, nbr, g_mu)
    np.add.at(dSig, nbr, G)
    np.add.at(dc, nbr, dc_pair)
    # Sigma_j = Rq diag(exp(2 ls)) Rq^T, Rq = R(q / |q|)
    ls = np.stack([th[3 * N:4 * N], th[4 * N:5 * N], th[5 * N:6 * N]], axis=1)
    q = np.stack([th[6 * N:7 * N], th[7 * N:8 * N], th[8 * N:9 * N], th[9 * N:10 * N]], axis=1)
    for j in range(N):
        qn = np.linalg.norm(q[j])
        qh = q[j] / qn
        Rq = _o.quat_to_rot(qh)
        s2 = np.exp(2.0 * ls[j])
        Gj = dSig[j]
        A = Rq.T @ Gj @ Rq
        for k in range(3):
            grad[(3 + k) * N + j] = 2.0 * s2[k] * A[k, k]
        dR = 2.0 * Gj @ Rq @ np.diag(s2)                          # dL/dRq (G symmetric)
        gq = np.array([np.sum(dR * D) for D in _drot_dquat(qh)])
        gq = (gq - qh * (qh @ gq)) / qn                            # through q / |q|
        for k in range(4):
            grad[(6 + k) * N + j] = gq[k]
        for k in range(3):
            grad[k * N + j] = dmu[j, k]
        grad[10 * N + j] = dc[j]
    # slice frames: x = R_i u + t_i ; Sigma_obs depends on R_i through R_i Sigma_PSF R_i^T
    dx_pix = -(gam[:, :, None] * Pv).sum(1)                      # dL/dx (P,3)
    GRi = np.zeros((M, 3, 3))
    Gti = np.zeros((M, 3))
    np.add.at(GRi, sl, np.einsum("pa,pb->pab", dx_pix, u))
    np.add.at(Gti, sl, dx_pix)
    Gobs = G.sum(1)                                               # (P,3,3) summed over neighbours
    Rs = R[sl]
    np.add.at(GRi, sl, 2.0 * np.einsum("pab,pbc,pc->pac", Gobs, Rs, var[sl]))
    # (R_i, t_i) -> (r, tau): R_i = Rod(r) R0_i, t_i = Rod(r) c0_i + tau
    pose = th[11 * N:].reshape(M, 6)
    i = 0
    for (s, k, _) in _slices(stacks):
        R0 = np.asarray(s["R"], np.float64)
        c0 = np.asarray(s["origin"], np.float64) + (k - 0.5 * (int(s["n_slices"]) - 1)) * float(s["thickness"]) * R0[:, 2]
        GRod = GRi[i] @ R0.T + np.outer(Gti[i], c0)
        for kk, D in enumerate(_drod_dr(pose[i, :3])):
            grad[11 * N + 6 * i + kk] = np.sum(GRod * D)
        grad[11 * N + 6 * i + 3:11 * N + 6 * i + 6] = Gti[i]
        i += 1
    g_reg = None
    if lambda_reg:
        L_reg, g_reg = _o.scale_reg(th, N, lambda_reg, s_target)
        loss += L_reg
        grad[3 * N:6 * N] += g_reg
    if not want_abs:
        return pred, loss, grad, nbr
    # per-pair contributions, each pushed through the same (linear) chains
    A = np.zeros_like(grad)
    absmu = np.zeros((N, 3))
    np.add.at(absmu, nbr, np.abs(g_mu))
    for k in range(3):
        A[k * N:(k + 1) * N] = absmu[:, k]
    absc = np.zeros(N)
    np.add.at(absc, nbr, np.abs(dc_pair))
    A[10 * N:11 * N] = absc
    qn_all = np.linalg.norm(q, axis=1)
    qh_all = q / qn_all[:, None]
    Rq_all = np.array([_o.quat_to_rot(qh_all[j]) for j in range(N)])
    s2_all = np.exp(2.0 * ls)
    Dq_all = np.array([_drot_dquat(qh_all[j]) for j in range(N)])       # (N,4,3,3)
    Rq_p, s2_p = Rq_all[nbr], s2_all[nbr]
    aR, aG = np.abs(Rq_p), np.abs(G)
    # ls_k: terms 2 s_k^2 Rq[a,k] G[a,b] Rq[b,k]
    dls_abs = 2.0 * s2_p * np.einsum("pkai,pkab,pkbi->pki", aR, aG, aR)
    absls = np.zeros((N, 3))
    np.add.at(absls, nbr, dls_abs)
    for k in range(3):
        A[(3 + k) * N:(4 + k) * N] = absls[:, k]
    # q: dL/dRq[a,b] = 2 sum_c G[a,c] Rq[c,b] s_b^2, then products with dR/dq_e, then the projection
    T = 2.0 * np.einsum("pkac,pkcb,pkb->pkab", aG, aR, s2_p)
    aD = np.abs(Dq_all[nbr])                                            # (P,K,4,3,3)
    te = np.einsum("pkab,pkeab->pke", T, aD)
    qh_p = np.abs(qh_all[nbr])
    absq_pair = (te + qh_p * np.einsum("pke,pke->pk", qh_p, te)[:, :, None]) / qn_all[nbr][:, :, None]
    absq = np.zeros((N, 4))
    np.add.at(absq, nbr, absq_pair)
    for k in range(4):
        A[(6 + k) * N:(7 + k) * N] = absq[:, k]
    gx_pair = -(gam[:, :, None] * Pv)                                   # (P,K,3)
    GR_pair = np.einsum("pka,pb->pkab", gx_pair, u) + 2.0 * np.einsum("pkab,pbc,pc->pkac", G, Rs, var[sl])
    R0s, c0s, dRods = [], [], []
    i = 0
    for (s_, k_, _) in _slices(stacks):
        R0 = np.asarray(s_["R"], np.float64)
        R0s.append(R0)
        c0s.append(np.asarray(s_["origin"], np.float64) + (k_ - 0.5 * (int(s_["n_slices"]) - 1)) *
                   float(s_["thickness"]) * R0[:, 2])
        dRods.append(np.array(_drod_dr(pose[i, :3])))
        i += 1
    R0s, c0s, dRods = np.array(R0s), np.array(c0s), np.array(dRods)
    GRod_pair = np.einsum("pkab,pcb->pkac", GR_pair, R0s[sl]) + np.einsum("pka,pb->pkab", gx_pair, c0s[sl])
    dr_pair = np.einsum("pkab,peab->pke", GRod_pair, dRods[sl])
    absr = np.zeros((M, 3))
    abst = np.zeros((M, 3))
    np.add.at(absr, sl, np.abs(dr_pair).sum(1))
    np.add.at(abst, sl, np.abs(gx_pair).sum(1))
    for i in range(M):
        A[11 * N + 6 * i:11 * N + 6 * i + 3] = absr[i]
        A[11 * N + 6 * i + 3:11 * N + 6 * i + 6] = abst[i]
    if g_reg is not None:
        A[3 * N:6 * N] += np.abs(g_reg)
    return pred, loss, grad, nbr, A
