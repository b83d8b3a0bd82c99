"""ctypes wrapper over the FP64 brute-force CPU oracle (``gsvr_oracle.c``).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference arm of ``bench.py`` import this module.  It does not
import the CUDA package and the CUDA package does not import it.

Inputs are plain numpy arrays and stack dictionaries as produced by the seeded
input generators: ``{"n_slices", "H", "W", "dx", "dy", "thickness", "R" (3x3,
columns = slice x, y, normal axes in world), "origin" (3), "fwhm" (3)}``.
The parameter vector is the component-major layout documented in
``gsvr_oracle.c`` (11 N Gaussian entries, then 6 per slice).

Every function computes the plain definition (Eq. 1, 3, 4 and the numerator of
Eq. 5 with the exact-convolution normalisation) by summing every
(pixel, Gaussian) pair in float64; see the C file for the passages followed.
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

_lib = None


class OrStack(C.Structure):
    _fields_ = [("n_slices", C.c_int32), ("H", C.c_int32), ("W", C.c_int32), ("pad_", C.c_int32),
                ("dx", C.c_double), ("dy", C.c_double), ("thickness", C.c_double),
                ("R", C.c_double * 9), ("origin", C.c_double * 3), ("fwhm", C.c_double * 3)]


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        _lib = C.CDLL(path)
        d, i64, vp = C.c_double, C.c_int64, C.c_void_p
        _lib.oracle_forward.argtypes = [C.c_int, vp, i64, vp, i64, vp, vp, d, C.c_int, C.c_int, vp, vp, vp]
        _lib.oracle_forward_backward.argtypes = [C.c_int, vp, i64, vp, i64, vp, vp, d, C.c_int, C.c_int, vp, vp,
                                                 vp, vp, vp, vp, vp, d, vp, vp]
        _lib.oracle_adam.argtypes = [i64, i64, vp, vp, vp, vp, vp, d, d, d, i64, vp]
        _lib.oracle_adam.restype = None
        _lib.oracle_build_slices.argtypes = [C.c_int, vp, vp, vp]
        _lib.oracle_build_slices.restype = i64
        _lib.oracle_slice_frames.argtypes = [C.c_int, vp, vp, vp, vp]
        _lib.oracle_quat_to_rot.argtypes = [vp, vp]
        _lib.oracle_quat_to_rot.restype = None
        _lib.oracle_rodrigues.argtypes = [vp, vp]
        _lib.oracle_rodrigues.restype = None
        _lib.oracle_gauss_cov.argtypes = [i64, vp, vp]
        _lib.oracle_gauss_cov.restype = None
        _lib.oracle_splitmix64.argtypes = [C.c_uint64, C.c_uint64]
        _lib.oracle_splitmix64.restype = C.c_uint64
        _lib.oracle_sample_positions.argtypes = [i64, i64, C.c_uint64, C.c_uint64, vp]
        _lib.oracle_num_threads.restype = C.c_int
        _lib.oracle_count_pairs.argtypes = [C.c_int, vp, i64, vp, i64, vp, d]
        _lib.oracle_count_pairs.restype = i64
        _lib.oracle_local_fd.argtypes = [C.c_int, vp, i64, vp, i64, vp, vp, d, C.c_int, d, i64, vp, vp, vp, vp, d, vp]
        _lib.oracle_local_fd.restype = C.c_int
        _lib.oracle_local_grad.argtypes = [C.c_int, vp, i64, vp, i64, vp, vp, d, C.c_int, d, d, i64, vp, vp, vp, vp,
                                           vp, vp, vp, vp, vp, vp, vp, vp, vp, vp]
        _lib.oracle_local_grad.restype = C.c_int
    return _lib


def _stacks(stacks):
    arr = (OrStack * max(1, len(stacks)))()
    for k, s in enumerate(stacks):
        a = arr[k]
        a.n_slices, a.H, a.W = int(s["n_slices"]), int(s["H"]), int(s["W"])
        a.dx, a.dy, a.thickness = float(s["dx"]), float(s["dy"]), float(s["thickness"])
        R = np.asarray(s["R"], dtype=np.float64).reshape(9)
        for e in range(9):
            a.R[e] = R[e]
        for e in range(3):
            a.origin[e] = float(s["origin"][e])
            a.fwhm[e] = float(s["fwhm"][e])
    return arr


def _f64(x):
    return np.ascontiguousarray(x, dtype=np.float64)


def _p(a):
    return a.ctypes.data if a is not None else None


def num_slices(stacks):
    return int(sum(int(s["n_slices"]) for s in stacks))


def num_pixels(stacks):
    return int(sum(int(s["n_slices"]) * int(s["H"]) * int(s["W"]) for s in stacks))


def num_threads():
    return int(lib().oracle_num_threads())


def scale_reg(theta, N, lambda_reg, s_target):
    """The scale regulariser of the paper's loss (Sec. 2.5, "Loss Function"):
    lambda_reg * sum_j sum_k (s_jk - s_target)^2 with s_jk = exp(ls_jk) the
    Gaussian's scales in mm; returns (value, gradient in the 3 N log-scales)."""
    N = int(N)
    s = np.exp(_f64(theta)[3 * N:6 * N])
    d = s - float(s_target)
    return float(lambda_reg) * float(np.sum(d * d)), 2.0 * float(lambda_reg) * d * s


def forward(stacks, theta, N, pix, I_obs=None, w_pix=1.0, norm_mode=0, loss_kind=0, lambda_reg=0.0, s_target=1.6,
            slw=None):
    """Predictions for the listed global pixels and the loss (float64): data
    term MSE (loss_kind 0) or L1 (1), plus the scale regulariser; slw (2 M:
    log sigma_i, log omega_i) switches on the per-slice outlier terms."""
    st = _stacks(stacks)
    th = _f64(theta)
    pix = np.ascontiguousarray(pix, dtype=np.int64)
    I = _f64(I_obs) if I_obs is not None else None
    pred = np.zeros(len(pix), np.float64)
    loss = np.zeros(1, np.float64)
    sw = _f64(slw) if slw is not None else None
    rc = lib().oracle_forward(len(stacks), C.addressof(st), int(N), _p(th), len(pix), _p(pix), _p(I),
                              float(w_pix), int(norm_mode), int(loss_kind), _p(sw), _p(pred), _p(loss))
    if rc != 0:
        raise RuntimeError("oracle_forward failed")
    L = float(loss[0])
    if lambda_reg:
        L += scale_reg(th, N, lambda_reg, s_target)[0]
    return pred, L


def forward_backward(stacks, theta, N, pix, I_obs, w_pix, norm_mode=0, sel=None, want_abs=True, cutoff=None,
                     loss_kind=0, lambda_reg=0.0, s_target=1.6, slw=None, slw_grad=None):
    """(pred, loss, grad, absgrad) in float64; grad has the parameter-vector layout.
    With `cutoff`, returns (pred, loss, grad, absgrad, trunc_pred, trunc_grad): the
    sums of |pair contributions| over the pairs below the cutoff, per output.
    loss_kind 0 / 1: MSE / L1 data term; lambda_reg > 0 adds the scale
    regulariser (its gradient terms counted in absgrad).  slw (2 M: log sigma_i,
    log omega_i) switches on the per-slice outlier terms; their gradient is
    written to slw_grad (2 M, when given)."""
    st = _stacks(stacks)
    th = _f64(theta)
    pix = np.ascontiguousarray(pix, dtype=np.int64)
    I = _f64(I_obs)
    M = num_slices(stacks)
    n = 11 * int(N) + 6 * M
    pred = np.zeros(len(pix), np.float64)
    loss = np.zeros(1, np.float64)
    grad = np.zeros(n, np.float64)
    absg = np.zeros(n, np.float64) if want_abs else None
    s = np.ascontiguousarray(sel, dtype=np.uint8) if sel is not None else None
    tp = np.zeros(len(pix), np.float64) if cutoff else None
    tg = np.zeros(n, np.float64) if cutoff else None
    if cutoff and absg is None:
        absg = np.zeros(n, np.float64)
    sw = _f64(slw) if slw is not None else None
    if slw_grad is not None:
        assert slw_grad.dtype == np.float64 and slw_grad.flags.c_contiguous and slw_grad.size == 2 * M
    rc = lib().oracle_forward_backward(len(stacks), C.addressof(st), int(N), _p(th), len(pix), _p(pix), _p(I),
                                       float(w_pix), int(norm_mode), int(loss_kind), _p(sw), _p(slw_grad), _p(s),
                                       _p(pred), _p(loss), _p(grad), _p(absg), float(cutoff or 0.0), _p(tp),
                                       _p(tg))
    if rc != 0:
        raise RuntimeError("oracle_forward_backward failed")
    if lambda_reg:
        Nn = int(N)
        Lr, gr = scale_reg(th, Nn, lambda_reg, s_target)
        loss[0] += Lr
        grad[3 * Nn:6 * Nn] += gr
        if absg is not None:
            absg[3 * Nn:6 * Nn] += np.abs(gr)
    if cutoff:
        return pred, float(loss[0]), grad, absg, tp, tg
    return pred, float(loss[0]), grad, absg


def count_pairs(stacks, theta, N, pix, cutoff=1e-7):
    """Pairs (listed pixel, Gaussian) whose exponent factor is at least `cutoff`."""
    st = _stacks(stacks)
    th = _f64(theta)
    pix = np.ascontiguousarray(pix, dtype=np.int64)
    n = lib().oracle_count_pairs(len(stacks), C.addressof(st), int(N), _p(th), len(pix), _p(pix), float(cutoff))
    if n < 0:
        raise RuntimeError("oracle_count_pairs failed")
    return int(n)


def adam(N, M, theta, grad, m, v, lr, beta1, beta2, eps, t, frozen=None):
    """One Adam step in float64; returns new (theta, m, v)."""
    th, mm, vv = _f64(theta).copy(), _f64(m).copy(), _f64(v).copy()
    g = _f64(grad)
    lr = _f64(lr)
    fz = np.ascontiguousarray(frozen, dtype=np.uint8) if frozen is not None else None
    lib().oracle_adam(int(N), int(M), _p(th), _p(g), _p(mm), _p(vv), _p(lr), float(beta1), float(beta2),
                      float(eps), int(t), _p(fz))
    return th, mm, vv


def slice_frames(stacks, theta_pose):
    """World rotation R_i (M,3,3) and centre t_i (M,3) of every slice."""
    st = _stacks(stacks)
    M = num_slices(stacks)
    pose = _f64(theta_pose).reshape(M * 6)
    R = np.zeros((M, 9), np.float64)
    t = np.zeros((M, 3), np.float64)
    lib().oracle_slice_frames(len(stacks), C.addressof(st), _p(pose), _p(R), _p(t))
    return R.reshape(M, 3, 3), t


def quat_to_rot(q):
    q = _f64(q)
    R = np.zeros(9, np.float64)
    lib().oracle_quat_to_rot(_p(q), _p(R))
    return R.reshape(3, 3)


def rodrigues(r):
    r = _f64(r)
    R = np.zeros(9, np.float64)
    lib().oracle_rodrigues(_p(r), _p(R))
    return R.reshape(3, 3)


def gauss_cov(theta, N):
    th = _f64(theta)
    S = np.zeros((int(N), 9), np.float64)
    lib().oracle_gauss_cov(int(N), _p(th), _p(S))
    return S.reshape(int(N), 3, 3)


def splitmix64(seed, ctr):
    return int(lib().oracle_splitmix64(C.c_uint64(seed), C.c_uint64(ctr)))


def sample_positions(n, n_s, seed, step):
    out = np.zeros(int(n_s), np.int64)
    rc = lib().oracle_sample_positions(int(n), int(n_s), C.c_uint64(seed), C.c_uint64(step), _p(out))
    if rc != 0:
        raise ValueError("bad sample size")
    return out


def local_fd(stacks, theta, N, pix, I_pix, w_pix, params, h, cut=1e-12, norm_mode=0, trunc_cut=1e-7):
    """Large cases: central differences of the loss over the listed pixels for
    the given parameter indices (steps h), the float64 predictions of those
    pixels and their sums of |terms| between trunc_cut and cut; pairs below
    `cut` are dropped (see oracle_local_fd).  Returns (fd, pred, trunc)."""
    st = _stacks(stacks)
    th = _f64(theta)
    px = np.ascontiguousarray(pix, dtype=np.int64)
    Ip = _f64(I_pix)
    pr = np.ascontiguousarray(params, dtype=np.int64)
    hh = _f64(h)
    fd = np.zeros(pr.size)
    pred = np.zeros(px.size)
    trunc = np.zeros(px.size)
    rc = lib().oracle_local_fd(len(stacks), st, int(N), th.ctypes.data, px.size, px.ctypes.data, Ip.ctypes.data,
                               float(w_pix), int(norm_mode), float(cut), pr.size, pr.ctypes.data, hh.ctypes.data,
                               fd.ctypes.data, pred.ctypes.data, float(trunc_cut), trunc.ctypes.data)
    if rc != 0:
        raise RuntimeError("oracle_local_fd failed")
    return fd, pred, trunc


def local_grad(stacks, theta, N, pix, I_pix, w_pix, sel, cut=1e-12, norm_mode=0, trunc_cut=1e-7):
    """Large cases: the analytic gradient of the MSE loss over the listed
    pixels (float64; pairs below `cut` dropped, pairs found through uniform
    grids; see oracle_local_grad).  Returns a dict:
    pred, trunc_pred (per listed pixel), loss;
    g_sel, a_sel, t_sel (11 x len(sel): gradient, sum of |terms| and that sum
    below trunc_cut, for every component of the selected Gaussians, rows in
    the parameter order mu_xyz, ls_012, q_wxyz, c);
    g_pose, a_pose, t_pose (6 M, the slice poses r, tau);
    b_sel, b_pose: the sums of |terms| with every residual weight
    2 w (I_hat_p - I_p) replaced by 2 w sum_j |c_j g_pj| (the scale at which a
    relative rounding error of the predictions moves each gradient entry);
    bt_sel, bt_pose: the same with 2 w trunc_pred_p (how far dropping the pairs
    below trunc_cut from the predictions moves each entry through the residuals)."""
    st = _stacks(stacks)
    th = _f64(theta)
    px = np.ascontiguousarray(pix, dtype=np.int64)
    Ip = _f64(I_pix)
    sl = np.ascontiguousarray(sel, dtype=np.int64)
    M = num_slices(stacks)
    out = {"pred": np.zeros(px.size), "trunc_pred": np.zeros(px.size), "loss": np.zeros(1)}
    for k in ("g_sel", "a_sel", "t_sel", "b_sel", "bt_sel"):
        out[k] = np.zeros((11, sl.size))
    for k in ("g_pose", "a_pose", "t_pose", "b_pose", "bt_pose"):
        out[k] = np.zeros(6 * M)
    rc = lib().oracle_local_grad(len(stacks), st, int(N), th.ctypes.data, px.size, px.ctypes.data,
                                 Ip.ctypes.data, float(w_pix), int(norm_mode), float(cut), float(trunc_cut),
                                 sl.size, _p(sl) if sl.size else None, *[_p(out[k]) for k in (
                                     "pred", "trunc_pred", "loss", "g_sel", "a_sel", "t_sel", "g_pose", "a_pose",
                                     "t_pose", "b_sel", "b_pose", "bt_sel", "bt_pose")])
    if rc != 0:
        raise RuntimeError("oracle_local_grad failed")
    out["loss"] = float(out["loss"][0])
    return out


def select_entries(N, M, sel):
    """Parameter-vector indices of local_grad's outputs: (11 x len(sel)) for
    the selected Gaussians' components, then the 6 M pose entries."""
    sel = np.asarray(sel, dtype=np.int64)
    comp = np.arange(11)[:, None] * int(N) + sel[None, :]
    return comp, 11 * int(N) + np.arange(6 * int(M))
