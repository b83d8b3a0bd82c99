"""Helpers shared by the GPU parity tests: tolerance checks and oracle calls.

Tolerances (stated targets: 1e-5 relative on forward values, 1e-4 relative on
gradients), read as follows:

- The CUDA path drops (pixel, Gaussian) pairs whose factor
  exp(-1/2 v^T Sigma_obs^-1 v) is below the cutoff (1e-7); the oracle sums every
  pair.  Each output may therefore differ by at most T = the sum of |terms| over
  the dropped pairs, which the oracle computes (trunc_pred, trunc_grad).
- Forward: |I_gpu - I_ref| <= 1e-5 max(|I_ref|, 1e-3 max|I_ref|) + T.  The floor
  keeps the relative test meaningful where the reference is ~0 (empty space).
- Gradients: every entry is a sum of signed terms (residuals of both signs), so
  the reference can cancel to ~0.  |g - g_ref| <= 1e-4 |g_ref| + tau A_ref + T,
  A_ref = sum of |terms| (float64, oracle): tau bounds the float32 rounding of
  the terms relative to their magnitude.
- Where residuals nearly cancel (a prediction close to its observation), the
  float32 rounding of the prediction itself, relative to the sum of |terms|
  it adds, moves the residual weight by more than tau of its own size.  The
  large-case tests therefore add tau B_ref, B_ref = the sum of |terms| with
  each residual weight 2 w (I_hat - I) replaced by 2 w sum_j |c_j g_pj|
  (oracle.local_grad's b_sel / b_pose).
- The tile kernels evaluate only the pairs inside the cut, so each prediction
  also lacks its truncated terms (up to trunc_pred), which moves every residual
  weight by up to 2 w trunc_pred.  The large-case tests add Bt_ref, the sum of
  |terms| at those residual weights (bt_sel / bt_pose).
"""
import numpy as np

FWD_RTOL = 1e-5
FWD_FLOOR = 1e-3
GRAD_RTOL = 1e-4
GRAD_ATOL_REL = 1e-6
CUTOFF = 1e-7


def forward_ok(pred, ref, trunc=None, rtol=FWD_RTOL, floor=FWD_FLOOR):
    scale = np.maximum(np.abs(ref), floor * max(np.abs(ref).max(), 1e-30))
    lim = rtol * scale + (trunc if trunc is not None else 0.0)
    err = np.abs(pred - ref)
    return err <= lim, float((err / lim).max()) if err.size else 0.0


def grad_limit(ref, absref, trunc=None, rtol=GRAD_RTOL, atol_rel=GRAD_ATOL_REL):
    return rtol * np.abs(ref) + atol_rel * absref + (trunc if trunc is not None else 0.0) + 1e-30


def grad_ok(g, ref, absref, trunc=None, rtol=GRAD_RTOL, atol_rel=GRAD_ATOL_REL):
    err = np.abs(g - ref)
    lim = grad_limit(ref, absref, trunc, rtol, atol_rel)
    ok = err <= lim
    plain = err <= rtol * np.abs(ref)
    return ok, float((err / lim).max()) if err.size else 0.0, float(plain.mean()) if err.size else 1.0


def rounding_floor(g, ref, absref, trunc):
    """Smallest tau that makes every entry pass: max over entries of
    (err - 1e-4 |ref| - T) / A (how much float32 rounding the case needed)."""
    err = np.abs(g - ref) - GRAD_RTOL * np.abs(ref) - trunc
    return float(np.max(err / np.maximum(absref, 1e-300))) if err.size else 0.0


def describe_grad(g, ref, absref, N, M, trunc=None):
    names = ["mu_x", "mu_y", "mu_z", "ls0", "ls1", "ls2", "qw", "qx", "qy", "qz", "c"]
    out = []
    err = np.abs(g - ref)
    lim = grad_limit(ref, absref, trunc)
    r = err / lim
    for k, nm in enumerate(names):
        if N == 0:
            break
        out.append("%s:%.3g" % (nm, r[k * N:(k + 1) * N].max()))
    if M:
        pr = r[11 * N:].reshape(M, 6)
        out.append("rot:%.3g tau:%.3g" % (pr[:, :3].max(), pr[:, 3:].max()))
    return " ".join(out)


def large_grad_check(g, ref, A, B, T, Bt, what):
    """Element-wise check of one gradient group at the large sizes:
    |g - ref| <= 1e-4 |ref| + tau (A + B) + T + Bt.  Prints the worst entry and
    the smallest tau that would pass; returns the worst err / tolerance."""
    err = np.abs(g - ref)
    lim = GRAD_RTOL * np.abs(ref) + GRAD_ATOL_REL * (A + B) + T + Bt + 1e-300
    r = err / lim
    k = int(np.argmax(r)) if r.size else 0
    need = float(np.max((err - GRAD_RTOL * np.abs(ref) - T - Bt) / np.maximum(A + B, 1e-300))) if r.size else 0.0
    plain = float(np.mean(err <= GRAD_RTOL * np.abs(ref))) if r.size else 1.0
    if r.size:
        print("%-12s n=%5d  max err/tol %.3f (g %.4e ref %.4e A %.3e B %.3e T %.3e Bt %.3e)  tau needed %.2e  "
              "plain 1e-4 relative %.3f" % (what, r.size, r[k], g[k], ref[k], A[k], B[k], T[k], Bt[k], need, plain))
    return float(r.max()) if r.size else 0.0
