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
"""
import numpy as np

FWD_RTOL = 1e-5
FWD_FLOOR = 1e-3
GRAD_RTOL = 1e-4
GRAD_ATOL_REL = 2e-6
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
