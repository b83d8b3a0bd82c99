"""Helpers shared by the GPU parity tests: tolerance checks and oracle calls."""
import numpy as np

# Forward values (stated target: 1e-5 relative).  Where the reference value is
# near zero (empty regions), relative error is ill-posed; the floor is 1e-3 of
# the largest value of the case.
FWD_RTOL = 1e-5
FWD_FLOOR = 1e-3

# Gradients (stated target: 1e-4 relative).  Every gradient entry is a sum of
# signed terms (residuals of both signs), so the reference can cancel to ~0;
# the float32 rounding of the terms is bounded by GRAD_ATOL_REL times the sum
# of their magnitudes A_ref (computed by the oracle in float64).
GRAD_RTOL = 1e-4
GRAD_ATOL_REL = 2e-5


def forward_ok(pred, ref, rtol=FWD_RTOL, floor=FWD_FLOOR):
    scale = np.maximum(np.abs(ref), floor * max(np.abs(ref).max(), 1e-30))
    err = np.abs(pred - ref)
    return err <= rtol * scale, float((err / scale).max()) if err.size else 0.0


def grad_ok(g, ref, absref, rtol=GRAD_RTOL, atol_rel=GRAD_ATOL_REL):
    err = np.abs(g - ref)
    lim = rtol * np.abs(ref) + atol_rel * absref + 1e-30
    ok = err <= lim
    plain = err <= rtol * np.abs(ref)
    return ok, float((err / lim).max()) if err.size else 0.0, float(plain.mean()) if err.size else 1.0


def describe_grad(g, ref, absref, N, M):
    names = ["mu_x", "mu_y", "mu_z", "ls0", "ls1", "ls2", "qw", "qx", "qy", "qz", "c"]
    out = []
    err = np.abs(g - ref)
    for k, nm in enumerate(names):
        sl = slice(k * N, (k + 1) * N)
        if N == 0:
            continue
        r = err[sl] / (GRAD_RTOL * np.abs(ref[sl]) + GRAD_ATOL_REL * absref[sl] + 1e-30)
        out.append("%s:%.3g" % (nm, r.max()))
    if M:
        pe = err[11 * N:].reshape(M, 6)
        pr = ref[11 * N:].reshape(M, 6)
        pa = absref[11 * N:].reshape(M, 6)
        r = pe / (GRAD_RTOL * np.abs(pr) + GRAD_ATOL_REL * pa + 1e-30)
        out.append("rot:%.3g tau:%.3g" % (r[:, :3].max(), r[:, 3:].max()))
    return " ".join(out)
