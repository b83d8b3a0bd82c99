"""ctypes binding of the slice-pose regression network (include/gsvr_cnn.h)
plus its data pipeline: training slices rendered by the library's own forward
model from randomised brain phantoms under random rigid motion, the auxiliary
input (stack orientation, slice-position embedding) and pose helpers.

Argument marshalling only: every layer runs in libgsvr.so's kernels; there is
no fallback when the library is missing.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import gsvr, inputs

lib = gsvr.lib
IMAGE, AUX, OUT = 128, 25, 6
EXPORTS = ["gsvr_cnn_create", "gsvr_cnn_destroy", "gsvr_cnn_last_error", "gsvr_cnn_views", "gsvr_cnn_forward",
           "gsvr_cnn_loss_backward", "gsvr_cnn_adam_step", "gsvr_cnn_conv_forward", "gsvr_cnn_conv_dgrad",
           "gsvr_cnn_conv_wgrad", "gsvr_cnn_gemm", "gsvr_cnn_sync_status"]

_vp, _i32, _i64, _u64, _f = C.c_void_p, C.c_int32, C.c_int64, C.c_uint64, C.c_float
_SIG = {
    "gsvr_cnn_create": ([C.POINTER(_vp), _i32, _vp, _i32, _u64], C.c_int),
    "gsvr_cnn_destroy": ([_vp], C.c_int),
    "gsvr_cnn_last_error": ([_vp], C.c_char_p),
    "gsvr_cnn_views": ([_vp, C.POINTER(_vp), C.POINTER(_vp), C.POINTER(_i64)], C.c_int),
    "gsvr_cnn_forward": ([_vp, _vp, _vp, _i32, _vp], C.c_int),
    "gsvr_cnn_loss_backward": ([_vp, _vp, _vp, _vp, _i32, _vp], C.c_int),
    "gsvr_cnn_adam_step": ([_vp, _f, _f, _f, _f, _i64], C.c_int),
    "gsvr_cnn_conv_forward": ([_vp, _vp, _i32, _i32, _i32, _i32, _vp, _vp, _i32, _i32, _vp, _vp], C.c_int),
    "gsvr_cnn_conv_dgrad": ([_vp, _vp, _i32, _i32, _i32, _i32, _vp, _i32, _vp, _vp, _vp], C.c_int),
    "gsvr_cnn_conv_wgrad": ([_vp, _vp, _vp, _i32, _i32, _i32, _i32, _i32, _vp, _vp], C.c_int),
    "gsvr_cnn_gemm": ([_vp, _vp, _vp, _i32, _i32, _i32, _vp, _i32, _vp], C.c_int),
    "gsvr_cnn_sync_status": ([_vp], C.c_int),
}
for _name, (_args, _res) in _SIG.items():
    _fn = getattr(lib, _name)
    _fn.argtypes = _args
    _fn.restype = _res


def _check(net, status):
    if status != gsvr.GSVR_OK:
        msg = lib.gsvr_cnn_last_error(net)
        raise gsvr.GsvrError(status, msg.decode() if msg else "")
    return status


def _dp(t):
    """Device pointer of a CUDA tensor (None -> NULL)."""
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return t.data_ptr()


def _stream(stream):
    return None if stream is None else int(stream.cuda_stream if hasattr(stream, "cuda_stream") else stream)


# ------------------------------------------------------------ layer primitives
def conv_forward(x, w, bias, relu=True, want_f32=False, stream=None):
    """x [B][H][W][Ci] bf16, w [Co][3][3][Ci] bf16, bias [Co] f32 (CUDA tensors)."""
    import torch
    B, H, W, Ci = x.shape
    Co = w.shape[0]
    y = torch.empty((B, (H + 1) // 2, (W + 1) // 2, Co), dtype=torch.bfloat16, device=x.device)
    y32 = torch.empty(y.shape, dtype=torch.float32, device=x.device) if want_f32 else None
    _check(None, lib.gsvr_cnn_conv_forward(_stream(stream), _dp(x), B, H, W, Ci, _dp(w), _dp(bias), Co, int(relu),
                                           _dp(y), _dp(y32)))
    return (y, y32) if want_f32 else y


def conv_dgrad(gy, w, H, W, mask=None, stream=None):
    """Input gradient (bf16, float32) of a conv layer; gy [B][OH][OW][Co] bf16."""
    import torch
    B, OH, OW, Co = gy.shape
    Ci = w.shape[3]
    dx = torch.empty((B, H, W, Ci), dtype=torch.bfloat16, device=gy.device)
    dx32 = torch.empty((B, H, W, Ci), dtype=torch.float32, device=gy.device)
    _check(None, lib.gsvr_cnn_conv_dgrad(_stream(stream), _dp(gy), B, H, W, Ci, _dp(w), Co, _dp(mask), _dp(dx),
                                         _dp(dx32)))
    return dx, dx32


def conv_wgrad(gy, x, stream=None):
    """(dw [Co][3][3][Ci], db [Co]) float32 of a conv layer."""
    import torch
    B, H, W, Ci = x.shape
    Co = gy.shape[3]
    dw = torch.zeros((Co, 3, 3, Ci), dtype=torch.float32, device=x.device)
    db = torch.zeros(Co, dtype=torch.float32, device=x.device)
    _check(None, lib.gsvr_cnn_conv_wgrad(_stream(stream), _dp(gy), _dp(x), B, H, W, Ci, Co, _dp(dw), _dp(db)))
    return dw, db


def sync_status():
    """Synchronise the device; raise GsvrError if a layer primitive's bounded wait ran out."""
    _check(None, lib.gsvr_cnn_sync_status(None))


def gemm(A, B, tensor_memory=1, stream=None):
    """C = A B^T (A [M][K], B [N][K] bf16 CUDA tensors) in float32; returns (C, status word).
    tensor_memory: 1 tcgen05 with tensor-map operand copies, 2 tcgen05 with per-thread copies, 0 mma.sync."""
    import torch
    M, K = A.shape
    N = B.shape[0]
    C = torch.zeros((M, N), dtype=torch.float32, device=A.device)
    status = torch.zeros(1, dtype=torch.int32, device=A.device)
    _check(None, lib.gsvr_cnn_gemm(_stream(stream), _dp(A), _dp(B), M, N, K, _dp(C), int(tensor_memory),
                                   _dp(status)))
    return C, status


# ---------------------------------------------------------------- the model
class PoseNet:
    """Owning wrapper of a gsvr_cnn; params / grads are zero-copy float32 views."""

    def __init__(self, max_batch=256, seed=0, device=0, stream=None):
        self.device = device
        self.stream = stream
        h = _vp()
        _check(None, lib.gsvr_cnn_create(C.byref(h), int(device), _stream(stream), int(max_batch), C.c_uint64(seed)))
        self.net = h
        self.max_batch = int(max_batch)
        p, g, n = _vp(), _vp(), _i64()
        _check(self.net, lib.gsvr_cnn_views(self.net, C.byref(p), C.byref(g), C.byref(n)))
        self.n_params = int(n.value)
        self.params = gsvr.device_view(p.value, self.n_params, device=device)
        self.grads = gsvr.device_view(g.value, self.n_params, device=device)

    def forward(self, x, aux):
        import torch
        B = x.shape[0]
        out = torch.empty((B, OUT), dtype=torch.float32, device=x.device)
        _check(self.net, lib.gsvr_cnn_forward(self.net, _dp(x), _dp(aux), int(B), _dp(out)))
        return out

    def loss_backward(self, x, aux, target):
        import torch
        loss = torch.zeros(1, dtype=torch.float64, device=x.device)
        _check(self.net, lib.gsvr_cnn_loss_backward(self.net, _dp(x), _dp(aux), _dp(target), int(x.shape[0]),
                                                    _dp(loss)))
        return loss

    def adam_step(self, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
        _check(self.net, lib.gsvr_cnn_adam_step(self.net, float(lr), float(beta1), float(beta2), float(eps), int(t)))

    def sync_status(self):
        """Synchronise; raise GsvrError(GSVR_ERR_TIMEOUT) if a bounded wait ran out since the last check."""
        _check(self.net, lib.gsvr_cnn_sync_status(self.net))

    def close(self):
        if self.net:
            lib.gsvr_cnn_destroy(self.net)
            self.net = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------- data pipeline
def slice_embedding(offset_mm):
    """16-d sinusoidal embedding of a slice's offset along its stack normal:
    (sin, cos)(2 pi z / L_k), wavelengths L_k = 8 mm x 2^k, k = 0..7."""
    z = np.asarray(offset_mm, np.float64)[..., None]
    L = 8.0 * 2.0 ** np.arange(8)
    ang = 2 * np.pi * z / L
    return np.concatenate([np.sin(ang), np.cos(ang)], axis=-1)


def aux_for_stacks(stacks):
    """Per slice (stack order): R0 row-major (9) and the slice-offset embedding (16)."""
    rows = []
    for s in stacks:
        n = s["n_slices"]
        off = (np.arange(n) - 0.5 * (n - 1)) * s["thickness"]
        R = np.broadcast_to(np.asarray(s["R"], np.float64).reshape(1, 9), (n, 9))
        rows.append(np.concatenate([R, slice_embedding(off)], axis=1))
    return np.concatenate(rows).astype(np.float32)


def _frames(aux):
    """Per-slice nominal rotations R0 [n][3][3] from the auxiliary input rows."""
    return np.asarray(aux, np.float64)[:, :9].reshape(-1, 3, 3)


def pose_target(motion, aux):
    """Network target of a per-slice motion (r rad, tau mm), expressed in the
    slice's own frame: r_s = R0^T r and tau_s = R0^T tau (R_i = Rod(r) R0 =
    R0 Rod(r_s), so r_s is the rotation applied in slice axes: its z part turns
    the image in plane, its x, y parts tilt it; tau_s is the in-plane shift and
    the shift along the normal), as (r_s, tau_s / 10)."""
    m = np.asarray(motion, np.float64)
    R0 = _frames(aux)
    r_s = np.einsum("nji,nj->ni", R0, m[:, :3])
    t_s = np.einsum("nji,nj->ni", R0, m[:, 3:])
    return np.concatenate([r_s, t_s / 10.0], axis=1).astype(np.float32)


def pose_from_output(out, aux):
    """World-frame motion (r, tau) of network outputs (the inverse of pose_target)."""
    o = np.asarray(out, np.float64)
    R0 = _frames(aux)
    r = np.einsum("nij,nj->ni", R0, o[:, :3])
    t = np.einsum("nij,nj->ni", R0, o[:, 3:] * 10.0)
    return np.concatenate([r, t], axis=1)


def normalise_slices(img):
    """Per-slice scale to unit mean over the slice's nonzero pixels (torch, device)."""
    import torch
    B = img.shape[0]
    flat = img.reshape(B, -1)
    nz = (flat > 1e-3).float()
    mean = (flat * nz).sum(1) / nz.sum(1).clamp(min=1.0)
    return img / mean.clamp(min=1e-3).reshape(B, 1, 1)


class SliceRenderer:
    """Renders training slices with the library's forward model: three
    orthogonal stacks of n_slices x 128 x 128 px at 1 x 1 mm, `thickness` mm,
    centred on the origin; one context reused for every phantom (Gaussians on
    an h-mm grid inside the phantom, per-slice motion set as the slice poses,
    every pixel evaluated).  Returns (images [M][128][128] float32 on the
    device, the motion used)."""

    def __init__(self, n_slices=32, thickness=3.5, h=1.5, device=0, stream=None):
        import torch
        self.stacks = [inputs.stack(n_slices, IMAGE, IMAGE, 1.0, 1.0, thickness, R)
                       for R in (inputs.AXIAL, inputs.CORONAL, inputs.SAGITTAL)]
        self.M = inputs.n_slices_total(self.stacks)
        self.h = h
        P = inputs.n_pixels_total(self.stacks)
        self.stream = stream if stream is not None else torch.cuda.Stream(device=device)
        case = {"stacks": self.stacks, "N": 1, "theta": np.zeros(11 + 6 * self.M, np.float32),
                "I": np.zeros(P, np.float32), "mask": np.ones(P, np.uint8)}
        case["theta"][6] = 1.0
        self.ctx = gsvr.Context(case, device=device, stream=self.stream.cuda_stream, tile_h=12, tile_w=12)
        self.aux = aux_for_stacks(self.stacks)
        # nominal world position of every pixel (for the acquisition mask)
        pos = []
        for st in self.stacks:
            n = st["n_slices"]
            a = (np.arange(IMAGE) - 0.5 * (IMAGE - 1)) * st["dy"]
            b = (np.arange(IMAGE) - 0.5 * (IMAGE - 1)) * st["dx"]
            A, Bg = np.meshgrid(a, b, indexing="ij")
            for k in range(n):
                c0 = st["origin"] + (k - 0.5 * (n - 1)) * st["thickness"] * st["R"][:, 2]
                pos.append(Bg.reshape(-1, 1) * st["R"][:, 0] + A.reshape(-1, 1) * st["R"][:, 1] + c0)
        self.pos = torch.from_numpy(np.concatenate(pos).astype(np.float32)).to("cuda:%d" % device)

    def mask(self, axes, dilate_mm=15.0):
        """Acquisition mask of every slice: the phantom's outer ellipsoid (semi-axes
        `axes`) dilated by dilate_mm, at the nominal pixel positions (as the
        simulated acquisitions)."""
        import torch
        ax = torch.tensor(np.asarray(axes, np.float32) + dilate_mm, device=self.pos.device)
        return ((self.pos / ax) ** 2).sum(1).reshape(self.M, IMAGE, IMAGE) <= 1.0

    def render(self, phantom, motion):
        theta_g, N = inputs.grid_gaussians(phantom, h=self.h, s=self.h)
        return self.render_gaussians(theta_g, N, motion)

    def render_gaussians(self, theta_g, N, motion):
        import torch
        self.ctx.set_gaussians(np.asarray(theta_g, np.float32), N)
        gsvr.gsvr_set_poses(self.ctx.ctx, np.asarray(motion, np.float32).reshape(-1))
        gsvr.gsvr_forward(self.ctx.ctx)
        # the forward runs on the renderer's stream: order the caller's stream after it
        torch.cuda.current_stream(self.stream.device).wait_stream(self.stream)
        img = self.ctx.pred.reshape(self.M, IMAGE, IMAGE).clone()
        return img

    def close(self):
        self.ctx.close()


def rician(img, frac, gen):
    """sqrt((I + n1)^2 + n2^2), n ~ N(0, (frac * max)^2) per slice (torch, device)."""
    import torch
    sd = frac * img.reshape(img.shape[0], -1).amax(1).clamp(min=1e-6).reshape(-1, 1, 1)
    n1 = torch.randn(img.shape, device=img.device, generator=gen) * sd
    n2 = torch.randn(img.shape, device=img.device, generator=gen) * sd
    return torch.sqrt((img + n1) ** 2 + n2 ** 2)


def content_fraction(img, level=0.1):
    """Fraction of each slice's pixels above `level` times the slice set's 99th
    percentile intensity (torch, device)."""
    import torch
    ref = torch.quantile(img.reshape(-1)[::97].float(), 0.99).clamp(min=1e-6)
    return (img > level * ref).float().reshape(img.shape[0], -1).mean(1)


def _phantom_grid(args):
    seed, jitter, h = args
    ph = inputs.BrainPhantom(seed, jitter=jitter)
    theta_g, N = inputs.grid_gaussians(ph, h=h, s=h)
    return theta_g.astype(np.float32), N, np.asarray(ph.axes)


def make_training_set(n_phantoms, motions_per_phantom=2, n_slices=20, max_deg=20.0, max_mm=10.0, noise=0.02,
                      seed=0, min_content=0.02, jitter=0.15, h=1.5, device=0, workers=8, log=None):
    """Training slices rendered by the forward model: phantoms of the
    canonical-frame family (seeds 10^6 (seed + 1) + p, disjoint from evaluation
    seeds; their Gaussian grids built on `workers` spawned host processes),
    Gaussians on an h-mm grid, per-slice motion U(+-max_deg) / U(+-max_mm),
    Rician noise, zero outside the acquisition mask (phantom dilated by 15 mm),
    per-slice unit-mean scaling; slices with less than min_content brain
    content are dropped.  Returns device tensors (x [n][128][128],
    aux [n][25], target [n][6])."""
    import multiprocessing as mp

    import torch
    rng = np.random.default_rng(seed)
    gen = torch.Generator(device="cuda:%d" % device).manual_seed(seed)
    ren = SliceRenderer(n_slices=n_slices, h=h, device=device)
    aux_all = torch.from_numpy(ren.aux).to("cuda:%d" % device)
    xs, auxs, tgts = [], [], []
    jobs = [(1_000_000 * (seed + 1) + p, jitter, h) for p in range(n_phantoms)]
    pool = mp.get_context("spawn").Pool(workers) if workers > 1 else None
    it = pool.imap(_phantom_grid, jobs, chunksize=4) if pool else map(_phantom_grid, jobs)
    try:
        for p, (theta_g, N, axes) in enumerate(it):
            msk = ren.mask(axes)
            for _ in range(motions_per_phantom):
                motion = inputs.random_motion(rng, ren.M, max_deg, max_mm)
                img = ren.render_gaussians(theta_g, N, motion)
                img = rician(img, noise, gen) * msk
                keep = content_fraction(img) > min_content
                xs.append(normalise_slices(img[keep]))
                auxs.append(aux_all[keep])
                tgts.append(torch.from_numpy(pose_target(motion, ren.aux)).to(img.device)[keep])
            if log and (p + 1) % max(1, n_phantoms // 10) == 0:
                log("rendered %d / %d phantoms, %d slices" % (p + 1, n_phantoms, sum(x.shape[0] for x in xs)))
    finally:
        if pool:
            pool.close()
            pool.join()
    ren.close()
    return torch.cat(xs), torch.cat(auxs), torch.cat(tgts)


def train(net, X, A, Y, epochs=20, batch=256, lr=1e-3, seed=0, val_frac=0.05, log=None):
    """Adam with a cosine learning-rate schedule over `epochs` passes of random
    batches; the last val_frac of the set is held out.  Returns the history
    [(epoch, train loss, validation loss, seconds)]."""
    import math
    import time

    import torch
    n = X.shape[0]
    n_val = max(batch, int(n * val_frac))
    n_tr = n - n_val
    g = torch.Generator(device=X.device).manual_seed(seed)
    hist, t, t0 = [], 0, time.time()
    for ep in range(epochs):
        lr_ep = lr * 0.5 * (1.0 + math.cos(math.pi * ep / epochs))
        perm = torch.randperm(n_tr, device=X.device, generator=g)
        tot = torch.zeros(1, dtype=torch.float64, device=X.device)
        steps = 0
        for s0 in range(0, n_tr - batch + 1, batch):
            idx = perm[s0:s0 + batch]
            tot += net.loss_backward(X.index_select(0, idx), A.index_select(0, idx), Y.index_select(0, idx))
            t += 1
            steps += 1
            net.adam_step(t, lr=lr_ep)
        vl = evaluate_loss(net, X[n_tr:], A[n_tr:], Y[n_tr:], batch)
        net.sync_status()
        hist.append((ep + 1, float(tot.item()) / max(steps, 1), vl, time.time() - t0))
        if log:
            log("epoch %d: train %.4f  val %.4f  (%.1f s)" % hist[-1])
    return hist


def predict(net, X, A, batch=256):
    """Network outputs for X, A in batches of at most the network's max_batch."""
    import torch
    batch = max(1, min(int(batch), net.max_batch))
    outs = [net.forward(X[s:s + batch].contiguous(), A[s:s + batch].contiguous()) for s in range(0, X.shape[0], batch)]
    return torch.cat(outs)


def evaluate_loss(net, X, A, Y, batch=256):
    out = predict(net, X, A, batch)
    return float(((out - Y) ** 2).mean().item())


def _rod(r):
    """Rotation matrices of axis-angle vectors r [n][3] (Rodrigues)."""
    r = np.asarray(r, np.float64)
    th = np.linalg.norm(r, axis=1)
    k = np.where(th[:, None] > 1e-12, r / np.maximum(th, 1e-300)[:, None], 0.0)
    K = np.zeros((r.shape[0], 3, 3))
    K[:, 0, 1], K[:, 0, 2], K[:, 1, 2] = -k[:, 2], k[:, 1], -k[:, 0]
    K[:, 1, 0], K[:, 2, 0], K[:, 2, 1] = k[:, 2], -k[:, 1], k[:, 0]
    s, c = np.sin(th)[:, None, None], np.cos(th)[:, None, None]
    return np.eye(3)[None] + s * K + (1.0 - c) * (K @ K)


def pose_errors_on_set(net, X, A, Y, batch=256):
    """Per-slice pose errors of the network and of the nominal (zero-motion)
    start on a rendered set (targets as pose_target): rotation angle of
    Rod(r_pred)^T Rod(r_true) in degrees and translation error in mm, both
    frame independent.  Returns a dict of arrays."""
    out = predict(net, X, A, batch).double().cpu().numpy()
    y = Y.double().cpu().numpy()
    Rp, Rt = _rod(out[:, :3]), _rod(y[:, :3])
    cosang = np.clip((np.einsum("nij,nij->n", Rp, Rt) - 1.0) / 2.0, -1.0, 1.0)
    return {"net_rot_deg": np.degrees(np.arccos(cosang)),
            "net_trans_mm": 10.0 * np.linalg.norm(out[:, 3:] - y[:, 3:], axis=1),
            "nominal_rot_deg": np.degrees(np.linalg.norm(y[:, :3], axis=1)),
            "nominal_trans_mm": 10.0 * np.linalg.norm(y[:, 3:], axis=1)}

