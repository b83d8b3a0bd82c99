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
           "gsvr_cnn_conv_wgrad"]

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
    "gsvr_cnn_conv_dgrad": ([_vp, _vp, _i32, _i32, _i32, _i32, _vp, _i32, _vp, _vp, _vp, _vp], C.c_int),
    "gsvr_cnn_conv_wgrad": ([_vp, _vp, _vp, _i32, _i32, _i32, _i32, _i32, _vp, _vp], C.c_int),
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
    dcol = torch.empty(B * OH * OW * 9 * Ci, dtype=torch.float32, device=gy.device)
    dx = torch.empty((B, H, W, Ci), dtype=torch.bfloat16, device=gy.device)
    dx32 = torch.empty((B, H, W, Ci), dtype=torch.float32, device=gy.device)
    _check(None, lib.gsvr_cnn_conv_dgrad(_stream(stream), _dp(gy), B, H, W, Ci, _dp(w), Co, _dp(mask), _dp(dcol),
                                         _dp(dx), _dp(dx32)))
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


def pose_target(motion):
    """Network target of a per-slice motion (r rad, tau mm): (r, tau / 10)."""
    m = np.asarray(motion, np.float64)
    return np.concatenate([m[:, :3], m[:, 3:] / 10.0], axis=1).astype(np.float32)


def pose_from_output(out):
    o = np.asarray(out, np.float64)
    return np.concatenate([o[:, :3], o[:, 3:] * 10.0], axis=1)


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

    def render(self, phantom, motion):
        theta_g, N = inputs.grid_gaussians(phantom, h=self.h, s=self.h)
        gsvr.gsvr_set_gaussians(self.ctx.ctx, N, theta_g.astype(np.float32))
        gsvr.gsvr_set_poses(self.ctx.ctx, np.asarray(motion, np.float32).reshape(-1))
        gsvr.gsvr_forward(self.ctx.ctx)
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
