"""FP64 reference of the learned pose-initialisation network (test
infrastructure only; see cnn_oracle.c).

Architecture (the slice-pose regressor standing in for the learned
pre-alignment that leaves the residual motion of Sec. 3.2): `len(channels) - 1`
conv 3x3 / stride 2 / pad 1 layers, each + bias + ReLU, NHWC; the last feature
map flattened position-major (its positions keep where the anatomy sits in the
slice, which a mean over positions would discard); concatenation with the
auxiliary vector (stack orientation and slice-position embedding); fc1 + ReLU;
fc2 -> 6 outputs
(r in rad, tau / 10 mm).  Loss = mean over the batch and the 6 outputs of the
squared error.

`forward_backward(..., bf16=True)` rounds to bfloat16 (round to nearest even)
at the points where the CUDA network stores bfloat16 operands: the input image,
the conv weights, every conv output (after ReLU) and every conv-output gradient
(after the ReLU mask).  Everything else is float64.
"""
import ctypes as C

import numpy as np

from . import oracle as _o

ARCH_CHANNELS = [1, 32, 64, 128, 256, 256, 512]
ARCH_HIDDEN = 256
ARCH_AUX = 25
ARCH_OUT = 6


def _lib():
    lib = _o.lib()
    if not getattr(lib, "_cnn_ready", False):
        i64, vp = C.c_int64, C.c_void_p
        lib.oracle_conv_fwd.argtypes = [i64, i64, i64, i64, i64, vp, vp, vp, C.c_int, vp, vp]
        lib.oracle_conv_fwd.restype = None
        lib.oracle_conv_dgrad.argtypes = [i64, i64, i64, i64, i64, vp, vp, vp, vp]
        lib.oracle_conv_dgrad.restype = None
        lib.oracle_conv_wgrad.argtypes = [i64, i64, i64, i64, i64, vp, vp, vp, vp, vp]
        lib.oracle_conv_wgrad.restype = None
        lib._cnn_ready = True
    return lib


def _p(a):
    return a.ctypes.data if a is not None else None


def _f(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def bf16(a):
    """Round float values to the nearest bfloat16 (ties to even), as float64."""
    f = np.ascontiguousarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    out = r.astype(np.uint32).view(np.float32).astype(np.float64)
    nan = np.isnan(f)
    out[nan] = np.nan
    return out


def conv_fwd(x, w, bias, relu=False, want_abs=False):
    """x [B][H][W][Ci], w [Co][3][3][Ci], bias [Co] -> y [B][OH][OW][Co] (and sum |terms|)."""
    x, w = _f(x), _f(w)
    B, H, W, Ci = x.shape
    Co = w.shape[0]
    y = np.empty((B, (H + 1) // 2, (W + 1) // 2, Co))
    a = np.empty_like(y) if want_abs else None
    b = _f(bias) if bias is not None else None
    _lib().oracle_conv_fwd(B, H, W, Ci, Co, _p(x), _p(w), _p(b), int(relu), _p(y), _p(a))
    return (y, a) if want_abs else y


def conv_dgrad(gy, w, H, W, want_abs=False):
    gy, w = _f(gy), _f(w)
    B, Co = gy.shape[0], gy.shape[3]
    Ci = w.shape[3]
    dx = np.empty((B, H, W, Ci))
    a = np.empty_like(dx) if want_abs else None
    _lib().oracle_conv_dgrad(B, H, W, Ci, Co, _p(gy), _p(w), _p(dx), _p(a))
    return (dx, a) if want_abs else dx


def conv_wgrad(gy, x, want_abs=False):
    gy, x = _f(gy), _f(x)
    B, H, W, Ci = x.shape
    Co = gy.shape[3]
    dw = np.empty((Co, 3, 3, Ci))
    db = np.empty(Co)
    a = np.empty_like(dw) if want_abs else None
    _lib().oracle_conv_wgrad(B, H, W, Ci, Co, _p(gy), _p(x), _p(dw), _p(db), _p(a))
    return (dw, db, a) if want_abs else (dw, db)


ARCH_POSITIONS = 4  # 2 x 2 final positions of a 128 x 128 input


def param_shapes(channels=ARCH_CHANNELS, hidden=ARCH_HIDDEN, aux=ARCH_AUX, out=ARCH_OUT, positions=ARCH_POSITIONS):
    """(name, shape) in the order of the flat parameter vector."""
    shapes = []
    for l in range(1, len(channels)):
        shapes.append(("conv%d.w" % l, (channels[l], 3, 3, channels[l - 1])))
        shapes.append(("conv%d.b" % l, (channels[l],)))
    shapes += [("fc1.w", (hidden, channels[-1] * positions + aux)), ("fc1.b", (hidden,)), ("fc2.w", (out, hidden)),
               ("fc2.b", (out,))]
    return shapes


def unflatten(vec, shapes):
    out, o = {}, 0
    for name, shp in shapes:
        n = int(np.prod(shp))
        out[name] = np.asarray(vec[o:o + n], dtype=np.float64).reshape(shp)
        o += n
    return out


def flatten(d, shapes):
    return np.concatenate([np.asarray(d[name], np.float64).reshape(-1) for name, _ in shapes])


def forward_backward(params, x, aux, target, bf16_points=True, want_grad=True):
    """params: dict name -> float64 array; x [B][H][W] slice images; aux [B][A];
    target [B][6].  Returns (loss, out [B][6], grads dict or None)."""
    rnd = bf16 if bf16_points else (lambda a: np.asarray(a, np.float64))
    nl = sum(1 for k in params if k.startswith("conv") and k.endswith(".w"))
    B = x.shape[0]
    acts = [rnd(np.asarray(x, np.float64)[..., None])]
    ws = [rnd(params["conv%d.w" % l]) for l in range(1, nl + 1)]
    for l in range(1, nl + 1):
        acts.append(rnd(conv_fwd(acts[-1], ws[l - 1], params["conv%d.b" % l], relu=True)))
    last = acts[-1]
    f = last.reshape(B, -1)
    h = np.concatenate([f, np.asarray(aux, np.float64)], axis=1)
    z1 = h @ params["fc1.w"].T + params["fc1.b"]
    a1 = np.maximum(z1, 0.0)
    out = a1 @ params["fc2.w"].T + params["fc2.b"]
    diff = out - np.asarray(target, np.float64)
    loss = float(np.mean(diff * diff))
    if not want_grad:
        return loss, out, None
    g = {}
    dout = 2.0 * diff / diff.size
    g["fc2.w"] = dout.T @ a1
    g["fc2.b"] = dout.sum(0)
    da1 = dout @ params["fc2.w"]
    dz1 = da1 * (z1 > 0)
    g["fc1.w"] = dz1.T @ h
    g["fc1.b"] = dz1.sum(0)
    dh = dz1 @ params["fc1.w"]
    gy = rnd(dh[:, :f.shape[1]].reshape(last.shape) * (last > 0))
    for l in range(nl, 0, -1):
        xin = acts[l - 1]
        g["conv%d.w" % l], g["conv%d.b" % l] = conv_wgrad(gy, xin)
        if l > 1:
            dx = conv_dgrad(gy, ws[l - 1], xin.shape[1], xin.shape[2])
            gy = rnd(dx * (xin > 0))
    return loss, out, g
