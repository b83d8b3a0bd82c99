"""ctypes binding of libgsvr.so, with the names of the C ABI (include/gsvr.h).

Argument marshalling only: every step of the forward model, the adjoint and
the optimiser runs in the library's CUDA kernels.  Importing this module loads
the library and raises ImportError when it is missing -- there is no fallback.

Arrays may be numpy arrays (host memory) or CUDA torch tensors (device
memory); the binding passes the pointer and the matching GSVR_MEM_* kind.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgsvr.so")

GSVR_OK = 0
STATUS_NAMES = {0: "GSVR_OK", 1: "GSVR_ERR_INVALID_ARG", 2: "GSVR_ERR_CUDA", 3: "GSVR_ERR_CAPACITY",
                4: "GSVR_ERR_NONFINITE", 5: "GSVR_ERR_TIMEOUT", 6: "GSVR_ERR_STATE", 7: "GSVR_ERR_NOMEM"}
globals().update({v: k for k, v in STATUS_NAMES.items()})
GSVR_MEM_HOST, GSVR_MEM_DEVICE = 0, 1
GSVR_NORM_EXACT, GSVR_NORM_LITERAL = 0, 1

EXPORTS = ["gsvr_abi_version", "gsvr_last_error", "gsvr_create", "gsvr_destroy", "gsvr_set_stacks",
           "gsvr_set_observations", "gsvr_set_gaussians", "gsvr_set_poses", "gsvr_set_frozen",
           "gsvr_set_pixel_sample", "gsvr_sample_pixels", "gsvr_forward", "gsvr_backward", "gsvr_adam_step",
           "gsvr_step_host", "gsvr_get_sample", "gsvr_get_views", "gsvr_get_stats", "gsvr_sync_status",
           "gsvr_timing_reset", "gsvr_get_kernel_times", "gsvr_count_pairs", "gsvr_forward_noalloc",
           "gsvr_alu_peaks", "gsvr_set_subjects", "gsvr_sample_pixels_subjects", "gsvr_get_subject_losses",
           "gsvr_graph_capture", "gsvr_graph_launch", "gsvr_set_step", "gsvr_set_tiling", "gsvr_get_tiling",
           "gsvr_tune_space_default", "gsvr_autotune", "gsvr_reserve", "gsvr_set_topk", "gsvr_get_topk_neighbors",
           "gsvr_set_objective", "gsvr_set_slice_weights", "gsvr_slice_weight_views", "gsvr_init_means",
           "gsvr_volume_metrics", "gsvr_fp64_peak", "gsvr_densify_accumulate", "gsvr_densify_stats",
           "gsvr_densify", "gsvr_ffma2_peak", "gsvr_set_subject_active", "gsvr_save", "gsvr_load",
           "gsvr_checkpoint_info", "gsvr_test_wait_timeout",
           "gsvr_set_sample_total"]
STAGES = ["sample", "prep", "bin", "fwd_eval", "bwd_eval", "grad", "adam", "unused"]


class GsvrError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, str(status)), msg))
        self.status = status


class StackDesc(C.Structure):
    _fields_ = [("n_slices", C.c_int32), ("H", C.c_int32), ("W", C.c_int32), ("reserved", C.c_int32),
                ("dx", C.c_float), ("dy", C.c_float), ("thickness", C.c_float), ("R", C.c_float * 9),
                ("origin", C.c_float * 3), ("fwhm", C.c_float * 3)]


class Config(C.Structure):
    _fields_ = [("cutoff_rel", C.c_float), ("tile_h", C.c_int32), ("tile_w", C.c_int32), ("norm_mode", C.c_int32),
                ("fixed_capacity", C.c_int32), ("timing", C.c_int32), ("cap_records", C.c_int64),
                ("cap_keys", C.c_int64), ("seed", C.c_uint64)]


class DensifyCfg(C.Structure):
    _fields_ = [("grad_threshold", C.c_float), ("log_scale_threshold", C.c_float), ("prune_amplitude", C.c_float),
                ("split_factor", C.c_float), ("clone_offset", C.c_float), ("mass_preserving", C.c_int32),
                ("max_gaussians", C.c_int64)]


class AdamCfg(C.Structure):
    _fields_ = [("lr_mu", C.c_float), ("lr_ls", C.c_float), ("lr_q", C.c_float), ("lr_c", C.c_float),
                ("lr_rot", C.c_float), ("lr_trans", C.c_float), ("beta1", C.c_float), ("beta2", C.c_float),
                ("eps", C.c_float), ("step_every", C.c_int32), ("gamma", C.c_float)]


class KernelTimes(C.Structure):
    _fields_ = [("ms", C.c_double * 8), ("calls", C.c_int64 * 8), ("pairs_evaluated", C.c_int64),
                ("kernel_launches", C.c_int64), ("bwd_pairs_evaluated", C.c_int64)]


class Tiling(C.Structure):
    _fields_ = [("tile_h", C.c_int32), ("tile_w", C.c_int32), ("fwd_px_per_thread", C.c_int32),
                ("fwd_blocks_per_sm", C.c_int32), ("bwd_blocks_per_sm", C.c_int32), ("queue_order", C.c_int32),
                ("ms", C.c_float)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class CheckpointHeader(C.Structure):
    _fields_ = [("version", C.c_int32), ("n_stacks", C.c_int32), ("n_slices", C.c_int32), ("reserved", C.c_int32),
                ("n_pixels", C.c_int64), ("n_gaussians", C.c_int64), ("step", C.c_int64)]


class Views(C.Structure):
    _fields_ = [("theta", C.c_void_p), ("grad", C.c_void_p), ("adam_m", C.c_void_p), ("adam_v", C.c_void_p),
                ("pred", C.c_void_p), ("rbar", C.c_void_p), ("loss", C.c_void_p), ("n_gauss", C.c_int64),
                ("n_slices", C.c_int64), ("n_pixels", C.c_int64), ("n_params", C.c_int64)]


class Stats(C.Structure):
    _fields_ = [("n_sampled", C.c_int64), ("n_records", C.c_int64), ("n_keys", C.c_int64),
                ("pairs_evaluated", C.c_int64), ("n_tiles", C.c_int64), ("tile_px_max", C.c_int64),
                ("cap_records", C.c_int64), ("cap_keys", C.c_int64)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError("libgsvr.so is not built (run __graft_entry__.build() or "
                          "python paper_2512_11624_b300/csrc/build.py); there is no fallback")
    lib = C.CDLL(LIB_PATH)
    vp, i32, i64, u64 = C.c_void_p, C.c_int32, C.c_int64, C.c_uint64
    sig = {
        "gsvr_abi_version": ([], i32),
        "gsvr_last_error": ([vp], C.c_char_p),
        "gsvr_create": ([C.POINTER(vp), C.c_int, vp, C.POINTER(Config)], C.c_int),
        "gsvr_destroy": ([vp], C.c_int),
        "gsvr_set_stacks": ([vp, i32, C.POINTER(StackDesc)], C.c_int),
        "gsvr_set_observations": ([vp, vp, vp, i32], C.c_int),
        "gsvr_set_gaussians": ([vp, i64, vp, i32], C.c_int),
        "gsvr_set_poses": ([vp, vp, i32], C.c_int),
        "gsvr_set_frozen": ([vp, vp], C.c_int),
        "gsvr_set_pixel_sample": ([vp, vp, i64, i32], C.c_int),
        "gsvr_sample_pixels": ([vp, i64, u64], C.c_int),
        "gsvr_forward": ([vp], C.c_int),
        "gsvr_backward": ([vp], C.c_int),
        "gsvr_adam_step": ([vp, C.POINTER(AdamCfg), i64], C.c_int),
        "gsvr_step_host": ([vp, vp, vp, i64, vp, vp], C.c_int),
        "gsvr_get_sample": ([vp, vp, i64, C.POINTER(i64)], C.c_int),
        "gsvr_get_views": ([vp, C.POINTER(Views)], C.c_int),
        "gsvr_get_stats": ([vp, C.POINTER(Stats)], C.c_int),
        "gsvr_sync_status": ([vp], C.c_int),
        "gsvr_timing_reset": ([vp], C.c_int),
        "gsvr_get_kernel_times": ([vp, C.POINTER(KernelTimes)], C.c_int),
        "gsvr_count_pairs": ([vp, C.POINTER(i64), C.POINTER(i64)], C.c_int),
        "gsvr_alu_peaks": ([C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_double)],
                           C.c_int),
        "gsvr_set_subjects": ([vp, i32, vp, vp], C.c_int),
        "gsvr_sample_pixels_subjects": ([vp, i64, u64], C.c_int),
        "gsvr_get_subject_losses": ([vp, vp, i32], C.c_int),
        "gsvr_set_subject_active": ([vp, vp], C.c_int),
        "gsvr_graph_capture": ([vp, i64, C.POINTER(AdamCfg)], C.c_int),
        "gsvr_graph_launch": ([vp, i32], C.c_int),
        "gsvr_set_step": ([vp, i64], C.c_int),
        "gsvr_set_tiling": ([vp, C.POINTER(Tiling)], C.c_int),
        "gsvr_set_topk": ([vp, C.c_int32, C.c_float, C.c_int32], C.c_int),
        "gsvr_set_objective": ([vp, C.c_int32, C.c_float, C.c_float], C.c_int),
        "gsvr_set_slice_weights": ([vp, C.c_int32, C.c_float, C.c_float], C.c_int),
        "gsvr_init_means": ([vp, vp, i64, C.c_float, u64, vp, vp, C.POINTER(i64)], C.c_int),
        "gsvr_slice_weight_views": ([vp, C.POINTER(vp), C.POINTER(vp), C.POINTER(i32)], C.c_int),
        "gsvr_get_topk_neighbors": ([vp, vp, vp, vp, i64, C.POINTER(i64)], C.c_int),
        "gsvr_reserve": ([vp, i64, i64], C.c_int),
        "gsvr_get_tiling": ([vp, C.POINTER(Tiling)], C.c_int),
        "gsvr_tune_space_default": ([C.POINTER(Tiling), i32, C.POINTER(i32)], C.c_int),
        "gsvr_autotune": ([vp, C.POINTER(Tiling), i32, i64, i32, C.POINTER(i32)], C.c_int),
        "gsvr_forward_noalloc": ([C.c_int, vp, i32, C.POINTER(StackDesc), i64, vp, vp, vp, i64, C.c_float, i32, vp,
                                  vp, C.c_char_p, i32], C.c_int),
        "gsvr_volume_metrics": ([C.c_int, vp, i64, i64, i64, vp, vp, vp, C.c_double, C.POINTER(C.c_double), vp,
                                 C.c_char_p, i32], C.c_int),
        "gsvr_fp64_peak": ([C.c_int, C.POINTER(C.c_double)], C.c_int),
        "gsvr_ffma2_peak": ([C.c_int, C.POINTER(C.c_double)], C.c_int),
        "gsvr_densify_accumulate": ([vp], C.c_int),
        "gsvr_densify_stats": ([vp, vp, C.POINTER(i32), i32], C.c_int),
        "gsvr_densify": ([vp, C.POINTER(DensifyCfg), C.POINTER(i64)], C.c_int),
        "gsvr_save": ([vp, C.c_char_p], C.c_int),
        "gsvr_test_wait_timeout": ([vp, i32, i64], C.c_int),
        "gsvr_set_sample_total": ([vp, i64], C.c_int),
        "gsvr_load": ([vp, C.c_char_p], C.c_int),
        "gsvr_checkpoint_info": ([C.c_char_p, C.POINTER(CheckpointHeader), C.c_char_p, i32], C.c_int),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    return lib


lib = _load()


def _check(ctx, status):
    if status != GSVR_OK:
        raise GsvrError(status, gsvr_last_error(ctx))
    return status


def _ptr(a):
    """(pointer, mem kind, keep-alive) of a numpy array or a torch tensor."""
    if a is None:
        return None, GSVR_MEM_HOST, None
    if isinstance(a, np.ndarray):
        a = np.ascontiguousarray(a)
        return a.ctypes.data, GSVR_MEM_HOST, a
    import torch
    if isinstance(a, torch.Tensor):
        a = a.contiguous()
        return a.data_ptr(), (GSVR_MEM_DEVICE if a.is_cuda else GSVR_MEM_HOST), a
    raise TypeError("expected a numpy array or a torch tensor")


def _typed(a, np_dtype, torch_dtype_name):
    if isinstance(a, np.ndarray):
        return np.ascontiguousarray(a, dtype=np_dtype)
    import torch
    dt = getattr(torch, torch_dtype_name)
    return a.to(dt).contiguous() if a.dtype != dt else a.contiguous()


# ------------------------------------------------------------------ C ABI names
def gsvr_abi_version():
    return int(lib.gsvr_abi_version())


def gsvr_last_error(ctx=None):
    s = lib.gsvr_last_error(ctx)
    return s.decode() if s else ""


def gsvr_create(device=0, stream=None, cutoff_rel=1e-7, tile_h=16, tile_w=16, norm_mode=GSVR_NORM_EXACT,
                fixed_capacity=0, cap_records=0, cap_keys=0, seed=0, timing=0):
    cfg = Config(cutoff_rel, tile_h, tile_w, norm_mode, fixed_capacity, timing, cap_records, cap_keys, seed)
    out = C.c_void_p()
    if stream is None:
        import torch
        stream = torch.cuda.current_stream(device).cuda_stream
    _check(None, lib.gsvr_create(C.byref(out), int(device), C.c_void_p(int(stream)), C.byref(cfg)))
    return out


def gsvr_destroy(ctx):
    return _check(ctx, lib.gsvr_destroy(ctx))


def stack_descs(stacks):
    arr = (StackDesc * len(stacks))()
    for k, s in enumerate(stacks):
        d = arr[k]
        d.n_slices, d.H, d.W = int(s["n_slices"]), int(s["H"]), int(s["W"])
        d.dx, d.dy, d.thickness = float(s["dx"]), float(s["dy"]), float(s["thickness"])
        R = np.asarray(s["R"], np.float64).reshape(9)
        for e in range(9):
            d.R[e] = float(R[e])
        for e in range(3):
            d.origin[e] = float(s["origin"][e])
            d.fwhm[e] = float(s["fwhm"][e])
    return arr


def gsvr_set_stacks(ctx, stacks):
    arr = stack_descs(stacks)
    return _check(ctx, lib.gsvr_set_stacks(ctx, len(stacks), arr))


def gsvr_set_observations(ctx, I, mask=None):
    I = _typed(I, np.float32, "float32")
    pI, mem, kI = _ptr(I)
    pm = None
    if mask is not None:
        mask = _typed(mask, np.uint8, "uint8")
        pm, mem_m, km = _ptr(mask)
        if mem_m != mem:
            raise ValueError("I and mask must live in the same memory")
    return _check(ctx, lib.gsvr_set_observations(ctx, pI, pm, mem))


def gsvr_set_gaussians(ctx, N, theta_g):
    t = _typed(theta_g, np.float32, "float32")
    p, mem, k = _ptr(t)
    return _check(ctx, lib.gsvr_set_gaussians(ctx, int(N), p, mem))


def gsvr_set_poses(ctx, pose):
    t = _typed(pose, np.float32, "float32")
    p, mem, k = _ptr(t)
    return _check(ctx, lib.gsvr_set_poses(ctx, p, mem))


def gsvr_set_frozen(ctx, frozen=None):
    if frozen is None:
        return _check(ctx, lib.gsvr_set_frozen(ctx, None))
    f = np.ascontiguousarray(frozen, dtype=np.uint8)
    return _check(ctx, lib.gsvr_set_frozen(ctx, f.ctypes.data))


def gsvr_set_pixel_sample(ctx, idx=None):
    if idx is None:
        return _check(ctx, lib.gsvr_set_pixel_sample(ctx, None, -1, GSVR_MEM_HOST))
    t = _typed(idx, np.int32, "int32")
    p, mem, k = _ptr(t)
    n = int(t.shape[0]) if hasattr(t, "shape") else len(t)
    return _check(ctx, lib.gsvr_set_pixel_sample(ctx, p, n, mem))


def gsvr_sample_pixels(ctx, n, step):
    return _check(ctx, lib.gsvr_sample_pixels(ctx, int(n), C.c_uint64(int(step))))


def gsvr_forward(ctx):
    return _check(ctx, lib.gsvr_forward(ctx))


def gsvr_backward(ctx):
    return _check(ctx, lib.gsvr_backward(ctx))


PAPER_LR = dict(lr_mu=2.5e-2, lr_ls=2.5e-2, lr_q=1e-2, lr_c=1e-2, lr_rot=2.5e-3, lr_trans=1e-1)


def adam_cfg(lr=None, beta1=0.9, beta2=0.999, eps=1e-8, step_every=0, gamma=1.0):
    lr = dict(PAPER_LR, **(lr or {}))
    return AdamCfg(lr["lr_mu"], lr["lr_ls"], lr["lr_q"], lr["lr_c"], lr["lr_rot"], lr["lr_trans"], beta1, beta2, eps,
                   int(step_every or 0), float(gamma))


def gsvr_adam_step(ctx, step, lr=None, beta1=0.9, beta2=0.999, eps=1e-8, step_every=0, gamma=1.0):
    cfg = adam_cfg(lr, beta1, beta2, eps, step_every, gamma)
    return _check(ctx, lib.gsvr_adam_step(ctx, C.byref(cfg), int(step)))


def gsvr_set_subject_active(ctx, active=None):
    """Retire (0) or return (1) subjects of the batched sampler; None = all active."""
    if active is None:
        return _check(ctx, lib.gsvr_set_subject_active(ctx, None))
    a = np.ascontiguousarray(np.asarray(active) != 0, dtype=np.uint8)
    return _check(ctx, lib.gsvr_set_subject_active(ctx, a.ctypes.data))


def gsvr_set_subjects(ctx, stack_subject, gauss_count):
    ss = np.ascontiguousarray(stack_subject, dtype=np.int32)
    gc = np.ascontiguousarray(gauss_count, dtype=np.int64)
    return _check(ctx, lib.gsvr_set_subjects(ctx, int(gc.size), ss.ctypes.data, gc.ctypes.data))


def gsvr_sample_pixels_subjects(ctx, n_per_subject, step):
    return _check(ctx, lib.gsvr_sample_pixels_subjects(ctx, int(n_per_subject), C.c_uint64(int(step))))


def gsvr_get_subject_losses(ctx, n):
    out = np.zeros(int(n), np.float64)
    _check(ctx, lib.gsvr_get_subject_losses(ctx, out.ctypes.data, int(n)))
    return out


def gsvr_graph_capture(ctx, n_per_subject, lr=None, beta1=0.9, beta2=0.999, eps=1e-8, step_every=0, gamma=1.0):
    cfg = adam_cfg(lr, beta1, beta2, eps, step_every, gamma)
    return _check(ctx, lib.gsvr_graph_capture(ctx, int(n_per_subject), C.byref(cfg)))


def gsvr_graph_launch(ctx, iterations=1):
    return _check(ctx, lib.gsvr_graph_launch(ctx, int(iterations)))


def gsvr_set_step(ctx, step):
    return _check(ctx, lib.gsvr_set_step(ctx, int(step)))


def tiling(tile_h=16, tile_w=16, fwd_px_per_thread=0, fwd_blocks_per_sm=0, bwd_blocks_per_sm=0, queue_order=0):
    return Tiling(tile_h, tile_w, fwd_px_per_thread, fwd_blocks_per_sm, bwd_blocks_per_sm, queue_order, 0.0)


def gsvr_set_tiling(ctx, t):
    if isinstance(t, dict):
        t = tiling(**{k: v for k, v in t.items() if k != "ms"})
    return _check(ctx, lib.gsvr_set_tiling(ctx, C.byref(t)))


def gsvr_set_topk(ctx, K, delta=1e-8, refresh_every=1):
    """Normalised top-K forward (K >= 1) or the plain sum (K = 0)."""
    return _check(ctx, lib.gsvr_set_topk(ctx, int(K), float(delta), int(refresh_every)))


def gsvr_set_objective(ctx, loss_kind=0, lambda_reg=0.0, s_target=1.6):
    """Data term (0 MSE, 1 L1) and scale regulariser of the loss."""
    return _check(ctx, lib.gsvr_set_objective(ctx, int(loss_kind), float(lambda_reg), float(s_target)))


def gsvr_init_means(ctx, n, lambda_init=0.0, seed=0, pose=None):
    """Content-adaptive means: (mu (3, n) float32 CUDA tensor, drawn pixels (n,) int32 CUDA tensor, total weight)."""
    import torch
    m = max(int(n), 0)  # the library checks n itself
    mu = torch.empty((3, m), dtype=torch.float32, device="cuda")
    pix = torch.empty(m, dtype=torch.int32, device="cuda")
    tot = C.c_int64(0)
    pp = None
    if pose is not None:
        pose = np.ascontiguousarray(pose, np.float32)
        pp = pose.ctypes.data
    _check(ctx, lib.gsvr_init_means(ctx, pp, int(n), float(lambda_init), C.c_uint64(int(seed)),
                                    mu.data_ptr() if m else None, pix.data_ptr() if m else None, C.byref(tot)))
    return mu, pix, int(tot.value)


def gsvr_set_slice_weights(ctx, enable=1, lr_log_sigma=1e-3, lr_log_omega=1e-2):
    """Per-slice intensity scale and aleatoric weight (log sigma_i, log omega_i)."""
    return _check(ctx, lib.gsvr_set_slice_weights(ctx, int(enable), float(lr_log_sigma), float(lr_log_omega)))


def gsvr_slice_weight_views(ctx):
    """(params, grads): zero-copy float32 CUDA tensors of 2 M entries each."""
    p, g, m = C.c_void_p(), C.c_void_p(), C.c_int32()
    _check(ctx, lib.gsvr_slice_weight_views(ctx, C.byref(p), C.byref(g), C.byref(m)))
    return device_view(p.value, 2 * m.value), device_view(g.value, 2 * m.value)


def gsvr_get_topk_neighbors(ctx, K):
    """(pix (n,), nbr (n, K), cnt (n,)) of the last top-K forward, in evaluation order."""
    n = C.c_int64(0)
    _check(ctx, lib.gsvr_get_topk_neighbors(ctx, None, None, None, 0, C.byref(n)))
    pix = np.zeros(n.value, np.int32)
    nbr = np.zeros((n.value, int(K)), np.int32)
    cnt = np.zeros(n.value, np.int32)
    _check(ctx, lib.gsvr_get_topk_neighbors(ctx, pix.ctypes.data, nbr.ctypes.data, cnt.ctypes.data, n.value,
                                            C.byref(n)))
    return pix, nbr, cnt


def gsvr_get_tiling(ctx):
    t = Tiling()
    _check(ctx, lib.gsvr_get_tiling(ctx, C.byref(t)))
    return t


def gsvr_tune_space_default():
    n = C.c_int32(0)
    _check(None, lib.gsvr_tune_space_default(None, 0, C.byref(n)))
    arr = (Tiling * n.value)()
    _check(None, lib.gsvr_tune_space_default(arr, n.value, C.byref(n)))
    return list(arr)


def gsvr_autotune(ctx, candidates=None, n_per_subject=0, iterations=5):
    """Time each launch shape (list of Tiling; default: the library's space) and
    apply the fastest.  Returns (best index, candidates with .ms filled)."""
    cands = list(candidates) if candidates is not None else gsvr_tune_space_default()
    arr = (Tiling * len(cands))(*cands)
    best = C.c_int32(-1)
    _check(ctx, lib.gsvr_autotune(ctx, arr, len(cands), int(n_per_subject), int(iterations), C.byref(best)))
    return best.value, list(arr)


def gsvr_reserve(ctx, cap_records, cap_keys):
    return _check(ctx, lib.gsvr_reserve(ctx, int(cap_records), int(cap_keys)))


def gsvr_step_host(ctx, theta, idx, grad_out=None, loss_out=None):
    """theta, idx, grad_out, loss_out: host arrays (numpy or pinned CPU tensors)."""
    pt, mt, kt = _ptr(theta)
    if idx is None:
        pi, n, ki = None, -1, None
    else:
        pi, mi, ki = _ptr(idx)
        n = int(idx.shape[0])
    pg, _, kg = _ptr(grad_out)
    pl, _, kl = _ptr(loss_out)
    return _check(ctx, lib.gsvr_step_host(ctx, pt, pi, n, pg, pl))


def gsvr_get_sample(ctx):
    n = C.c_int64()
    _check(ctx, lib.gsvr_get_sample(ctx, None, 0, C.byref(n)))
    out = np.zeros(max(int(n.value), 1), np.int32)
    _check(ctx, lib.gsvr_get_sample(ctx, out.ctypes.data, out.size, C.byref(n)))
    return out[:int(n.value)]


def gsvr_get_views(ctx):
    v = Views()
    _check(ctx, lib.gsvr_get_views(ctx, C.byref(v)))
    return v


def gsvr_get_stats(ctx):
    s = Stats()
    _check(ctx, lib.gsvr_get_stats(ctx, C.byref(s)))
    return {f: int(getattr(s, f)) for f, _ in Stats._fields_}


def gsvr_sync_status(ctx):
    return _check(ctx, lib.gsvr_sync_status(ctx))


def gsvr_timing_reset(ctx):
    return _check(ctx, lib.gsvr_timing_reset(ctx))


def gsvr_get_kernel_times(ctx):
    t = KernelTimes()
    _check(ctx, lib.gsvr_get_kernel_times(ctx, C.byref(t)))
    return {"ms": {STAGES[k]: float(t.ms[k]) for k in range(7)},
            "calls": {STAGES[k]: int(t.calls[k]) for k in range(7)},
            "pairs_evaluated": int(t.pairs_evaluated), "kernel_launches": int(t.kernel_launches),
            "bwd_pairs_evaluated": int(t.bwd_pairs_evaluated)}


def gsvr_count_pairs(ctx):
    u, e = C.c_int64(), C.c_int64()
    _check(ctx, lib.gsvr_count_pairs(ctx, C.byref(u), C.byref(e)))
    return int(u.value), int(e.value)


def gsvr_alu_peaks(device=0):
    """(FFMA instructions/s, ex2.approx instructions/s, SM count) measured on `device`."""
    f, e, n = C.c_double(), C.c_double(), C.c_double()
    _check(None, lib.gsvr_alu_peaks(int(device), C.byref(f), C.byref(e), C.byref(n)))
    return f.value, e.value, int(n.value)


def gsvr_densify_accumulate(ctx):
    """Add the last backward's ||dL/dmu_j|| and dL/dmu_j to the densification statistics."""
    return _check(ctx, lib.gsvr_densify_accumulate(ctx))


def gsvr_densify_stats(ctx, N, acc=None, count=None):
    """Without `acc`: read the statistics, (acc (N, 4) float32, pass count).
    With `acc` ((N, 4) float32) and `count`: write them."""
    if acc is None:
        a = np.zeros((int(N), 4), np.float32)
        c = C.c_int32(0)
        _check(ctx, lib.gsvr_densify_stats(ctx, a.ctypes.data if N else None, C.byref(c), 0))
        return a, int(c.value)
    a = np.ascontiguousarray(acc, np.float32).reshape(int(N), 4)
    c = C.c_int32(int(count))
    _check(ctx, lib.gsvr_densify_stats(ctx, a.ctypes.data if N else None, C.byref(c), 1))
    return a, int(count)


def gsvr_densify(ctx, grad_threshold, log_scale_threshold, prune_amplitude=0.0, split_factor=1.6,
                 clone_offset=0.5, mass_preserving=1, max_gaussians=0):
    """Split / clone / prune; returns (new N, split, cloned, pruned)."""
    cfg = DensifyCfg(float(grad_threshold), float(log_scale_threshold), float(prune_amplitude), float(split_factor),
                     float(clone_offset), int(mass_preserving), int(max_gaussians))
    out = (C.c_int64 * 4)()
    _check(ctx, lib.gsvr_densify(ctx, C.byref(cfg), out))
    return tuple(int(x) for x in out)


def gsvr_ffma2_peak(device=0):
    """Packed float32 FMA (f32x2) instructions/s measured on `device`."""
    d = C.c_double()
    _check(None, lib.gsvr_ffma2_peak(int(device), C.byref(d)))
    return d.value


def gsvr_fp64_peak(device=0):
    """float64 DFMA instructions/s measured on `device`."""
    d = C.c_double()
    _check(None, lib.gsvr_fp64_peak(int(device), C.byref(d)))
    return d.value


def gsvr_volume_metrics(X, Y, mask=None, data_range=1.0, ssim_map=None, stream=None):
    """(PSNR, SSIM, NCC) of the float32 CUDA volume X (D, H, W) against Y over
    `mask` (uint8 CUDA tensor of the same shape, or None for every voxel);
    `ssim_map`, a float64 CUDA tensor of the same shape, receives the SSIM map.
    Synchronises the stream."""
    import torch
    if X.dim() != 3 or tuple(Y.shape) != tuple(X.shape):
        raise ValueError("X and Y must be volumes (D, H, W) of one shape")
    for t, dt in ((X, torch.float32), (Y, torch.float32)):
        if not t.is_cuda or t.dtype != dt:
            raise ValueError("X and Y must be float32 CUDA tensors")
    X, Y = X.contiguous(), Y.contiguous()
    if mask is not None:
        if tuple(mask.shape) != tuple(X.shape) or mask.dtype != torch.uint8 or not mask.is_cuda:
            raise ValueError("mask must be a uint8 CUDA tensor shaped like X")
        mask = mask.contiguous()
    if ssim_map is not None and (tuple(ssim_map.shape) != tuple(X.shape) or ssim_map.dtype != torch.float64 or
                                 not ssim_map.is_contiguous()):
        raise ValueError("ssim_map must be a contiguous float64 CUDA tensor shaped like X")
    device = X.device.index
    if stream is None:
        stream = torch.cuda.current_stream(device).cuda_stream
    D, H, W = X.shape
    out = (C.c_double * 3)()
    buf = C.create_string_buffer(256)
    st = lib.gsvr_volume_metrics(int(device), C.c_void_p(int(stream)), int(D), int(H), int(W), X.data_ptr(),
                                 Y.data_ptr(), mask.data_ptr() if mask is not None else None, float(data_range),
                                 out, ssim_map.data_ptr() if ssim_map is not None else None, buf, 256)
    if st != GSVR_OK:
        raise GsvrError(st, buf.value.decode())
    return out[0], out[1], out[2]


def gsvr_forward_noalloc(stacks, N, theta, I, idx, pred, loss, device=0, stream=None, cutoff_rel=1e-7,
                         norm_mode=GSVR_NORM_EXACT):
    """Context-free forward that allocates no device memory (for callers that
    cannot call cudaMalloc); all arrays are CUDA tensors: theta (11N + 6M float32),
    I and pred (one float32 per global pixel), idx (int32 sampled pixels, or None
    for every pixel), loss (one float64).  Synchronises the stream."""
    import torch
    if stream is None:
        stream = torch.cuda.current_stream(device).cuda_stream
    arr = stack_descs(stacks)
    buf = C.create_string_buffer(256)
    pi = idx.data_ptr() if idx is not None else None
    n = int(idx.numel()) if idx is not None else -1
    st = lib.gsvr_forward_noalloc(int(device), C.c_void_p(int(stream)), len(stacks), arr, int(N),
                                  theta.data_ptr() if N > 0 else None, I.data_ptr(), pi, n, float(cutoff_rel),
                                  int(norm_mode), pred.data_ptr(), loss.data_ptr(), buf, 256)
    if st != GSVR_OK:
        raise GsvrError(st, buf.value.decode())
    return st


def gsvr_set_sample_total(ctx, n_total):
    """Pixel weight 1 / n_total (the global sample size of a sharded reconstruction); 0 = own sample size."""
    return _check(ctx, lib.gsvr_set_sample_total(ctx, int(n_total)))


def gsvr_test_wait_timeout(ctx, n_forwards=1, limit_ns=2_000_000):
    """Test hook: the next n forwards run out one bounded device wait (see gsvr.h)."""
    return _check(ctx, lib.gsvr_test_wait_timeout(ctx, int(n_forwards), int(limit_ns)))


def gsvr_save(ctx, path):
    """Write the context's optimisation state to `path` (see gsvr.h)."""
    return _check(ctx, lib.gsvr_save(ctx, os.fsencode(path)))


def gsvr_load(ctx, path):
    """Restore a state written by gsvr_save (stacks and observations set first)."""
    return _check(ctx, lib.gsvr_load(ctx, os.fsencode(path)))


def gsvr_checkpoint_info(path):
    """Check a checkpoint file without a context or GPU; returns its header as a dict."""
    h = CheckpointHeader()
    buf = C.create_string_buffer(256)
    st = lib.gsvr_checkpoint_info(os.fsencode(path), C.byref(h), buf, 256)
    if st != GSVR_OK:
        raise GsvrError(st, buf.value.decode())
    return {k: getattr(h, k) for k, _ in CheckpointHeader._fields_ if k != "reserved"}


# --------------------------------------------------------------- torch views
class _CudaArray:
    def __init__(self, ptr, shape, typestr):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr, "data": (int(ptr), False),
                                         "version": 2, "strides": None}


def device_view(ptr, n, dtype="float32", device=0):
    """Zero-copy torch view of a context-owned device buffer."""
    import torch
    ts = {"float32": "<f4", "float64": "<f8"}[dtype]
    return torch.as_tensor(_CudaArray(ptr, (int(n),), ts), device="cuda:%d" % device)


class Context:
    """Owning wrapper: one gsvr context set up from a case dictionary
    (``stacks``, ``N``, ``theta``, ``I``, ``mask``) as made by the input generators.

    ``theta``, ``grad``, ``pred``, ``rbar``, ``loss_t`` are zero-copy views of
    context-owned buffers, written on the context's stream: with a stream of
    its own, order the reading stream after it (``wait_stream``) or call
    ``gsvr_sync_status`` first.  Changing the Gaussian count reallocates the
    parameter buffers: use ``set_gaussians``, which refreshes the views."""

    def __init__(self, case, device=0, stream=None, **cfg):
        self.device = device
        self.ctx = gsvr_create(device, stream, **cfg)
        self.N = int(case["N"])
        self.stacks = case["stacks"]
        gsvr_set_stacks(self.ctx, self.stacks)
        gsvr_set_observations(self.ctx, np.asarray(case["I"], np.float32), np.asarray(case["mask"], np.uint8))
        th = np.asarray(case["theta"], np.float32)
        gsvr_set_gaussians(self.ctx, self.N, th[:11 * self.N])
        self.M = int(sum(s["n_slices"] for s in self.stacks))
        gsvr_set_poses(self.ctx, th[11 * self.N:11 * self.N + 6 * self.M])
        self.refresh_views()

    def refresh_views(self):
        v = gsvr_get_views(self.ctx)
        self.n_params = int(v.n_params)
        self.n_pixels = int(v.n_pixels)
        self.theta = device_view(v.theta, v.n_params, device=self.device)
        self.grad = device_view(v.grad, v.n_params, device=self.device)
        self.adam_m = device_view(v.adam_m, v.n_params, device=self.device)
        self.adam_v = device_view(v.adam_v, v.n_params, device=self.device)
        self.pred = device_view(v.pred, v.n_pixels, device=self.device)
        self.rbar = device_view(v.rbar, v.n_pixels, device=self.device)
        self.loss_t = device_view(v.loss, 1, "float64", device=self.device)

    def set_gaussians(self, theta_g, N):
        """Replace the Gaussians (11 N floats, host or device); poses are kept."""
        gsvr_set_gaussians(self.ctx, int(N), theta_g)
        self.N = int(N)
        self.refresh_views()

    def save(self, path):
        """gsvr_save: the optimisation state to a checkpoint file."""
        gsvr_save(self.ctx, path)

    def load(self, path):
        """gsvr_load, then refresh N and the views (the Gaussian count may change)."""
        gsvr_load(self.ctx, path)
        self.N = int(gsvr_checkpoint_info(path)["n_gaussians"])
        self.refresh_views()

    def densify(self, grad_threshold, log_scale_threshold, **kw):
        """gsvr_densify, then refresh N and the views; returns (N, split, cloned, pruned)."""
        out = gsvr_densify(self.ctx, grad_threshold, log_scale_threshold, **kw)
        self.N = out[0]
        self.refresh_views()
        return out

    def forward(self):
        gsvr_forward(self.ctx)

    def backward(self):
        gsvr_backward(self.ctx)

    def loss(self):
        gsvr_sync_status(self.ctx)
        return float(self.loss_t.item())

    def stats(self):
        return gsvr_get_stats(self.ctx)

    def sample_index(self):
        """Global pixel indices of the current sample, in the library's order (device int64)."""
        import torch
        return torch.from_numpy(gsvr_get_sample(self.ctx).astype("int64")).to(self.theta.device)

    def close(self):
        if self.ctx is not None:
            gsvr_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
