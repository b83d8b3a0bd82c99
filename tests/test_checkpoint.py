"""Checkpoint / resume (gsvr_save, gsvr_load, gsvr_checkpoint_info).

CPU: a file written here from the format that include/gsvr.h documents is
accepted by gsvr_checkpoint_info with the header it holds; a missing file, a
bad magic, another version, a flipped byte (hash), a truncated file, an
unknown or repeated section and a missing required section are each rejected.

GPU: a context is run for a few Adam steps with a non-default launch shape,
the paper's L1 objective with the scale regulariser, per-slice weights and a
frozen slice, then saved; a fresh context (default launch shape) holding the
same stacks and observations loads the file; the next step (same pixel sample)
gives bitwise the same predictions, loss, Gaussian gradient, Adam update of
the Gaussians and per-slice weights on both (slice-pose gradients are float
atomics whose order depends on thread timing: equal to rounding)."""
import os
import struct

import numpy as np
import pytest

from paper_2512_11624_b300 import inputs


def fnv1a(b):
    h = 1469598103934665603
    for x in b:
        h = ((h ^ x) * 1099511628211) & 0xFFFFFFFFFFFFFFFF
    return h


def stack_desc_bytes(s):
    R = np.asarray(s["R"], np.float32).reshape(9)
    return struct.pack("<4i3f9f3f3f", int(s["n_slices"]), int(s["H"]), int(s["W"]), 0, float(s["dx"]),
                       float(s["dy"]), float(s["thickness"]), *R, *np.asarray(s["origin"], np.float32),
                       *np.asarray(s["fwhm"], np.float32))


def section(tag, payload):
    return struct.pack("<IIQ", tag, 0, len(payload)) + payload


def make_file(stacks, N, step, version=1, sections=None, extra=b""):
    M = inputs.n_slices_total(stacks)
    P = inputs.n_pixels_total(stacks)
    np_ = 11 * N + 6 * M
    if sections is None:
        cfg = struct.pack("<fiQ6i", 1e-7, 0, 5, 16, 16, 0, 0, 0, 0)
        geo = struct.pack("<iiq", len(stacks), M, P) + b"".join(stack_desc_bytes(s) for s in stacks)
        par = struct.pack("<q", N) + np.arange(3 * np_, dtype=np.float32).tobytes()
        sections = [section(1, cfg), section(2, geo), section(3, par), section(4, struct.pack("<Q", step))]
    body = b"GSVRCKPT" + struct.pack("<II", version, len(sections)) + b"".join(sections) + extra
    return body + struct.pack("<Q", fnv1a(body))


def test_checkpoint_info_accepts_the_documented_format(tmp_path):
    from paper_2512_11624_b300 import gsvr
    case = inputs.tiny(0)
    path = tmp_path / "ok.ckpt"
    path.write_bytes(make_file(case["stacks"], 7, 123))
    h = gsvr.gsvr_checkpoint_info(str(path))
    assert h == {"version": 1, "n_stacks": 1, "n_slices": 8, "n_pixels": 8 * 32 * 32, "n_gaussians": 7, "step": 123}


def test_checkpoint_info_rejects_bad_files(tmp_path):
    from paper_2512_11624_b300 import gsvr
    st = inputs.tiny(0)["stacks"]
    good = make_file(st, 3, 1)
    cfg = struct.pack("<fiQ6i", 1e-7, 0, 5, 16, 16, 0, 0, 0, 0)
    M, P = 8, 8 * 32 * 32
    geo = struct.pack("<iiq", 1, M, P) + stack_desc_bytes(st[0])
    par = struct.pack("<q", 3) + np.zeros(3 * (33 + 48), np.float32).tobytes()
    stp = struct.pack("<Q", 1)
    bad = {
        "magic": b"GSVRCKPX" + good[8:],
        "version": make_file(st, 3, 1, version=2),
        "hash": good[:40] + bytes([good[40] ^ 1]) + good[41:],
        "truncated": good[:-9],
        "short": good[:12],
        "unknown section": make_file(st, 3, 1, sections=[section(1, cfg), section(2, geo), section(3, par),
                                                          section(4, stp), section(99, b"x")]),
        "repeated section": make_file(st, 3, 1, sections=[section(1, cfg), section(2, geo), section(3, par),
                                                           section(4, stp), section(4, stp)]),
        "missing step": make_file(st, 3, 1, sections=[section(1, cfg), section(2, geo), section(3, par)]),
        "parameter size": make_file(st, 3, 1, sections=[section(1, cfg), section(2, geo), section(3, par[:-4]),
                                                         section(4, stp)]),
        "trailing bytes": make_file(st, 3, 1, extra=b"\0"),
    }
    for name, data in bad.items():
        p = tmp_path / ("bad_%s.ckpt" % name.replace(" ", "_"))
        p.write_bytes(data)
        with pytest.raises(gsvr.GsvrError) as ei:
            gsvr.gsvr_checkpoint_info(str(p))
        assert ei.value.status == gsvr.GSVR_ERR_INVALID_ARG, name
    with pytest.raises(gsvr.GsvrError):
        gsvr.gsvr_checkpoint_info(str(tmp_path / "missing.ckpt"))


@pytest.mark.gpu
def test_resume_is_bitwise_identical(tmp_path):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2512_11624_b300 import gsvr
    case = inputs.random_case(8, 900, [(5, 40, 36), (4, 33, 41)], n_stacks=2, motion_deg=8.0, motion_mm=3.0)
    M = inputs.n_slices_total(case["stacks"])
    n_s = int(0.6 * inputs.n_pixels_total(case["stacks"]))
    lr = {"lr_mu": 2e-3, "lr_ls": 2e-3, "lr_q": 1e-3, "lr_c": 2e-3, "lr_rot": 1e-3, "lr_trans": 1e-2}

    def step(ctx, k):
        gsvr.gsvr_sample_pixels(ctx.ctx, n_s, k)
        ctx.forward()
        ctx.backward()
        sample = gsvr.gsvr_get_sample(ctx.ctx)  # pred is written at the sampled pixels only
        out = {"sample": sample, "pred": ctx.pred.cpu().numpy()[sample], "loss": ctx.loss(),
               "grad": ctx.grad.cpu().numpy().copy()}
        gsvr.gsvr_adam_step(ctx.ctx, k + 1, lr=lr, step_every=3, gamma=0.5)
        gsvr.gsvr_sync_status(ctx.ctx)
        out.update(theta=ctx.theta.cpu().numpy().copy(), m=ctx.adam_m.cpu().numpy().copy(),
                   v=ctx.adam_v.cpu().numpy().copy(), slw=gsvr.gsvr_slice_weight_views(ctx.ctx)[0].cpu().numpy().copy())
        return out

    a = gsvr.Context(case, seed=77)
    gsvr.gsvr_set_tiling(a.ctx, gsvr.tiling(8, 12, queue_order=1))
    gsvr.gsvr_set_objective(a.ctx, 1, 1e-4, 1.2)
    gsvr.gsvr_set_slice_weights(a.ctx, 1, 1e-3, 1e-2)
    gsvr.gsvr_set_frozen(a.ctx, np.array([1 if i == 2 else 0 for i in range(M)], np.uint8))
    gsvr.gsvr_set_step(a.ctx, 41)
    for k in range(4):
        step(a, k)
    path = str(tmp_path / "mid.ckpt")
    a.save(path)
    h = gsvr.gsvr_checkpoint_info(path)
    assert h["n_gaussians"] == case["N"] and h["n_slices"] == M and h["step"] == 41
    ref = step(a, 4)
    a.close()

    # a fresh context: same stacks and observations, default launch shape and objective,
    # other Gaussians (a different count) -- everything else comes from the file
    other = dict(case)
    other["N"] = 100
    other["theta"] = np.concatenate([case["theta"][:0], np.random.default_rng(0).uniform(0.1, 1, 1100),
                                     np.zeros(6 * M)]).astype(np.float32)
    b = gsvr.Context(other, seed=1)
    b.load(path)
    assert b.N == case["N"]
    got = step(b, 4)
    t = gsvr.gsvr_get_tiling(b.ctx)
    assert (t.tile_h, t.tile_w, t.queue_order) == (8, 12, 1)
    b.close()
    # forward, Gaussian gradient, Adam update of the Gaussians, per-slice weights: bitwise
    N = case["N"]
    for k in ("sample", "pred", "slw"):
        assert np.array_equal(got[k], ref[k]), k
    for k in ("grad", "theta", "m", "v"):
        assert np.array_equal(got[k][:11 * N], ref[k][:11 * N]), k
    assert got["loss"] == ref["loss"]
    # slice poses: their gradients are float atomics in a timing-dependent order (equal to rounding)
    gp, rp = got["grad"][11 * N:], ref["grad"][11 * N:]
    assert np.all(np.abs(gp - rp) <= 1e-5 * np.abs(rp).max() + 1e-30)
    assert np.allclose(got["theta"][11 * N:], ref["theta"][11 * N:], rtol=1e-6, atol=1e-6)
    # a checkpoint of other stacks is refused
    c = gsvr.Context(inputs.tiny(0))
    with pytest.raises(gsvr.GsvrError) as ei:
        c.load(path)
    assert ei.value.status == gsvr.GSVR_ERR_STATE
    c.close()
