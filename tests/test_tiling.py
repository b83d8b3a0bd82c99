"""Launch shapes (tile size, forward pixels per thread, persistent CTAs per SM,
work-queue order) change how the work is cut, never what is computed: every
shape against the FP64 oracle, re-tiling a live context (subjects, frozen
slices and parameters kept), rejection of invalid shapes, and the autotuner."""
import numpy as np
import pytest

from paper_2512_11624_b300 import inputs
from tests.gpu_util import CUTOFF, forward_ok, grad_ok, describe_grad

SHAPES = [dict(tile_h=16, tile_w=16), dict(tile_h=8, tile_w=8, fwd_px_per_thread=1),
          dict(tile_h=12, tile_w=12, queue_order=1), dict(tile_h=32, tile_w=8, fwd_blocks_per_sm=1, bwd_blocks_per_sm=1),
          dict(tile_h=8, tile_w=32, fwd_px_per_thread=4, queue_order=1), dict(tile_h=12, tile_w=16, fwd_px_per_thread=2),
          dict(tile_h=5, tile_w=7, fwd_px_per_thread=1, fwd_blocks_per_sm=3),
          dict(tile_h=12, tile_w=12, fwd_blocks_per_sm=-1, bwd_blocks_per_sm=-1, queue_order=1),
          dict(tile_h=8, tile_w=16, fwd_px_per_thread=8), dict(tile_h=6, tile_w=20, fwd_px_per_thread=8),
          # forward row bands: 4 (32 x 16), 6 (24 x 32, 96-thread CTAs), 8 (32 x 32) and 16 (32 x 32, 4 px)
          dict(tile_h=32, tile_w=16), dict(tile_h=24, tile_w=32), dict(tile_h=32, tile_w=32),
          dict(tile_h=32, tile_w=32, fwd_px_per_thread=4),
          # 16-pixel runs: a whole 16-wide row per thread; ragged 12-wide rows; banded at 32 x 32
          dict(tile_h=16, tile_w=16, fwd_px_per_thread=16), dict(tile_h=8, tile_w=12, fwd_px_per_thread=16),
          dict(tile_h=32, tile_w=32, fwd_px_per_thread=16)]


def test_default_space_is_valid_host_logic():
    """Host only: the built-in candidate space is non-empty and every shape in it
    satisfies the documented limits."""
    from paper_2512_11624_b300 import gsvr
    space = gsvr.gsvr_tune_space_default()
    assert len(space) >= 8
    for t in space:
        px = t.fwd_px_per_thread or (8 if t.tile_w > 16 else (16 if t.tile_w > 12 else (4 if t.tile_w == 12 else 2)))
        assert 4 <= t.tile_h <= 32 and 4 <= t.tile_w <= 32 and px in (1, 2, 4, 8, 16)
        assert t.tile_h * -(-t.tile_w // px) <= 256
        assert t.queue_order in (0, 1)


@pytest.fixture(scope="module")
def G():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2512_11624_b300 import gsvr
    return gsvr


def ref_of(oracle, case):
    pix = np.arange(inputs.n_pixels_total(case["stacks"]))
    return pix, oracle.forward_backward(case["stacks"], case["theta"].astype(np.float64), case["N"], pix,
                                        case["I"].astype(np.float64), 1.0 / len(pix), cutoff=CUTOFF)


@pytest.mark.gpu
def test_every_shape_matches_oracle_on_one_context(G, oracle):
    case = inputs.random_case(61, 250, [(3, 37, 29), (2, 20, 41)], n_stacks=2, motion_deg=10.0, motion_mm=3.0)
    pix, (p_ref, L_ref, g_ref, a_ref, t_pred, t_grad) = ref_of(oracle, case)
    M = inputs.n_slices_total(case["stacks"])
    ctx = G.Context(case)
    for shape in SHAPES:
        G.gsvr_set_tiling(ctx.ctx, shape)
        got = G.gsvr_get_tiling(ctx.ctx)
        assert (got.tile_h, got.tile_w, got.queue_order) == (shape["tile_h"], shape["tile_w"],
                                                             shape.get("queue_order", 0))
        ctx.forward()
        ctx.backward()
        G.gsvr_sync_status(ctx.ctx)
        assert ctx.stats()["n_sampled"] == len(pix)
        ok, worst = forward_ok(ctx.pred.cpu().numpy().astype(np.float64), p_ref, t_pred)
        assert ok.all(), (shape, worst)
        g = ctx.grad.cpu().numpy().astype(np.float64)
        gok, gworst, _ = grad_ok(g, g_ref, a_ref, t_grad)
        assert gok.all(), (shape, describe_grad(g, g_ref, a_ref, case["N"], M, t_grad))
    ctx.close()


@pytest.mark.gpu
def test_invalid_shapes_leave_context_unchanged(G):
    case = inputs.random_case(62, 30, [(2, 20, 20)])
    ctx = G.Context(case, tile_h=12, tile_w=12)
    before = G.gsvr_get_tiling(ctx.ctx).as_dict()
    for bad in [dict(tile_h=32, tile_w=32, fwd_px_per_thread=1), dict(tile_h=3, tile_w=16),
                dict(tile_h=16, tile_w=33), dict(tile_h=16, tile_w=16, fwd_px_per_thread=3),
                dict(tile_h=16, tile_w=16, queue_order=2), dict(tile_h=16, tile_w=16, bwd_blocks_per_sm=-2)]:
        with pytest.raises(G.GsvrError) as e:
            G.gsvr_set_tiling(ctx.ctx, bad)
        assert e.value.status == G.GSVR_ERR_INVALID_ARG
        assert G.gsvr_get_tiling(ctx.ctx).as_dict() == before
    ctx.close()


@pytest.mark.gpu
def test_retiling_keeps_subjects_frozen_slices_and_parameters(G):
    from tests.test_batched import three_subjects
    cases = three_subjects()
    b = inputs.concat_cases(cases)
    ctx = G.Context(b, tile_h=16, tile_w=16)
    G.gsvr_set_subjects(ctx.ctx, b["stack_subject"], b["gauss_count"])
    frozen = np.zeros(ctx.M, np.uint8)
    frozen[[0, 5]] = 1
    G.gsvr_set_frozen(ctx.ctx, frozen)
    ctx.forward()
    ctx.backward()
    l16 = G.gsvr_get_subject_losses(ctx.ctx, len(cases))
    th16 = ctx.theta.cpu().numpy().copy()
    G.gsvr_set_tiling(ctx.ctx, dict(tile_h=8, tile_w=8, queue_order=1))
    assert np.array_equal(ctx.theta.cpu().numpy(), th16)
    ctx.forward()
    ctx.backward()
    l8 = G.gsvr_get_subject_losses(ctx.ctx, len(cases))
    assert np.allclose(l8, l16, rtol=2e-5, atol=0)
    lr = dict(lr_mu=1e-2, lr_ls=1e-2, lr_q=1e-2, lr_c=1e-2, lr_rot=1e-2, lr_trans=1e-1)
    G.gsvr_adam_step(ctx.ctx, 1, lr=lr)
    th = ctx.theta.cpu().numpy()
    pose = th[11 * b["N"]:].reshape(-1, 6)
    assert np.array_equal(pose[[0, 5]], th16[11 * b["N"]:].reshape(-1, 6)[[0, 5]])  # frozen slices kept
    assert not np.array_equal(pose[1], th16[11 * b["N"]:].reshape(-1, 6)[1])
    ctx.close()


@pytest.mark.gpu
def test_autotune_times_candidates_and_applies_fastest(G, oracle):
    case = inputs.random_case(63, 300, [(3, 40, 40)], n_stacks=2, motion_deg=5.0)
    ctx = G.Context(case)
    cands = [G.tiling(16, 16), G.tiling(8, 8, 1), G.tiling(32, 32, 1), G.tiling(12, 12, 0, 0, 0, 1)]
    best, res = G.gsvr_autotune(ctx.ctx, cands, n_per_subject=1500, iterations=3)
    assert res[2].ms == -1.0  # invalid shape skipped
    valid = [0, 1, 3]
    assert all(res[k].ms > 0 for k in valid)
    assert best == min(valid, key=lambda k: res[k].ms)
    t = G.gsvr_get_tiling(ctx.ctx)
    assert (t.tile_h, t.tile_w, t.fwd_px_per_thread, t.queue_order) == (res[best].tile_h, res[best].tile_w,
                                                                       res[best].fwd_px_per_thread,
                                                                       res[best].queue_order)
    # the tuned context still computes the method's values
    G.gsvr_set_pixel_sample(ctx.ctx, np.arange(inputs.n_pixels_total(case["stacks"]), dtype=np.int32))
    ctx.forward()
    ctx.backward()
    pix, (p_ref, L_ref, g_ref, a_ref, t_pred, t_grad) = ref_of(oracle, case)
    ok, worst = forward_ok(ctx.pred.cpu().numpy().astype(np.float64), p_ref, t_pred)
    assert ok.all(), worst
    ctx.close()
