"""The pose network's tensor-core kernels (through the C ABI) against the FP64
oracle on the same bfloat16-rounded operands: conv forward, input gradient
and weight / bias gradient, layer by layer at ragged sizes (2e-3 relative plus
a float32-accumulation floor), then the whole network's loss and gradients,
the Adam step, and a short fit."""
import numpy as np
import pytest

from oracle import cnn as ocnn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def T():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2512_11624_b300 import cnn
    return torch, cnn


def bf(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).to(torch.bfloat16).cuda()


def close(got, ref, absref, rtol=2e-3, atol_rel=1e-5):
    err = np.abs(got - ref)
    lim = rtol * np.abs(ref) + atol_rel * absref + 1e-30
    return err <= lim, float((err / lim).max()) if err.size else 0.0


SHAPES = [(2, 9, 7, 8, 16), (3, 16, 16, 32, 64), (1, 33, 17, 16, 40), (2, 4, 4, 64, 128), (1, 8, 8, 256, 512)]


@pytest.mark.parametrize("B,H,W,Ci,Co", SHAPES)
def test_conv_forward(T, B, H, W, Ci, Co):
    torch, cnn = T
    rng = np.random.default_rng(B * 1000 + H * 10 + Ci)
    x = ocnn.bf16(rng.normal(size=(B, H, W, Ci)))
    w = ocnn.bf16(rng.normal(size=(Co, 3, 3, Ci)) / np.sqrt(9 * Ci))
    b = rng.normal(size=Co).astype(np.float32).astype(np.float64)
    for relu in (False, True):
        y, y32 = cnn.conv_forward(bf(torch, x), bf(torch, w), torch.from_numpy(b.astype(np.float32)).cuda(), relu=relu,
                                  want_f32=True)
        ref, absref = ocnn.conv_fwd(x, w, b, relu=False, want_abs=True)
        if relu:
            ref = np.maximum(ref, 0.0)
        got = y32.cpu().numpy().astype(np.float64)
        ok, worst = close(got, ref, absref)
        assert ok.all(), worst
        assert np.array_equal(y.float().cpu().numpy(), ocnn.bf16(got).astype(np.float32))
    cnn.sync_status()


def test_first_layer_direct(T):
    torch, cnn = T
    rng = np.random.default_rng(7)
    x = ocnn.bf16(rng.uniform(0, 2, size=(3, 21, 18, 1)))
    w = ocnn.bf16(rng.normal(size=(32, 3, 3, 1)) / 3)
    b = rng.normal(size=32).astype(np.float32).astype(np.float64) * 0.1
    y = cnn.conv_forward(bf(torch, x), bf(torch, w), torch.from_numpy(b.astype(np.float32)).cuda(), relu=True)
    ref, absref = ocnn.conv_fwd(x, w, b, relu=True, want_abs=True)
    got = y.float().cpu().numpy().astype(np.float64)
    # bf16 output: one rounding of a float32 sum within 2e-3 of the exact value
    ok, worst = close(got, ref, absref, rtol=2 ** -8 + 2e-6, atol_rel=1e-5)
    assert ok.all(), worst
    gy = ocnn.bf16(rng.normal(size=ref.shape))
    dw, db = cnn.conv_wgrad(bf(torch, gy), bf(torch, x))
    rdw, rdb, adw = ocnn.conv_wgrad(gy, x, want_abs=True)
    ok, worst = close(dw.cpu().numpy().astype(np.float64), rdw, adw)
    assert ok.all(), worst
    assert np.allclose(db.cpu().numpy(), rdb, rtol=2e-3, atol=1e-5 * np.abs(gy).sum(axis=(0, 1, 2)).max())


@pytest.mark.parametrize("B,H,W,Ci,Co", SHAPES)
def test_conv_dgrad(T, B, H, W, Ci, Co):
    torch, cnn = T
    rng = np.random.default_rng(B * 77 + W)
    OH, OW = (H + 1) // 2, (W + 1) // 2
    gy = ocnn.bf16(rng.normal(size=(B, OH, OW, Co)))
    w = ocnn.bf16(rng.normal(size=(Co, 3, 3, Ci)) / np.sqrt(9 * Ci))
    ref, absref = ocnn.conv_dgrad(gy, w, H, W, want_abs=True)
    dx, dx32 = cnn.conv_dgrad(bf(torch, gy), bf(torch, w), H, W)
    ok, worst = close(dx32.cpu().numpy().astype(np.float64), ref, absref)
    assert ok.all(), worst
    mask = ocnn.bf16(rng.normal(size=(B, H, W, Ci)))
    dxm, dxm32 = cnn.conv_dgrad(bf(torch, gy), bf(torch, w), H, W, mask=bf(torch, mask))
    gotm = dxm32.cpu().numpy()
    assert np.all(gotm[mask <= 0] == 0)
    assert np.array_equal(gotm[mask > 0], dx32.cpu().numpy()[mask > 0])
    assert np.array_equal(dxm.float().cpu().numpy(), ocnn.bf16(gotm).astype(np.float32))
    cnn.sync_status()


@pytest.mark.parametrize("B,H,W,Ci,Co", SHAPES)
def test_conv_wgrad(T, B, H, W, Ci, Co):
    torch, cnn = T
    rng = np.random.default_rng(B * 5 + H * 3 + Co)
    OH, OW = (H + 1) // 2, (W + 1) // 2
    gy = ocnn.bf16(rng.normal(size=(B, OH, OW, Co)))
    x = ocnn.bf16(rng.normal(size=(B, H, W, Ci)))
    rdw, rdb, adw = ocnn.conv_wgrad(gy, x, want_abs=True)
    dw, db = cnn.conv_wgrad(bf(torch, gy), bf(torch, x))
    ok, worst = close(dw.cpu().numpy().astype(np.float64), rdw, adw)
    assert ok.all(), worst
    adb = np.abs(gy).sum(axis=(0, 1, 2))
    ok, worst = close(db.cpu().numpy().astype(np.float64), rdb, adb)
    assert ok.all(), worst


@pytest.mark.parametrize("M,N,K", [(128, 128, 64), (300, 200, 72), (1000, 300, 520), (7, 129, 8), (4096, 512, 2304)])
def test_gemm_tensor_memory(T, M, N, K):
    """The tcgen05 GEMM (tensor-memory accumulators) with tensor-map operand
    copies (1) and with per-thread copies (2), and the mma.sync GEMM (0),
    against a float64 product of the same bfloat16 operands, at tile-aligned,
    ragged and one-row-short shapes.  Both accumulate in float32, so each
    element stays within 1e-5 of the exact value relative to sum_k |a b|
    (a float32 sum of at most 2304 terms)."""
    torch, cnn = T
    g = torch.Generator(device="cuda").manual_seed(M + N + K)
    A = torch.randn((M, K), device="cuda", generator=g).to(torch.bfloat16)
    B = torch.randn((N, K), device="cuda", generator=g).to(torch.bfloat16)
    ref = (A.double() @ B.double().T).cpu().numpy()
    absref = (A.double().abs() @ B.double().abs().T).cpu().numpy()
    for tm in (1, 2, 0):
        C, status = cnn.gemm(A, B, tensor_memory=tm)
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        ok, worst = close(C.cpu().numpy().astype(np.float64), ref, absref, rtol=1e-5, atol_rel=1e-5)
        assert ok.all(), (tm, worst)


def oracle_params(net):
    shapes = ocnn.param_shapes()
    return shapes, ocnn.unflatten(net.params.cpu().numpy().astype(np.float64), shapes)


def test_network_loss_and_gradients(T):
    """Whole network at batch 3: loss within 1e-3, every parameter tensor's
    gradient within 5e-2 relative L2 of the oracle's and at cosine >= 0.999.
    The network's gradient is a discontinuous function of its float32 sums:
    a pre-activation within float32 rounding of 0 passes the ReLU on one side
    and not on the other, and one such flip among the 12,288 conv5 outputs of
    this case moves every earlier layer's gradient by ~2e-2 (measured: all
    per-layer kernels agree with the oracle to <= 3e-7 relative L2 when fed the
    same inputs, see the layer tests above, while exactly one conv5 ReLU mask
    differs).  Later layers, upstream of the flip, agree to ~1e-3."""
    torch, cnn = T
    rng = np.random.default_rng(11)
    net = cnn.PoseNet(max_batch=4, seed=3)
    B = 3
    x = rng.uniform(0, 2, size=(B, 128, 128)).astype(np.float32)
    x[:, :20] = 0.0
    aux = rng.normal(size=(B, 25)).astype(np.float32)
    tgt = rng.normal(size=(B, 6)).astype(np.float32) * 0.1
    xt, at, tt = (torch.from_numpy(v).cuda() for v in (x, aux, tgt))
    out = net.forward(xt, at).cpu().numpy()
    loss = float(net.loss_backward(xt, at, tt).cpu().numpy()[0])
    g = net.grads.cpu().numpy().astype(np.float64)
    shapes, p = oracle_params(net)
    L, oout, og = ocnn.forward_backward(p, x.astype(np.float64), aux, tgt, bf16_points=True)
    assert np.allclose(out, oout, rtol=1e-2, atol=1e-3 * np.abs(oout).max())
    assert abs(loss - L) <= 1e-3 * L
    gv = ocnn.unflatten(g, shapes)
    for name, _ in shapes:
        ref = og[name]
        rel = np.linalg.norm(gv[name] - ref) / max(np.linalg.norm(ref), 1e-30)
        cos = float(np.dot(gv[name].ravel(), ref.ravel()) /
                    max(np.linalg.norm(gv[name]) * np.linalg.norm(ref), 1e-300))
        print("%s rel %.3e cos %.6f" % (name, rel, cos))
        assert rel <= 5e-2 and cos >= 0.999, (name, rel, cos)
    net.sync_status()
    net.close()


def test_adam_step_matches_textbook(T):
    torch, cnn = T
    net = cnn.PoseNet(max_batch=2, seed=5)
    rng = np.random.default_rng(2)
    g = rng.normal(size=net.n_params).astype(np.float32)
    p0 = net.params.cpu().numpy().astype(np.float64)
    net.grads.copy_(torch.from_numpy(g))
    net.adam_step(1, lr=1e-3)
    m = 0.1 * g.astype(np.float64)
    v = 0.001 * g.astype(np.float64) ** 2
    want = p0 - 1e-3 * (m / 0.1) / (np.sqrt(v / 0.001) + 1e-8)
    assert np.allclose(net.params.cpu().numpy(), want, rtol=1e-5, atol=1e-7)
    net.close()


def test_fit_reduces_loss(T):
    torch, cnn = T
    rng = np.random.default_rng(4)
    net = cnn.PoseNet(max_batch=16, seed=9)
    x = torch.from_numpy(rng.uniform(0, 1, size=(16, 128, 128)).astype(np.float32)).cuda()
    aux = torch.from_numpy(rng.normal(size=(16, 25)).astype(np.float32)).cuda()
    tgt = torch.from_numpy(rng.normal(size=(16, 6)).astype(np.float32) * 0.2).cuda()
    first = None
    for t in range(1, 61):
        L = float(net.loss_backward(x, aux, tgt).cpu()[0])
        first = L if first is None else first
        net.adam_step(t, lr=1e-3)
    assert L < 0.2 * first, (first, L)
    net.close()


def test_predict_batches_within_max_batch(T):
    """cnn.predict splits its input into batches of at most the network's
    max_batch (whatever batch is asked) and gives each sample the output a
    single-sample forward gives it."""
    torch, cnn = T
    rng = np.random.default_rng(12)
    net = cnn.PoseNet(max_batch=4, seed=2)
    x = torch.from_numpy(rng.uniform(0, 1, size=(10, 128, 128)).astype(np.float32)).cuda()
    aux = torch.from_numpy(rng.normal(size=(10, 25)).astype(np.float32)).cuda()
    out = cnn.predict(net, x, aux, batch=256).cpu().numpy()
    assert out.shape == (10, 6)
    for k in (0, 5, 9):
        one = net.forward(x[k:k + 1].contiguous(), aux[k:k + 1].contiguous()).cpu().numpy()
        assert np.allclose(out[k], one[0], rtol=1e-3, atol=1e-4)  # other batch shapes may take other GEMM paths
    net.close()
