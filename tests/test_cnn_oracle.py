"""Pins of the FP64 network oracle (CPU): convolution against torch's float64
conv2d (a library special case) and its autograd, a delta input against the
closed form of the convolution, bfloat16 rounding against torch's conversion
and hand-worked values, and the whole network's gradient against central
finite differences and against a float64 torch autograd of the same graph."""
import numpy as np
import pytest
import torch

from oracle import cnn

F = torch.nn.functional


def t_conv(x, w, b=None):
    xt = torch.from_numpy(x).permute(0, 3, 1, 2)
    wt = torch.from_numpy(w).permute(0, 3, 1, 2)
    return F.conv2d(xt, wt, None if b is None else torch.from_numpy(b), stride=2, padding=1).permute(0, 2, 3, 1)


@pytest.mark.parametrize("B,H,W,Ci,Co", [(2, 9, 7, 3, 4), (1, 8, 8, 8, 16), (3, 5, 12, 1, 2), (1, 1, 1, 2, 3)])
def test_conv_matches_torch_float64(B, H, W, Ci, Co):
    rng = np.random.default_rng(B * 100 + H)
    x, w, b = rng.normal(size=(B, H, W, Ci)), rng.normal(size=(Co, 3, 3, Ci)), rng.normal(size=Co)
    y = cnn.conv_fwd(x, w, b)
    assert np.allclose(y, t_conv(x, w, b).numpy(), rtol=1e-12, atol=1e-12)
    yr = cnn.conv_fwd(x, w, b, relu=True)
    assert np.array_equal(yr, np.maximum(y, 0.0))
    gy = rng.normal(size=y.shape)
    xt = torch.from_numpy(x).requires_grad_()
    wt = torch.from_numpy(w).requires_grad_()
    bt = torch.from_numpy(b).requires_grad_()
    yt = F.conv2d(xt.permute(0, 3, 1, 2), wt.permute(0, 3, 1, 2), bt, stride=2, padding=1).permute(0, 2, 3, 1)
    (yt * torch.from_numpy(gy)).sum().backward()
    assert np.allclose(cnn.conv_dgrad(gy, w, H, W), xt.grad.numpy(), rtol=1e-12, atol=1e-12)
    dw, db = cnn.conv_wgrad(gy, x)
    assert np.allclose(dw, wt.grad.numpy(), rtol=1e-12, atol=1e-12)
    assert np.allclose(db, bt.grad.numpy(), rtol=1e-12, atol=1e-12)


def test_conv_delta_input_reads_the_kernel():
    """x = unit impulse at (ih, iw, ci): output (oh, ow, co) is w[co][kh][kw][ci]
    with ih = 2 oh - 1 + kh, iw = 2 ow - 1 + kw when those taps exist, else 0."""
    rng = np.random.default_rng(3)
    H, W, Ci, Co = 7, 6, 2, 3
    w = rng.normal(size=(Co, 3, 3, Ci))
    for ih, iw, ci in [(0, 0, 0), (3, 2, 1), (6, 5, 0), (5, 0, 1)]:
        x = np.zeros((1, H, W, Ci))
        x[0, ih, iw, ci] = 1.0
        y = cnn.conv_fwd(x, w, None)
        for oh in range(y.shape[1]):
            for ow in range(y.shape[2]):
                kh, kw = ih + 1 - 2 * oh, iw + 1 - 2 * ow
                want = w[:, kh, kw, ci] if (0 <= kh < 3 and 0 <= kw < 3) else np.zeros(Co)
                assert np.array_equal(y[0, oh, ow], want)


def test_bf16_rounding():
    v = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, 1.0 + 2 ** -9, -2.5, 0.0, 3.0e38, 1e-40])
    got = cnn.bf16(v)
    assert got[0] == 1.0 and got[1] == 1.0  # tie -> even
    assert got[2] == 1.0 + 2 ** -6  # tie -> even (odd mantissa rounds up)
    assert got[3] == 1.0 and got[4] == -2.5 and got[5] == 0.0
    rng = np.random.default_rng(4)
    x = rng.normal(size=10000) * np.exp(rng.uniform(-20, 20, size=10000))
    ref = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(cnn.bf16(x), ref)


def tiny_net(rng, channels=(1, 2, 3), hidden=4, aux=3):
    shapes = cnn.param_shapes(list(channels), hidden, aux, 6, positions=4)
    p = {name: rng.normal(size=shp) * 0.5 for name, shp in shapes}
    return shapes, p


def test_network_gradient_matches_central_differences():
    rng = np.random.default_rng(5)
    shapes, p = tiny_net(rng)
    x = rng.uniform(0, 1, size=(2, 8, 8))
    aux = rng.normal(size=(2, 3))
    tgt = rng.normal(size=(2, 6))
    L, _, g = cnn.forward_backward(p, x, aux, tgt, bf16_points=False)
    vec = cnn.flatten(p, shapes)
    gvec = cnn.flatten(g, shapes)
    for k in range(vec.size):
        h = 1e-6 * max(1.0, abs(vec[k]))
        vp, vm = vec.copy(), vec.copy()
        vp[k] += h
        vm[k] -= h
        Lp = cnn.forward_backward(cnn.unflatten(vp, shapes), x, aux, tgt, bf16_points=False, want_grad=False)[0]
        Lm = cnn.forward_backward(cnn.unflatten(vm, shapes), x, aux, tgt, bf16_points=False, want_grad=False)[0]
        fd = (Lp - Lm) / (2 * h)
        assert abs(fd - gvec[k]) <= 1e-6 * max(abs(fd), 1e-3 * np.abs(gvec).max()), (k, fd, gvec[k])


def test_network_matches_torch_autograd_float64():
    rng = np.random.default_rng(6)
    shapes, p = tiny_net(rng, channels=(1, 4, 8, 8), hidden=5, aux=2)
    x = rng.uniform(0, 1, size=(3, 16, 12))
    aux = rng.normal(size=(3, 2))
    tgt = rng.normal(size=(3, 6))
    L, out, g = cnn.forward_backward(p, x, aux, tgt, bf16_points=False)
    tp = {k: torch.from_numpy(v.copy()).requires_grad_() for k, v in p.items()}
    a = torch.from_numpy(x)[:, None]
    for l in range(1, 4):
        a = F.relu(F.conv2d(a, tp["conv%d.w" % l].permute(0, 3, 1, 2), tp["conv%d.b" % l], stride=2, padding=1))
    f = a.permute(0, 2, 3, 1).reshape(a.shape[0], -1)  # position-major flatten of the NHWC map
    h = torch.cat([f, torch.from_numpy(aux)], 1)
    o = F.relu(h @ tp["fc1.w"].T + tp["fc1.b"]) @ tp["fc2.w"].T + tp["fc2.b"]
    Lt = ((o - torch.from_numpy(tgt)) ** 2).mean()
    Lt.backward()
    assert abs(L - float(Lt.detach())) <= 1e-12 * abs(L)
    assert np.allclose(out, o.detach().numpy(), rtol=1e-12, atol=1e-14)
    for k in p:
        assert np.allclose(g[k], tp[k].grad.numpy(), rtol=1e-10, atol=1e-13), k


def test_architecture_parameter_count():
    shapes = cnn.param_shapes()
    conv = sum(int(np.prod(s)) for n, s in shapes if n.startswith("conv"))
    assert conv == 2158080  # six 3x3 conv layers 1-32-64-128-256-256-512 with biases
    assert sum(int(np.prod(s)) for _, s in shapes) == conv + (2048 + 25) * 256 + 256 + 256 * 6 + 6
