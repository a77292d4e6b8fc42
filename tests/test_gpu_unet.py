"""The U-Net of the learned preconditioner (precond.UNet) on the library's kernels:
the 2x pooling and upsampling kernels against the oracle, the network's backward pass
(with its skip connections) against the oracle's chain on the network's own BF16
activations, and a training run that fits a teacher network."""
import numpy as np
import pytest

from helpers import rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import precond as P  # noqa: E402

SHAPE = (5, 7, 9)  # odd sizes: every level has clipped pooling cells


def _vals(t):
    """FP64 values of a BF16 or FP32 tensor."""
    if t.dtype == torch.bfloat16:
        return P.bf16_value(t.contiguous().view(torch.int16).cpu().numpy().view(np.uint16))
    return t.double().cpu().numpy()


def _lib():
    from paper_1504_08340_gb300.fwi import load_library

    return load_library()


@pytest.mark.parametrize("shape", [SHAPE, (4, 6, 8), (1, 3, 2)])
def test_pool_and_upsample_kernels(shape):
    import ctypes as C

    lib = _lib()
    s = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    p = lambda t: C.c_void_p(t.data_ptr())  # noqa: E731
    rng = np.random.default_rng(5)
    Cn = 3
    cs = tuple((n + 1) // 2 for n in shape)
    x = torch.tensor(rng.standard_normal((Cn, *shape)), dtype=torch.float32, device="cuda").to(torch.bfloat16)
    y = torch.empty((Cn, *cs), dtype=torch.bfloat16, device="cuda")
    assert lib.fwi_nn_pool2_forward(p(x), Cn, *shape, p(y), s) == 0
    ref = P.pool2(_vals(x))
    assert np.abs(_vals(y) - ref).max() <= 2 ** -8 * np.abs(ref).max()
    xc = torch.tensor(rng.standard_normal((Cn, *cs)), dtype=torch.float32, device="cuda").to(torch.bfloat16)
    yf = torch.empty((Cn, *shape), dtype=torch.bfloat16, device="cuda")
    assert lib.fwi_nn_upsample2_forward(p(xc), Cn, *shape, p(yf), s) == 0
    assert np.array_equal(_vals(yf), P.upsample2(_vals(xc), shape))
    dyc = torch.tensor(rng.standard_normal((Cn, *cs)), dtype=torch.float32, device="cuda")
    dx = torch.full((Cn, *shape), 0.25, dtype=torch.float32, device="cuda")
    assert lib.fwi_nn_pool2_backward(p(dyc), Cn, *shape, 1, p(dx), s) == 0  # accumulate
    assert rel_l2(_vals(dx), 0.25 + P.pool2_backward(_vals(dyc), shape)) < 1e-6
    dyf = torch.tensor(rng.standard_normal((Cn, *shape)), dtype=torch.float32, device="cuda")
    dxc = torch.empty((Cn, *cs), dtype=torch.float32, device="cuda")
    assert lib.fwi_nn_upsample2_backward(p(dyf), Cn, *shape, 0, p(dxc), s) == 0
    assert rel_l2(_vals(dxc), P.upsample2_backward(_vals(dyf))) < 1e-6
    assert lib.fwi_nn_pool2_forward(p(x), 0, *shape, p(y), s) == 1  # size check before any work


def _oracle_backward(net, a, target):
    """The U-Net's backward chain from the oracle's primitives, on the network's own
    activations a (FP64 values) and BF16 weights."""
    (s0, s1, s2), (w0, w1, w2) = net.shapes, net.widths
    w = {n: _vals(l.w) for n, l, _ in net.convs}
    grads = {}
    L, dy = P.mse(a["y"], target)

    def layer(name, dy, x, cin):
        grads[name] = P.conv3d_backward_weight(dy, x)
        return P.conv3d_backward_data(dy, w[name], cin) if cin else None

    g = P.relu_backward(layer("d0b", dy, a["d0a"], w0), a["d0a"])
    gcat0 = layer("d0a", g, a["cat0"], w1 + w0)
    g = P.relu_backward(P.upsample2_backward(gcat0[:w1]), a["d1b"])
    g = P.relu_backward(layer("d1b", g, a["d1a"], w1), a["d1a"])
    gcat1 = layer("d1a", g, a["cat1"], w2 + w1)
    g = P.relu_backward(P.upsample2_backward(gcat1[:w2]), a["bb"])
    g = P.relu_backward(layer("bb", g, a["ba"], w2), a["ba"])
    g = layer("ba", g, a["p1"], w1)
    g = P.relu_backward(gcat1[w2:] + P.pool2_backward(g, s1), a["cat1"][w2:])
    g = P.relu_backward(layer("e1b", g, a["e1a"], w1), a["e1a"])
    g = layer("e1a", g, a["p0"], w0)
    g = P.relu_backward(gcat0[w1:] + P.pool2_backward(g, s0), a["cat0"][w1:])
    g = P.relu_backward(layer("e0b", g, a["e0a"], w0), a["e0a"])
    layer("e0a", g, a["x"], 0)
    return L, grads


def test_unet_backward_matches_oracle_and_trains():
    from paper_1504_08340_gb300.precond import UNet

    rng = np.random.default_rng(3)
    x32 = torch.tensor(rng.standard_normal((4, *SHAPE)), dtype=torch.float32, device="cuda")
    teacher = UNet(4, 2, (4, 6, 8), SHAPE, seed=9)
    target = teacher(x32)
    net = UNet(4, 2, (4, 6, 8), SHAPE, seed=1, lr=3e-3)
    x = net.to_bf16(x32)
    acts = net.forward(x)
    a = {k: _vals(v) for k, v in acts.items()}
    # layer-local forward checks: a pooled, an upsampled and a concatenated-input layer
    assert np.abs(a["p0"] - P.pool2(a["cat0"][6:])).max() <= 2 ** -8 * np.abs(a["p0"]).max()
    assert np.array_equal(a["cat1"][:8], P.upsample2(a["bb"], net.shapes[1]))
    ref = np.maximum(P.conv3d(a["cat1"], _vals(net.layer["d1a"].w), _vals(net.layer["d1a"].b)), 0)
    assert np.abs(a["d1a"] - ref).max() <= 2 ** -8 * np.abs(ref).max() + 1e-6
    L_ref, grads = _oracle_backward(net, a, target.double().cpu().numpy())
    loss0 = net.train_step(x, target)
    assert loss0 == pytest.approx(L_ref, rel=1e-6)
    for name, l, _ in net.convs:
        dw, db = grads[name]
        assert rel_l2(l.g_w32.cpu().numpy(), dw) < 1e-4, name
        assert rel_l2(l.g_b.cpu().numpy(), db) < 1e-4, name
    losses = [loss0] + [net.train_step(x, target) for _ in range(199)]
    assert all(np.isfinite(losses))
    assert losses[-1] < losses[0] / 10, (losses[0], losses[-1])


def test_unet_size_of_the_configuration():
    """The configuration's network: about one million parameters at widths (28, 56, 112)."""
    from paper_1504_08340_gb300.precond import UNet

    net = UNet(4, 2, (28, 56, 112), (9, 9, 9))
    assert 0.9e6 < net.num_params() < 1.2e6
