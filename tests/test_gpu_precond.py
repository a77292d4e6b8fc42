"""Parity of the learned preconditioner's kernels (fwi_precond.h) with the FP64 oracle
(oracle/precond.py), and a training run of the ConvNet built on them.

Tolerances follow the arithmetic: a forward output is the FP32 sum rounded to BF16,
so it is within 2^-8 of the exact value relative to its size (half a BF16 step plus
the FP32 sum's error); the FP32 backward sums of at most a few thousand products
agree with FP64 to 1e-5 relative (the tensor-core backward-data sums to the bound of
_bwd_data_tol); bitwise where nothing is rounded differently
(ReLU masks, BF16 conversions, the BF16 copy Adam writes)."""
import ctypes as C

import numpy as np
import pytest

from helpers import rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import precond as P  # noqa: E402

SHAPE = (5, 9, 11)  # 495 voxels: ragged against 256-thread blocks


def _lib():
    from paper_1504_08340_gb300.fwi import load_library

    return load_library()


def _s():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _p(t):
    return C.c_void_p(t.data_ptr())


def _bf16(a):
    """(device BF16 tensor, FP64 values) of the BF16 rounding of a."""
    bits = P.bf16_bits(np.asarray(a, dtype=np.float32))
    t = torch.from_numpy(bits.view(np.int16).copy()).view(torch.bfloat16).cuda()
    return t, P.bf16_value(bits)


def _f32(a):
    return torch.tensor(np.asarray(a, dtype=np.float32)).cuda()


def _bits(t):
    return t.cpu().view(torch.int16).numpy().view(np.uint16)


def _vals(t):
    return P.bf16_value(_bits(t))


@pytest.mark.parametrize("cin,cout,relu", [(3, 10, 1), (4, 8, 0), (1, 1, 0)])
def test_conv_forward(cin, cout, relu):
    rng = np.random.default_rng(cin * 100 + cout)
    xd, xv = _bf16(rng.standard_normal((cin, *SHAPE)))
    wd, wv = _bf16(rng.standard_normal((cout, cin, 27)) / np.sqrt(27 * cin))
    b = rng.standard_normal(cout).astype(np.float32)
    y = torch.empty((cout, *SHAPE), dtype=torch.bfloat16, device="cuda")
    bd = _f32(b)
    assert _lib().fwi_nn_conv3d_forward(_p(xd), _p(wd), _p(bd), cin, cout, *SHAPE, relu, _p(y), _s()) == 0
    ref = P.conv3d(xv, wv, b.astype(np.float64))
    if relu:
        ref = np.maximum(ref, 0)
    got = _vals(y)
    assert np.all(np.abs(got - ref) <= 2.0 ** -8 * np.abs(ref) + 1e-5)
    # away from rounding ties the BF16 patterns agree exactly
    assert np.mean(_bits(y) == P.bf16_bits(ref)) > 0.99


@pytest.mark.parametrize("cin,cout,shape", [(37, 300, (7, 13, 17)), (32, 112, (6, 16, 16)), (112, 16, (3, 5, 9))])
def test_conv_forward_tensor_core_tiles(cin, cout, shape):
    # the tensor-core tiling at its edges: two output-channel tiles (256 + 44), input
    # channels off the 8-channel core width (K = 27 x 40, ragged against 64-wide chunks),
    # voxel counts off the 128-voxel tile, and wide K (27 x 112)
    rng = np.random.default_rng(cin + cout)
    xd, xv = _bf16(rng.standard_normal((cin, *shape)))
    wd, wv = _bf16(rng.standard_normal((cout, cin, 27)) / np.sqrt(27 * cin))
    b = rng.standard_normal(cout).astype(np.float32)
    y = torch.empty((cout, *shape), dtype=torch.bfloat16, device="cuda")
    assert _lib().fwi_nn_conv3d_forward(_p(xd), _p(wd), _p(_f32(b)), cin, cout, *shape, 1, _p(y), _s()) == 0
    ref = np.maximum(P.conv3d(xv, wv, b.astype(np.float64)), 0)
    got = _vals(y)
    assert np.all(np.abs(got - ref) <= 2.0 ** -8 * np.abs(ref) + 1e-5)
    assert np.mean(_bits(y) == P.bf16_bits(ref)) > 0.99
    # the same call again gives the same bits
    y2 = torch.empty_like(y)
    assert _lib().fwi_nn_conv3d_forward(_p(xd), _p(wd), _p(_f32(b)), cin, cout, *shape, 1, _p(y2), _s()) == 0
    assert torch.equal(y.view(torch.int16), y2.view(torch.int16))


def _bwd_data_tol(cout):
    """Relative L2 bound of the backward-data sums: K = 27 x 3 x ceil(cout / 8) x 8 exact
    products (three BF16 parts of each FP32 gradient value, BF16 weights) accumulated in
    FP32 on the tensor cores. A random walk of round-to-nearest adds would give about
    2^-24 sqrt(K). The tensor cores' internal accumulation is not a sequence of
    round-to-nearest adds (it measured about twice that estimate at K = 9072), so the bound
    takes four times it: 2^-22 sqrt(K)."""
    k = 27 * 3 * ((cout + 7) // 8 * 8)
    return 2.0 ** -22 * np.sqrt(k)


@pytest.mark.parametrize("cin,cout", [(3, 10), (9, 2)])
def test_conv_backward_data(cin, cout):
    rng = np.random.default_rng(7 + cin)
    dy = rng.standard_normal((cout, *SHAPE)).astype(np.float32)
    wd, wv = _bf16(rng.standard_normal((cout, cin, 27)))
    dx = torch.empty((cin, *SHAPE), dtype=torch.float32, device="cuda")
    dyd = _f32(dy)
    assert _lib().fwi_nn_conv3d_backward_data(_p(dyd), _p(wd), cin, cout, *SHAPE, _p(dx), _s()) == 0
    ref = P.conv3d_backward_data(dy.astype(np.float64), wv, cin)
    assert rel_l2(dx.cpu().numpy(), ref) < _bwd_data_tol(cout)
    assert np.abs(dx.cpu().numpy() - ref).max() <= 1e-5 * np.abs(ref).max()


@pytest.mark.parametrize("cin,cout,shape", [(300, 37, (3, 5, 9)), (32, 112, (6, 16, 16))])
def test_conv_backward_data_tensor_core_tiles(cin, cout, shape):
    # two output tiles of the GEMM (256 + 44 input channels), gradient channels off the
    # 8-channel core width (three BF16 parts each), voxel counts off the 128-voxel tile;
    # FP32 accuracy from the split gradient, and the same bits on a second call
    rng = np.random.default_rng(cin * 3 + cout)
    dy = (rng.standard_normal((cout, *shape)) * np.exp(rng.uniform(-8, 8, (cout, *shape)))).astype(np.float32)
    wd, wv = _bf16(rng.standard_normal((cout, cin, 27)))
    dx = torch.empty((cin, *shape), dtype=torch.float32, device="cuda")
    dyd = _f32(dy)
    assert _lib().fwi_nn_conv3d_backward_data(_p(dyd), _p(wd), cin, cout, *shape, _p(dx), _s()) == 0
    ref = P.conv3d_backward_data(dy.astype(np.float64), wv, cin)
    assert rel_l2(dx.cpu().numpy(), ref) < _bwd_data_tol(cout)
    dx2 = torch.empty_like(dx)
    assert _lib().fwi_nn_conv3d_backward_data(_p(dyd), _p(wd), cin, cout, *shape, _p(dx2), _s()) == 0
    assert torch.equal(dx, dx2)


@pytest.mark.parametrize("cin,cout,shape", [(3, 5, SHAPE), (2, 3, (20, 20, 24)), (37, 300, (7, 20, 33))])
def test_conv_backward_weight(cin, cout, shape):
    """The second shape spans five 2048-voxel slices of the partial sums, the last ragged;
    the third nine tensor-core row tiles (27 x 40 tap-channel rows and the bias row), two
    output-channel tiles (256 + 44) and three slices."""
    lib = _lib()
    rng = np.random.default_rng(17 + cin)
    dy = rng.standard_normal((cout, *shape)).astype(np.float32)
    xd, xv = _bf16(rng.standard_normal((cin, *shape)))
    work = torch.empty(lib.fwi_nn_conv3d_backward_weight_work(cin, cout, *shape), dtype=torch.float32, device="cuda")
    dw = torch.empty((cout, cin, 27), dtype=torch.float32, device="cuda")
    db = torch.empty(cout, dtype=torch.float32, device="cuda")
    dyd = _f32(dy)
    assert lib.fwi_nn_conv3d_backward_weight(_p(dyd), _p(xd), cin, cout, *shape, _p(dw), _p(db), _p(work), _s()) == 0
    dw_ref, db_ref = P.conv3d_backward_weight(dy.astype(np.float64), xv)
    assert rel_l2(dw.cpu().numpy(), dw_ref) < 1e-5
    assert rel_l2(db.cpu().numpy(), db_ref) < 1e-5
    # fixed-order sums: a second call gives the same bits
    dw2 = torch.empty_like(dw)
    assert lib.fwi_nn_conv3d_backward_weight(_p(dyd), _p(xd), cin, cout, *shape, _p(dw2), None, _p(work), _s()) == 0
    assert torch.equal(dw, dw2)


def test_relu_backward_mse_and_conversions():
    lib = _lib()
    rng = np.random.default_rng(5)
    n = 3001
    a = rng.standard_normal(n).astype(np.float32)
    a[:8] = [0.0, -0.0, 1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -8, -3.5, 1e-30, -1e-30]
    yd, yv = _bf16(a)
    bits = torch.empty(n, dtype=torch.bfloat16, device="cuda")
    ad = _f32(a)
    assert lib.fwi_nn_to_bf16(_p(ad), n, _p(bits), _s()) == 0
    assert np.array_equal(_bits(bits), P.bf16_bits(a))
    back = torch.empty(n, dtype=torch.float32, device="cuda")
    assert lib.fwi_nn_from_bf16(_p(bits), n, _p(back), _s()) == 0
    assert np.array_equal(back.cpu().numpy().astype(np.float64), yv)
    dy = rng.standard_normal(n).astype(np.float32)
    out = torch.empty(n, dtype=torch.float32, device="cuda")
    dyd = _f32(dy)
    assert lib.fwi_nn_relu_backward(_p(dyd), _p(yd), n, _p(out), _s()) == 0
    assert np.array_equal(out.cpu().numpy(), np.where(yv > 0, dy, 0.0).astype(np.float32))
    t = rng.standard_normal(n).astype(np.float32)
    g = torch.empty(n, dtype=torch.float32, device="cuda")
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    work = torch.empty(1024, dtype=torch.float64, device="cuda")
    td = _f32(t)
    assert lib.fwi_nn_mse(_p(yd), _p(td), n, _p(g), _p(loss), _p(work), _s()) == 0
    L_ref, g_ref = P.mse(yv, t.astype(np.float64))
    assert loss.item() == pytest.approx(L_ref, rel=1e-6)
    assert rel_l2(g.cpu().numpy(), g_ref) < 1e-6


def test_adam_steps():
    lib = _lib()
    rng = np.random.default_rng(6)
    n = 777
    p0 = rng.standard_normal(n).astype(np.float32)
    master, m, v = _f32(p0), torch.zeros(n, device="cuda"), torch.zeros(n, device="cuda")
    w = torch.empty(n, dtype=torch.bfloat16, device="cuda")
    p_ref, m_ref, v_ref = p0.astype(np.float64), np.zeros(n), np.zeros(n)
    # the hyperparameters reach the kernel as FP32 values: the oracle takes the same ones
    lr, b1, b2, eps = (float(np.float32(h)) for h in (1e-2, 0.9, 0.999, 1e-8))
    for t in range(1, 4):
        g = rng.standard_normal(n).astype(np.float32)
        gd = _f32(g)
        assert lib.fwi_nn_adam(_p(master), _p(w), _p(gd), _p(m), _p(v), n, lr, b1, b2, eps, t, _s()) == 0
        p_ref, m_ref, v_ref = P.adam(p_ref, g.astype(np.float64), m_ref, v_ref, t, lr, b1, b2, eps)
    assert rel_l2(master.cpu().numpy(), p_ref) < 1e-6
    assert rel_l2(m.cpu().numpy(), m_ref) < 1e-6 and rel_l2(v.cpu().numpy(), v_ref) < 1e-6
    assert np.array_equal(_bits(w), P.bf16_bits(master.cpu().numpy()))


def test_convnet_backprop_and_training():
    """The chained backward pass of ConvNet equals the oracle's on the same activations,
    and 100 Adam steps fit a teacher network of the same shape (the loss drops more than
    tenfold; an FP64 oracle simulation of the same run drops about 70-fold)."""
    from paper_1504_08340_gb300.precond import ConvNet

    rng = np.random.default_rng(11)
    x32 = rng.standard_normal((4, *SHAPE)).astype(np.float32)
    teacher = ConvNet((4, 8, 2), SHAPE, seed=7)
    x32d = _f32(x32)
    target = teacher(x32d)
    net = ConvNet((4, 8, 2), SHAPE, seed=0, lr=1e-2)
    x = net.to_bf16(x32d)
    acts = net.forward(x)
    a = [_vals(t) for t in acts]
    w = [_vals(l["w"]) for l in net.layers]
    # oracle gradients from the network's own activations and BF16 weights
    L_ref, dy = P.mse(a[2], target.cpu().numpy().astype(np.float64))
    dw1, db1 = P.conv3d_backward_weight(dy, a[1])
    dy1 = P.relu_backward(P.conv3d_backward_data(dy, w[1], 8), a[1])
    dw0, db0 = P.conv3d_backward_weight(dy1, a[0])
    loss0 = net.train_step(x, target)
    assert loss0 == pytest.approx(L_ref, rel=1e-6)
    for l, (dw, db) in zip(net.layers, ((dw0, db0), (dw1, db1))):
        assert rel_l2(l["g_w32"].cpu().numpy(), dw) < 1e-5
        assert rel_l2(l["g_b"].cpu().numpy(), db) < 1e-5
    losses = [loss0] + [net.train_step(x, target) for _ in range(99)]
    assert all(np.isfinite(losses))
    assert losses[-1] < losses[0] / 10
