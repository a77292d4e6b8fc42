"""Pins of the preconditioner oracle (oracle/precond.py) against independent
references: scipy's correlation, brute-force loops, the adjoint identities that
define the backward passes, Adam's first step in closed form, and torch's BF16
conversion (CPU only)."""
import numpy as np
import pytest

from oracle import precond as P


def _rng(seed):
    return np.random.default_rng(seed)


def test_single_channel_conv_is_scipy_correlate():
    ndimage = pytest.importorskip("scipy.ndimage")
    rng = _rng(0)
    x = rng.standard_normal((1, 5, 6, 7))
    k = rng.standard_normal((3, 3, 3))
    y = P.conv3d(x, k.reshape(1, 1, 27), np.array([0.25]))
    ref = ndimage.correlate(x[0], k, mode="constant", cval=0.0) + 0.25
    assert np.allclose(y[0], ref, rtol=1e-13, atol=1e-13)


def test_conv_matches_brute_force_loops():
    rng = _rng(1)
    ci, co, D, H, W = 3, 2, 2, 3, 4
    x = rng.standard_normal((ci, D, H, W))
    w = rng.standard_normal((co, ci, 3, 3, 3))
    b = rng.standard_normal(co)
    y = P.conv3d(x, w.reshape(co, ci, 27), b)
    for o in range(co):
        for z in range(D):
            for yy in range(H):
                for xx in range(W):
                    s = b[o]
                    for c in range(ci):
                        for kz in range(3):
                            for ky in range(3):
                                for kx in range(3):
                                    zz, y2, x2 = z + kz - 1, yy + ky - 1, xx + kx - 1
                                    if 0 <= zz < D and 0 <= y2 < H and 0 <= x2 < W:
                                        s += w[o, c, kz, ky, kx] * x[c, zz, y2, x2]
                    assert y[o, z, yy, xx] == pytest.approx(s, rel=1e-12, abs=1e-12)


def test_backward_passes_are_the_adjoints():
    """<conv(x, w), dy> = <x, bwd_data(dy, w)> = <w, bwd_weight(dy, x)>, and the bias
    gradient is the sum of dy: the defining identities of the two transposes."""
    rng = _rng(2)
    ci, co, shape = 3, 4, (5, 4, 6)
    x = rng.standard_normal((ci, *shape))
    w = rng.standard_normal((co, ci, 27))
    b = rng.standard_normal(co)
    dy = rng.standard_normal((co, *shape))
    lhs = np.sum(P.conv3d(x, w) * dy)
    assert np.sum(x * P.conv3d_backward_data(dy, w, ci)) == pytest.approx(lhs, rel=1e-12)
    dw, db = P.conv3d_backward_weight(dy, x)
    assert np.sum(w * dw) == pytest.approx(lhs, rel=1e-12)
    assert np.sum((P.conv3d(x, w, b) - P.conv3d(x, w)) * dy) == pytest.approx(np.sum(b * db), rel=1e-12)


def test_mse_and_relu_backward():
    y = np.array([1.0, -2.0, 3.0, 0.5])
    t = np.array([0.0, -2.0, 1.0, 1.5])
    loss, g = P.mse(y, t)
    assert loss == pytest.approx((1 + 0 + 4 + 1) / 8)
    assert np.allclose(g, (y - t) / 4)
    assert np.array_equal(P.relu_backward(np.ones(4), np.array([0.0, 2.0, -1.0, 1e-30])), [0, 1, 0, 1])


def test_adam_first_step_closed_form():
    """With zero moments, step 1 moves every parameter by lr g / (|g| + eps)."""
    rng = _rng(3)
    p = rng.standard_normal(10)
    g = rng.standard_normal(10)
    p1, m, v = P.adam(p, g, np.zeros(10), np.zeros(10), 1, lr=0.01, eps=1e-8)
    assert np.allclose(p1, p - 0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)
    # a constant gradient keeps moving by about lr a step
    p2, _, _ = P.adam(p1, g, m, v, 2, lr=0.01, eps=1e-8)
    assert np.allclose(p1 - p2, 0.01 * np.sign(g), rtol=1e-6)


def test_bf16_rounding():
    one = 1.0
    cases = {one: one, one + 2 ** -8: one, one + 3 * 2 ** -8: one + 2 ** -6, one + 2 ** -8 + 2 ** -20: one + 2 ** -7,
             -2.5: -2.5, 0.0: 0.0, 3.0e-39: None}
    for x, want in cases.items():
        if want is not None:
            assert P.bf16_round(np.float32(x)) == want, x
    torch = pytest.importorskip("torch")
    x = _rng(4).standard_normal(4096).astype(np.float32) * np.float32(1e3)
    ref = torch.tensor(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(P.bf16_round(x), ref)
    assert np.array_equal(P.bf16_value(P.bf16_bits(x)), ref)


@pytest.mark.parametrize("shape", [(4, 6, 8), (5, 7, 9), (1, 3, 2)])
def test_pool_and_upsample_pins(shape):
    """Pooling a constant field gives the constant; pooling what upsampling produced gives
    the coarse field back (every voxel of a cell holds its value); the backward passes are
    the transposed maps (dot-product test); a brute-force mean on one cell."""
    rng = _rng(21)
    C = 3
    x = rng.standard_normal((C,) + shape)
    cz, cy, cx = ((n + 1) // 2 for n in shape)
    assert np.allclose(P.pool2(np.full((C,) + shape, 2.5)), 2.5, rtol=0, atol=1e-15)
    xc = rng.standard_normal((C, cz, cy, cx))
    assert np.allclose(P.pool2(P.upsample2(xc, shape)), xc, rtol=0, atol=1e-14)
    dyc = rng.standard_normal((C, cz, cy, cx))
    assert np.isclose((P.pool2(x) * dyc).sum(), (x * P.pool2_backward(dyc, shape)).sum(), rtol=1e-12)
    dyf = rng.standard_normal((C,) + shape)
    assert np.isclose((P.upsample2(xc, shape) * dyf).sum(), (xc * P.upsample2_backward(dyf)).sum(), rtol=1e-12)
    # the last cell along every axis of an odd grid holds one voxel along that axis
    q = (cz - 1, cy - 1, cx - 1)
    block = x[:, 2 * q[0]:2 * q[0] + 2, 2 * q[1]:2 * q[1] + 2, 2 * q[2]:2 * q[2] + 2]
    assert np.allclose(P.pool2(x)[:, q[0], q[1], q[2]], block.reshape(C, -1).mean(axis=1), rtol=1e-14)
