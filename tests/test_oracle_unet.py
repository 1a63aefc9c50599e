"""Pins of the float64 U-Net oracle: central finite differences of the loss against the
backward pass, the adjoint identities of its building blocks, and the residual design (a zero
output layer returns the diffusion fill exactly). CPU only."""
import numpy as np
import pytest

from oracle import unet as U

WIDTHS = (4, 6, 6, 8)


def _setup(seed=0, N=2, H=16, W=16, cin=3):
    rng = np.random.default_rng(seed)
    p = U.init_params(rng, cin, WIDTHS)
    x = rng.normal(size=(N, H, W, cin))
    fill = rng.normal(size=(N, H, W))
    target = rng.normal(size=(N, H, W))
    hidden = (rng.random((N, H, W)) < 0.4).astype(float)
    return p, x, fill, target, hidden


def _loss(p, x, fill, target, hidden):
    res, _ = U.forward(p, x, WIDTHS)
    return U.loss_and_grad_out(res, fill, target, hidden)[0]


def test_im2col_col2im_adjoint():
    rng = np.random.default_rng(1)
    x = rng.normal(size=(2, 5, 7, 3))
    c = rng.normal(size=(2 * 5 * 7, 27))
    assert np.isclose((U.im2col(x) * c).sum(), (x * U.col2im(c, x.shape)).sum(), rtol=1e-12)


def test_pool_and_upsample_adjoints():
    rng = np.random.default_rng(2)
    x = rng.normal(size=(2, 6, 8, 3))
    dy = rng.normal(size=(2, 3, 4, 3))
    u = rng.normal(size=(2, 6, 8, 3))
    assert np.isclose((U.upsample(dy) * u).sum(), (dy * U.upsample_backward(u)).sum(), rtol=1e-12)
    g = U.maxpool_backward(x, dy)
    # the gradient lands on the window maxima only and sums to dy per window
    assert np.allclose(U.upsample_backward(g), dy)
    assert np.all((g != 0) <= (x == U.upsample(U.maxpool(x))))


def test_conv_matches_direct_loops():
    rng = np.random.default_rng(3)
    x = rng.normal(size=(1, 4, 5, 2))
    w = rng.normal(size=(3, 3, 2, 3))
    b = rng.normal(size=3)
    y = U.conv3x3(x, w, b)
    for yy in range(4):
        for xx in range(5):
            for co in range(3):
                s = b[co]
                for ky in range(3):
                    for kx in range(3):
                        sy, sx = yy + ky - 1, xx + kx - 1
                        if 0 <= sy < 4 and 0 <= sx < 5:
                            s += x[0, sy, sx] @ w[ky, kx, :, co]
                assert np.isclose(y[0, yy, xx, co], s, rtol=1e-12)


@pytest.mark.parametrize("name", ["e1a.w", "e2b.w", "e4a.b", "d3a.w", "d1b.w", "out.w", "out.b"])
def test_gradients_central_differences(name):
    p, x, fill, target, hidden = _setup()
    res, a = U.forward(p, x, WIDTHS)
    _, dres = U.loss_and_grad_out(res, fill, target, hidden)
    g = U.backward(p, a, dres, WIDTHS)
    rng = np.random.default_rng(4)
    flat = p[name].reshape(-1)
    for k in rng.choice(flat.size, size=min(6, flat.size), replace=False):
        eps = 1e-6
        old = flat[k]
        flat[k] = old + eps
        lp = _loss(p, x, fill, target, hidden)
        flat[k] = old - eps
        lm = _loss(p, x, fill, target, hidden)
        flat[k] = old
        fd = (lp - lm) / (2 * eps)
        an = g[name].reshape(-1)[k]
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(fd)) + 1e-9, (name, k, fd, an)


def test_zero_output_layer_returns_fill():
    p, x, fill, target, hidden = _setup(5)
    p["out.w"][:] = 0
    p["out.b"][:] = 0
    res, _ = U.forward(p, x, WIDTHS)
    assert np.all(res == 0)
    pred = fill + res
    assert np.array_equal(pred, fill)


def test_loss_counts_hidden_cells_only():
    """Masked MSE: the mean of (fill + residual - target)^2 over hidden cells; visible cells add
    nothing and get no gradient."""
    rng = np.random.default_rng(9)
    res, fill, target = rng.normal(size=(3, 2, 6, 5))
    hidden = np.zeros((2, 6, 5))
    hidden[0, 1, 2] = hidden[1, 4, 0] = hidden[1, 5, 4] = 1.0
    loss, g = U.loss_and_grad_out(res, fill, target, hidden)
    d = (fill + res - target)[hidden == 1]
    assert loss == pytest.approx((d ** 2).sum() / 3, rel=1e-12)
    assert np.all(g[hidden == 0] == 0)
    np.testing.assert_allclose(g[hidden == 1], 2 * d / 3, rtol=1e-12)


# --------------------------------------------------------------------------- storage rounding

def test_round_bf16_values_and_ties():
    """Nearest bfloat16, ties to even: 1 + 2^-8 lies halfway between 1 and 1 + 2^-7 and goes
    to 1 (even); 1 + 3 * 2^-8 goes to 1 + 2^-6; exact bf16 values, signs, zero stay."""
    v = np.array([1 + 2 ** -8, 1 + 3 * 2 ** -8, 1 + 2 ** -7, -3.0, 0.0, 1 + 2 ** -9, 1 + 2 ** -8 + 2 ** -20])
    exp = np.array([1.0, 1 + 2 ** -6, 1 + 2 ** -7, -3.0, 0.0, 1.0, 1 + 2 ** -7])
    assert np.array_equal(U.round_bf16(v), exp)


def _bf16_exact(t):
    return np.array_equal(U.round_bf16(t), t)


def test_storage_rounding_rounds_every_stored_tensor():
    """With store=round_bf16 every activation and every stored activation gradient is a bf16
    value, and the stored gradients are the ones a BF16 run keeps: the head's gradient, each
    convolution's data gradient, the three upsampled-gradient sums and the three skip sums."""
    p, x, fill, target, hidden = _setup(seed=4)
    for k in p:
        if k.endswith(".w") and k != "out.w":
            p[k] = U.round_bf16(p[k])
    x = U.round_bf16(x)
    res, a = U.forward(p, x, WIDTHS, store=U.round_bf16)
    for k, t in a.items():
        if k.endswith(".out") or k in ("e1", "e2", "e3", "e4", "d3", "d2", "d1"):
            assert _bf16_exact(t), k
    _, dres = U.loss_and_grad_out(res, fill, target, hidden)
    tr = {}
    U.backward(p, a, dres, WIDTHS, store=U.round_bf16, trace=tr)
    convs, _ = U.layer_shapes(3, WIDTHS)
    names = {"head", "up2", "up3", "up4", "skip1", "skip2", "skip3"} | {n + ".dx" for n, _, _ in convs}
    assert set(tr) == names
    for k, t in tr.items():
        assert _bf16_exact(t), k
        assert np.abs(t).sum() > 0, k


def test_storage_rounding_stays_near_the_exact_network():
    """Rounding the stored tensors perturbs the result, but only as rounding can: the residual
    within 2e-2 of float64 and every gradient pointing the same way (cosine > 0.9) -- a
    rounding that flips a ReLU or a max-pool choice near a tie moves a far layer's gradient by
    up to tens of per cent on a small network, so no tighter bound holds for every layer."""
    p, x, fill, target, hidden = _setup(seed=5, H=32, W=32)
    r0, a0 = U.forward(p, x, WIDTHS)
    r1, a1 = U.forward(p, x, WIDTHS, store=U.round_bf16)
    assert np.linalg.norm(r1 - r0) / np.linalg.norm(r0) < 2e-2
    g0 = U.backward(p, a0, U.loss_and_grad_out(r0, fill, target, hidden)[1], WIDTHS)
    g1 = U.backward(p, a1, U.loss_and_grad_out(r1, fill, target, hidden)[1], WIDTHS, store=U.round_bf16)
    for k in g0:
        a, b = g1[k].ravel(), g0[k].ravel()
        assert (a @ b) / (np.linalg.norm(a) * np.linalg.norm(b)) > 0.9, k
    # without store the result is the plain float64 network, bit for bit
    r2, a2 = U.forward(p, x, WIDTHS, store=None)
    assert np.array_equal(r2, r0)
