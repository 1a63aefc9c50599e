"""Float64 oracle of the inpainting U-Net (forward, backward, masked-MSE loss).

TEST INFRASTRUCTURE ONLY: used by the test suite to check the CUDA training and inference
kernels; nothing in the library imports it.

The network (the paper only motivates neural networks that read map layers and produce a new
layer; this layout is the reading stated in the design notes): levels of widths c = (c1, c2, c3, c4); each
level two 3x3 convolutions (zero padding) with ReLU; 2x2 max-pooling between encoder levels;
nearest-neighbour upsampling and channel concatenation [upsampled, skip] in the decoder; a
final 1x1 convolution gives a residual added to the diffusion fill. Tensors are NHWC.
Convolutions are written as im2col followed by a matrix product (the library matmul is the
only primitive used).

Storage rounding (optional, ``store=round_bf16``): a network run in BF16 keeps its activations
and its activation gradients in BF16 between layers while every sum runs in a wider format.
With ``store`` given, forward and backward round exactly the tensors such a run stores: each
convolution's output after bias and ReLU, the 1x1 head's gradient into the last activation,
every convolution's data gradient, the 2x2 sums of the upsampled part of a decoder input's
gradient, and the sum of a skip gradient and a pooled gradient. Weights, inputs, weight and
bias gradients and the loss are left to the caller (the weights and inputs are rounded before
the call when they are stored in BF16). Without ``store`` every value stays float64.
"""
from __future__ import annotations

import numpy as np


def round_bf16(x):
    """float64 -> nearest bfloat16 value (ties to even), as float64: the value is rounded to
    float32 first, then its low 16 bits are rounded away."""
    f = np.ascontiguousarray(np.asarray(x, np.float64).astype(np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return u.view(np.float32).astype(np.float64).reshape(np.shape(x))


def _keep(x):
    return x


def layer_shapes(cin: int, widths):
    """(name, C_in, C_out) of every 3x3 convolution, in execution order, then the 1x1."""
    c1, c2, c3, c4 = widths
    return [("e1a", cin, c1), ("e1b", c1, c1), ("e2a", c1, c2), ("e2b", c2, c2),
            ("e3a", c2, c3), ("e3b", c3, c3), ("e4a", c3, c4), ("e4b", c4, c4),
            ("d3a", c4 + c3, c3), ("d3b", c3, c3), ("d2a", c3 + c2, c2), ("d2b", c2, c2),
            ("d1a", c2 + c1, c1), ("d1b", c1, c1)], ("out", c1, 1)


def init_params(rng, cin: int, widths, scale: float = 1.0):
    convs, (_, co_in, _) = layer_shapes(cin, widths)
    p = {}
    for name, ci, co in convs:
        p[name + ".w"] = rng.normal(0, scale * np.sqrt(2.0 / (9 * ci)), size=(3, 3, ci, co))
        p[name + ".b"] = rng.normal(0, 0.01, size=co)
    p["out.w"] = rng.normal(0, 0.1 / np.sqrt(co_in), size=(co_in, 1))
    p["out.b"] = np.zeros(1)
    return p


def im2col(x):
    """[N,H,W,C] -> [N*H*W, 9*C] with zero padding; column order (ky, kx, c)."""
    N, H, W, C = x.shape
    xp = np.zeros((N, H + 2, W + 2, C), x.dtype)
    xp[:, 1:-1, 1:-1] = x
    cols = [xp[:, ky:ky + H, kx:kx + W, :] for ky in range(3) for kx in range(3)]
    return np.concatenate(cols, axis=3).reshape(N * H * W, 9 * C)


def col2im(cols, shape):
    """Adjoint of im2col: [N*H*W, 9*C] -> [N,H,W,C] (sums overlapping taps)."""
    N, H, W, C = shape
    cols = cols.reshape(N, H, W, 9, C)
    xp = np.zeros((N, H + 2, W + 2, C), cols.dtype)
    t = 0
    for ky in range(3):
        for kx in range(3):
            xp[:, ky:ky + H, kx:kx + W, :] += cols[:, :, :, t, :]
            t += 1
    return xp[:, 1:-1, 1:-1]


def conv3x3(x, w, b):
    N, H, W, _ = x.shape
    y = im2col(x) @ w.reshape(-1, w.shape[3]) + b
    return y.reshape(N, H, W, w.shape[3])


def conv3x3_backward(x, w, dy):
    N, H, W, _ = x.shape
    co = w.shape[3]
    d = dy.reshape(-1, co)
    dw = (im2col(x).T @ d).reshape(w.shape)
    db = d.sum(axis=0)
    dx = col2im(d @ w.reshape(-1, co).T, x.shape)
    return dx, dw, db


def maxpool(x):
    N, H, W, C = x.shape
    v = x.reshape(N, H // 2, 2, W // 2, 2, C)
    return v.max(axis=(2, 4))


def maxpool_backward(x, dy):
    """Gradient to the first maximum of each 2x2 window (row-major order)."""
    N, H, W, C = x.shape
    v = x.reshape(N, H // 2, 2, W // 2, 2, C).transpose(0, 1, 3, 5, 2, 4).reshape(N, H // 2, W // 2, C, 4)
    am = v.argmax(axis=4)
    g = np.zeros_like(v)
    np.put_along_axis(g, am[..., None], dy[..., None], axis=4)
    g = g.reshape(N, H // 2, W // 2, C, 2, 2).transpose(0, 1, 4, 2, 5, 3).reshape(N, H, W, C)
    return g


def upsample(x):
    return x.repeat(2, axis=1).repeat(2, axis=2)


def upsample_backward(dy):
    N, H, W, C = dy.shape
    return dy.reshape(N, H // 2, 2, W // 2, 2, C).sum(axis=(2, 4))


def forward(p, x, widths, store=None):
    """x: [N,H,W,Cin] -> residual [N,H,W] and the activations the backward pass needs.
    store: rounding applied to every stored activation (see the module notes)."""
    store = store or _keep
    convs, _ = layer_shapes(x.shape[3], widths)
    a = {"in": x}

    def cr(name, t):
        y = conv3x3(t, p[name + ".w"], p[name + ".b"])
        r = store(np.maximum(y, 0.0))
        a[name + ".in"] = t
        a[name + ".out"] = r
        return r

    e1 = cr("e1b", cr("e1a", x))
    e2 = cr("e2b", cr("e2a", maxpool(e1)))
    e3 = cr("e3b", cr("e3a", maxpool(e2)))
    e4 = cr("e4b", cr("e4a", maxpool(e3)))
    d3 = cr("d3b", cr("d3a", np.concatenate([upsample(e4), e3], axis=3)))
    d2 = cr("d2b", cr("d2a", np.concatenate([upsample(d3), e2], axis=3)))
    d1 = cr("d1b", cr("d1a", np.concatenate([upsample(d2), e1], axis=3)))
    out = d1 @ p["out.w"] + p["out.b"]
    a.update(e1=e1, e2=e2, e3=e3, e4=e4, d3=d3, d2=d2, d1=d1)
    return out[..., 0], a


def loss_and_grad_out(res, fill, target, hidden):
    """Masked MSE over hidden cells of (fill + residual) against the target."""
    cnt = max(1, int(hidden.sum()))
    diff = (fill + res - target) * hidden
    return float((diff ** 2).sum() / cnt), 2.0 * diff / cnt


def backward(p, a, dres, widths, store=None, trace=None):
    """Gradients of every parameter given d loss / d residual [N,H,W]. store: rounding applied
    to every stored activation gradient (see the module notes); trace (a dict, optional)
    receives each of those stored gradients under a name."""
    store = store or _keep
    g = {}

    def keep(name, t):
        t = store(t)
        if trace is not None:
            trace[name] = t
        return t

    d1 = a["d1"]
    do = dres[..., None]
    g["out.w"] = d1.reshape(-1, d1.shape[3]).T @ do.reshape(-1, 1)
    g["out.b"] = np.array([do.sum()])
    dt = keep("head", do @ p["out.w"].T)

    def crb(name, dt):
        dt = dt * (a[name + ".out"] > 0)
        dx, dw, db = conv3x3_backward(a[name + ".in"], p[name + ".w"], dt)
        g[name + ".w"], g[name + ".b"] = dw, db
        return keep(name + ".dx", dx)

    def split(dcat, c_up):
        return dcat[..., :c_up], dcat[..., c_up:]

    c1, c2, c3, c4 = widths
    dcat = crb("d1a", crb("d1b", dt))
    du, de1 = split(dcat, c2)
    dcat = crb("d2a", crb("d2b", keep("up2", upsample_backward(du))))
    du, de2 = split(dcat, c3)
    dcat = crb("d3a", crb("d3b", keep("up3", upsample_backward(du))))
    du, de3 = split(dcat, c4)
    de4 = crb("e4a", crb("e4b", keep("up4", upsample_backward(du))))
    de3 = keep("skip3", de3 + maxpool_backward(a["e3"], de4))
    de3 = crb("e3a", crb("e3b", de3))
    de2 = keep("skip2", de2 + maxpool_backward(a["e2"], de3))
    de2 = crb("e2a", crb("e2b", de2))
    de1 = keep("skip1", de1 + maxpool_backward(a["e1"], de2))
    crb("e1a", crb("e1b", de1))
    return g
