"""Learned inpainting around the library's kernels: input preparation (diffusion fill and the
three input channels), initialisation, a training loop and RMSE evaluation. Every numeric step
runs in the library (mem_inpaint_diffusion, mem_unet_*); this module only arranges tensors.

Inputs of the network per cell: (diffusion fill - mean of the known heights), the hidden mask,
and 0.1 log(variance) with variance 1e-4 m^2 for observed and 1 m^2 for hidden cells. The
network predicts a residual added to the diffusion fill; the loss scores hidden cells only.
"""
from __future__ import annotations

import math

import numpy as np

from . import mem as M


def param_layout(cin, widths):
    """(name, shape) of every parameter in the flat order of the library."""
    c1, c2, c3, c4 = widths
    convs = [("e1a", cin, c1), ("e1b", c1, c1), ("e2a", c1, c2), ("e2b", c2, c2),
             ("e3a", c2, c3), ("e3b", c3, c3), ("e4a", c3, c4), ("e4b", c4, c4),
             ("d3a", c4 + c3, c3), ("d3b", c3, c3), ("d2a", c3 + c2, c2), ("d2b", c2, c2),
             ("d1a", c2 + c1, c1), ("d1b", c1, c1)]
    out = []
    for name, ci, co in convs:
        out.append((name + ".w", (3, 3, ci, co)))
        out.append((name + ".b", (co,)))
    out.append(("out.w", (c1, 1)))
    out.append(("out.b", (1,)))
    return out


def init_params(seed, cin, widths, out_scale=0.1):
    """He-normal 3x3 weights, small biases, a small output layer (float32, flat)."""
    rng = np.random.default_rng(seed)
    parts = []
    for name, shape in param_layout(cin, widths):
        if name == "out.w":
            parts.append(rng.normal(0, out_scale / math.sqrt(shape[0]), size=shape))
        elif name.endswith(".w"):
            parts.append(rng.normal(0, math.sqrt(2.0 / (9 * shape[2])), size=shape))
        else:
            parts.append(np.zeros(shape))
    return np.concatenate([p.ravel() for p in parts]).astype(np.float32)


def prepare(h_obs, known, tol=1e-5):
    """h_obs, known: cuda [n,H,W] (float32, uint8). Returns x3 [n,H,W,3], fill [n,H,W],
    hidden [n,H,W] uint8, the per-crop mean of known heights [n] -- the diffusion fill and the
    normalisation both run in the library (mem_inpaint_diffusion, mem_unet_prepare)."""
    h_obs, known = h_obs.contiguous(), known.contiguous()
    fill, _ = M.inpaint_diffusion(h_obs, known, tol=tol)
    x3, hidden, mean = M.unet_prepare(h_obs, known, fill)
    return x3, fill, hidden, mean


def rmse_hidden(pred, target, hidden):
    m = hidden.bool()
    d = (pred - target)[m]
    return float(d.pow(2).mean().sqrt().item()) if d.numel() else 0.0
