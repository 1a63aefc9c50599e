"""Learned inpainting on the BF16 tensor-core kernels: forward pass and parameter gradients
against the float64 oracle, and a short training run that must beat the diffusion fill."""
import numpy as np
import pytest

from oracle import unet as U
from paper_2309_16818_gb300 import synth

pytestmark = pytest.mark.gpu

WIDTHS = (32, 32, 32, 32)


@pytest.fixture(scope="module")
def torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _bf16(a):
    return synth.bf16_bits_to_f32(synth.f32_to_bf16_bits(np.asarray(a, np.float32))).astype(np.float64)


def _unflatten(flat, cin, widths):
    from paper_2309_16818_gb300.inpaint import param_layout
    p, o = {}, 0
    for name, shape in param_layout(cin, widths):
        n = int(np.prod(shape))
        p[name] = flat[o:o + n].reshape(shape).astype(np.float64)
        o += n
    return p


def _cos(a, b):
    return float((a * b).sum() / (np.linalg.norm(a) * np.linalg.norm(b) + 1e-30))


@pytest.mark.parametrize("H,W", [(32, 32), (32, 24)])
def test_forward_and_gradients_match_float64_oracle(torch, H, W):
    from paper_2309_16818_gb300 import mem as M
    from paper_2309_16818_gb300.inpaint import init_params
    rng = np.random.default_rng(0)
    N = 2
    flat = init_params(1, 3, WIDTHS, out_scale=1.0)
    x3 = rng.normal(size=(N, H, W, 3)).astype(np.float32)
    fill = rng.normal(size=(N, H, W)).astype(np.float32)
    target = rng.normal(size=(N, H, W)).astype(np.float32)
    hidden = (rng.random((N, H, W)) < 0.5).astype(np.uint8)
    net = M.UNet(3, WIDTHS)
    net.set_params(torch.from_numpy(flat).cuda())
    tx = torch.from_numpy(x3).cuda()
    tf = torch.from_numpy(fill).cuda()
    pred = net.forward(tx, tf).cpu().numpy()
    g, loss = net.gradients(tx, tf, torch.from_numpy(target).cuda(), torch.from_numpy(hidden).cuda())
    g = g.cpu().numpy()
    # oracle on the same (bf16-rounded) weights and inputs, everything else in float64
    p = _unflatten(flat, 3, WIDTHS)
    for k in p:
        if k.endswith(".w") and k != "out.w":
            p[k] = _bf16(p[k])
    res, acts = U.forward(p, _bf16(x3), WIDTHS)
    lo, dres = U.loss_and_grad_out(res, fill.astype(np.float64), target, hidden.astype(np.float64))
    go = U.backward(p, acts, dres, WIDTHS)
    # forward: bf16 activations between 14 layers -> a few parts in a thousand of the residual
    err = np.linalg.norm(pred - (fill + res)) / np.linalg.norm(res)
    assert err < 2e-2, err
    assert abs(float(loss.item()) - lo) <= 2e-2 * lo
    # gradients: activations and gradients are stored in bf16 (2^-9 relative rounding) along a
    # path of up to 28 roundings, and a rounding can flip a ReLU or a max-pool choice near a
    # tie, which reroutes a gradient; with random weights the layers farthest from the loss
    # (and the bottleneck biases, summed over only a few pixels) reach 0.1-0.15 relative
    gg = _unflatten(g, 3, WIDTHS)
    worst = []
    for name in go:
        a, b = gg[name].ravel(), go[name].ravel()
        c = _cos(a, b)
        rel = np.linalg.norm(a - b) / (np.linalg.norm(b) + 1e-30)
        worst.append((rel, c, name))
        assert c > 0.98 and rel < 0.2, (name, c, rel)
    # the layers next to the loss are much closer
    for rel, c, name in worst:
        if name.startswith(("out", "d1b")):
            assert rel < 0.03, (name, rel)


def test_forward_at_crop_size_with_several_tiles_per_block(torch):
    """Crops of 256 x 256 (the inference crop size), eight of them: the persistent convolution
    blocks then each take several 16 x 16 tiles in turn (ring slots and both accumulator buffers
    reused). Two of the crops are checked against the float64 oracle on the same bf16-rounded
    weights and inputs; the inference widths (32, 64, 128, 128)."""
    from paper_2309_16818_gb300 import mem as M
    from paper_2309_16818_gb300.inpaint import init_params
    widths = (32, 64, 128, 128)
    rng = np.random.default_rng(4)
    N, S = 8, 256
    flat = init_params(2, 3, widths, out_scale=1.0)
    x3 = rng.normal(size=(N, S, S, 3)).astype(np.float32)
    fill = rng.normal(size=(N, S, S)).astype(np.float32)
    net = M.UNet(3, widths)
    net.set_params(torch.from_numpy(flat).cuda())
    pred = net.forward(torch.from_numpy(x3).cuda(), torch.from_numpy(fill).cuda()).cpu().numpy()
    net.check()
    p = _unflatten(flat, 3, widths)
    for k in p:
        if k.endswith(".w") and k != "out.w":
            p[k] = _bf16(p[k])
    for i in (0, N - 1):
        res, _ = U.forward(p, _bf16(x3[i:i + 1]), widths)
        err = np.linalg.norm(pred[i] - (fill[i] + res[0])) / np.linalg.norm(res[0])
        assert err < 2e-2, (i, err)


def test_training_beats_diffusion_fill(torch, capsys):
    """Train on occlusion-hole crops for a few hundred Adam steps; on held-out crops the U-Net
    (diffusion fill + learned residual) must have a lower RMSE on the hidden cells than the
    diffusion fill alone."""
    from paper_2309_16818_gb300 import inpaint as I
    from paper_2309_16818_gb300 import mem as M
    S, n_train, n_test, steps, bs = 64, 256, 48, 400, 16
    gt_tr, kn_tr = synth.inpaint_crops(n_train, size=S, seed=11, lo=0.15, hi=0.6)
    gt_te, kn_te = synth.inpaint_crops(n_test, size=S, seed=12, lo=0.15, hi=0.6)
    rng = np.random.default_rng(3)

    def observed(gt, kn):
        return np.where(kn == 1, gt + rng.normal(0, 0.01, size=gt.shape), 0.0).astype(np.float32)

    dev = "cuda"
    h_tr = torch.from_numpy(observed(gt_tr, kn_tr)).to(dev)
    k_tr = torch.from_numpy(kn_tr).to(dev)
    t_tr = torch.from_numpy(gt_tr).to(dev)
    x_tr, f_tr, hid_tr, _ = I.prepare(h_tr, k_tr)
    net = M.UNet(3, (32, 64, 128, 128))
    net.set_params(torch.from_numpy(I.init_params(5, 3, (32, 64, 128, 128))).to(dev))
    losses = []
    for s in range(steps):
        idx = torch.from_numpy(rng.choice(n_train, size=bs, replace=False)).to(dev)
        l = net.train_step(x_tr[idx].contiguous(), f_tr[idx].contiguous(), t_tr[idx].contiguous(),
                           hid_tr[idx].contiguous(), lr=1e-3 if s < 300 else 3e-4)
        if s % 50 == 0 or s == steps - 1:
            losses.append(float(l.item()))
    h_te = torch.from_numpy(observed(gt_te, kn_te)).to(dev)
    k_te = torch.from_numpy(kn_te).to(dev)
    t_te = torch.from_numpy(gt_te).to(dev)
    x_te, f_te, hid_te, _ = I.prepare(h_te, k_te)
    pred = net.forward(x_te, f_te)
    r_net = I.rmse_hidden(pred, t_te, hid_te)
    r_dif = I.rmse_hidden(f_te, t_te, hid_te)
    with capsys.disabled():
        print(f"\ntraining losses {['%.2e' % x for x in losses]}")
        print(f"held-out RMSE on hidden cells: U-Net {r_net:.4f} m, diffusion {r_dif:.4f} m")
    assert np.isfinite(r_net) and r_net < r_dif
