"""Diffusion inpainting, the batched-path autotuner, and the error of reduced-precision
feature storage against a float64 oracle, through the C ABI."""
import numpy as np
import pytest

import oracle as O
from paper_2309_16818_gb300 import synth

from helpers import compare_states, gpu_state, make_pair, upload_state

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.mark.parametrize("size,n", [(64, 6), (256, 2)])
def test_diffusion_inpainting_matches_exact_solution(torch, size, n):
    from paper_2309_16818_gb300 import mem as M
    h, k = synth.inpaint_crops(n, size=size, seed=size)
    hin = np.where(k == 1, h, np.float32(123.0))  # unknown cells carry garbage
    out, its = M.inpaint_diffusion(torch.from_numpy(hin).cuda(), torch.from_numpy(k).cuda(),
                                   tol=1e-6, max_iters=50000)
    out = out.cpu().numpy()
    its = its.cpu().numpy()
    for b in range(n):
        ex = O.harmonic_fill_exact(hin[b], k[b])
        assert its[b] < 50000
        # float32 sweeps stop once the largest update is below tol = 1e-6 (float32 rounding of a
        # mean of heights ~0.5 m is ~1e-7, so a smaller tol is not reachable); the remaining
        # error is at most about tol times the number of sweeps the slowest mode needs to decay,
        # ~ size / pi for over-relaxation: the bound below is tol * size
        err = np.abs(out[b] - ex).max()
        assert err < 1e-6 * size, (b, err, its[b])
        assert np.array_equal(out[b][k[b] == 1], hin[b][k[b] == 1])


def test_diffusion_per_crop_relaxation_cuts_sweeps(torch):
    """The shared-memory fill sizes its over-relaxation per crop from the largest distance of an
    unknown cell to a known one. On occlusion-hole crops of 256 x 256 the fixed factor of a
    256-cell square needs ~500-540 sweeps per crop (its error shrinks by omega - 1 = 0.976 per
    sweep whatever the holes); the per-crop factor must need far fewer, never more than the
    fixed one, and still reach the exact solution."""
    from paper_2309_16818_gb300 import mem as M
    h, k = synth.inpaint_crops(8, size=256, seed=7)
    out, its = M.inpaint_diffusion(torch.from_numpy(h).cuda(), torch.from_numpy(k).cuda(), tol=1e-6)
    its = its.cpu().numpy()
    out = out.cpu().numpy()
    assert its.max() <= 560 and its.mean() < 350, its
    for b in range(2):
        ex = O.harmonic_fill_exact(h[b], k[b])
        assert np.abs(out[b] - ex).max() < 1e-6 * 256, b


def test_diffusion_edge_cases(torch):
    from paper_2309_16818_gb300 import mem as M
    # all known: unchanged; none known: every cell keeps the mean (0); 1 x 1 and ragged sizes
    h = np.random.default_rng(0).normal(size=(3, 5, 7)).astype(np.float32)
    k = np.ones_like(h, dtype=np.uint8)
    k[1] = 0
    k[2, 2, 3] = 0
    out, _ = M.inpaint_diffusion(torch.from_numpy(h).cuda(), torch.from_numpy(k).cuda())
    out = out.cpu().numpy()
    assert np.array_equal(out[0], h[0])
    assert np.all(out[1] == 0.0)
    ex = O.harmonic_fill_exact(h[2], k[2])
    assert abs(out[2, 2, 3] - ex[2, 3]) < 1e-5
    one, _ = M.inpaint_diffusion(torch.zeros((1, 1, 1), device="cuda"),
                                 torch.zeros((1, 1, 1), dtype=torch.uint8, device="cuda"))
    assert float(one.item()) == 0.0


def _batch_sources(torch, rgb, feat):
    return [(torch.from_numpy(rgb).cuda(), [0]),
            (torch.from_numpy(feat.view(np.int16)).cuda().view(torch.bfloat16), [1])]


def test_autotune_keeps_state_and_results(torch):
    B = 12
    c = synth.config4(n_maps=B, n_lo=500, n_hi=6000)
    layers = [dict(channels=3, rule=O.LATEST), dict(channels=16, rule=O.GAUSS, dtype=O.BF16)]
    g, _ = make_pair(c["W"], c["res"], layers, n_maps=B)
    xyz, rgb, feat, _, T = synth.concat_clouds(c["clouds"])
    dx = torch.from_numpy(xyz).cuda()
    srcs = _batch_sources(torch, rgb, feat)
    g.fuse_pointcloud_batch(c["offsets"], dx, T, srcs)
    before = [gpu_state(g, b) for b in range(B)]
    tune, times = g.autotune_batch(c["offsets"], dx, T, srcs, reps=2)
    assert len(times) >= 6 and all(t > 0 for t in times)
    after = [gpu_state(g, b) for b in range(B)]
    for s0, s1 in zip(before, after):
        for key in ("h", "var", "valid", "n_acc", "n_rej"):
            assert np.array_equal(s0[key], s1[key])
        for a0, a1 in zip(s0["layers"], s1["layers"]):
            assert np.array_equal(a0, a1)
    # a second batched call with the chosen schedule still matches the oracle
    for b, cl in enumerate(c["clouds"]):
        o = O.OracleMap(O.Params(W=c["W"], res=c["res"], layers=[O.Layer(3, O.LATEST),
                                                              O.Layer(16, O.GAUSS, store=O.BF16)]))
        o.fuse_points(cl.xyz, cl.T, [(cl.rgb, [0]), ((cl.feat,), [1])])
        upload_state(g, o, map_index=b)
        o.fuse_points(cl.xyz, cl.T, [(cl.rgb, [0]), ((cl.feat,), [1])])
        c.setdefault("o", []).append(o)
    g.fuse_pointcloud_batch(c["offsets"], dx, T, srcs)
    for b in range(B):
        compare_states(gpu_state(g, b), c["o"][b], what=f"tuned map {b}")


def test_reduced_precision_error_against_float64(torch, capsys):
    """Per-layer error of BF16 / F16 / F32 feature storage against an oracle that keeps every
    value in float64, over three scans of a 40k-point cloud (Gaussian rule, 16 features)."""
    c = synth.config4(n_maps=1, n_lo=40_000, n_hi=40_001)
    cl = c["clouds"][0]
    layers = [dict(channels=16, rule=O.GAUSS, var_meas=1.0, dtype=d) for d in (O.BF16, O.F16, O.F32)]
    g, _ = make_pair(c["W"], c["res"], layers)
    o64 = O.OracleMap(O.Params(W=c["W"], res=c["res"], layers=[O.Layer(16, O.GAUSS, var_meas=1.0)] * 3),
                      round_store=False)
    feat_t = torch.from_numpy(cl.feat.view(np.int16)).cuda().view(torch.bfloat16)
    rows = []
    for k in range(3):
        g.fuse_pointcloud(torch.from_numpy(cl.xyz).cuda(), cl.T, [(feat_t, [0, 1, 2])])
        o64.fuse_points(cl.xyz, cl.T, [((cl.feat,), [0, 1, 2])])
        s = gpu_state(g)
        for l, name, bound in ((0, "bf16", 3 * 2.0 ** -8), (1, "f16", 3 * 2.0 ** -11), (2, "f32", 1e-5)):
            ob = o64.obs[l] == 1
            ref = o64.layer_values(l)[ob]
            err = np.abs(s["layers"][l][ob] - ref) / np.maximum(np.abs(ref), 1e-2)
            rows.append((k, name, float(err.max()), float(err.mean())))
            assert err.max() <= bound, (k, name, err.max())
    with capsys.disabled():
        print("\nscan storage max_rel_err mean_rel_err (vs float64 oracle, floor 1e-2)")
        for r in rows:
            print(f"{r[0]} {r[1]} {r[2]:.3e} {r[3]:.3e}")
