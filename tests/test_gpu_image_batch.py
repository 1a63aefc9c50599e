"""CUDA image association / fusion and the batched point path against the oracle,
element by element, through the C ABI."""
import numpy as np
import pytest

import oracle as O
from paper_2309_16818_gb300 import synth

from helpers import compare_states, cuda_xyz, gpu_state, make_pair, upload_state

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


IMG_LAYERS = [dict(channels=64, rule=O.GAUSS, var_meas=1.0), dict(channels=20, rule=O.DIRICHLET),
              dict(channels=20, rule=O.CLASSMAX), dict(channels=64, rule=O.EXPAVG, w=0.3)]


@pytest.mark.parametrize("scale,feat_store", [(0.25, O.F32), (0.5, O.BF16)])
def test_image_fusion_cameras(torch, scale, feat_store):
    c = synth.config3(scale=scale)
    layers = [dict(IMG_LAYERS[0], dtype=feat_store)] + IMG_LAYERS[1:]
    g, o = make_pair(c["W"], c["res"], layers)
    pre = c["prefill"]
    o.move(c["robot"][:2])
    g.move(c["robot"][:2])
    o.fuse_points(pre.xyz, pre.T)
    assert o.valid.sum() > 5000
    for i, cam in enumerate(c["cameras"]):
        upload_state(g, o)
        H, Wi = cam.H, cam.Wi
        feat = cam.feat.reshape(H * Wi, -1)
        seg = cam.seg.reshape(H * Wi, -1)
        ro = o.fuse_image(H, Wi, [(feat, [0, 3]), (seg, [1, 2])], cam.K, cam.T)
        vis = torch.empty(c["W"] ** 2, dtype=torch.uint8, device="cuda")
        pix = torch.empty(c["W"] ** 2, dtype=torch.int32, device="cuda")
        g.fuse_image(H, Wi, cam.K, cam.T,
                     [(torch.from_numpy(cam.feat).cuda(), [0, 3]), (torch.from_numpy(cam.seg).cuda(), [1, 2])],
                     vis=vis, pix=pix)
        g.check()
        assert ro["n_visible"] > 1000
        assert np.array_equal(vis.cpu().numpy(), ro["vis"]), f"camera {i}: visibility"
        assert np.array_equal(pix.cpu().numpy(), ro["pix"]), f"camera {i}: pixel indices"
        compare_states(gpu_state(g), o, what=f"camera {i}")


def test_image_bf16_pixels_and_empty_frustum(torch):
    c = synth.config3(scale=0.25, n_feat=16)
    layers = [dict(channels=16, rule=O.GAUSS, var_meas=0.5, dtype=O.BF16), dict(channels=16, rule=O.LATEST)]
    g, o = make_pair(c["W"], c["res"], layers)
    o.fuse_points(c["prefill"].xyz, c["prefill"].T)
    cam = c["cameras"][0]
    bits = synth.f32_to_bf16_bits(cam.feat)
    upload_state(g, o)
    ro = o.fuse_image(cam.H, cam.Wi, [((bits.reshape(cam.H * cam.Wi, -1),), [0, 1])], cam.K, cam.T)
    t = torch.from_numpy(bits.view(np.int16)).cuda().view(torch.bfloat16)
    vis = torch.empty(c["W"] ** 2, dtype=torch.uint8, device="cuda")
    g.fuse_image(cam.H, cam.Wi, cam.K, cam.T, [(t, [0, 1])], vis=vis)
    assert np.array_equal(vis.cpu().numpy(), ro["vis"])
    compare_states(gpu_state(g), o, what="bf16 pixels")
    # a camera looking straight up sees nothing
    T = cam.T.copy()
    T[:3, :3] = np.eye(3)  # optical axis = world +z
    g.fuse_image(cam.H, cam.Wi, cam.K, T, [(t, [0, 1])], vis=vis)
    ro = o.fuse_image(cam.H, cam.Wi, [((bits.reshape(cam.H * cam.Wi, -1),), [0, 1])], cam.K, T)
    assert ro["n_visible"] == 0 and int(vis.sum()) == 0


def _batch_sources(torch, rgb, feat):
    return [(torch.from_numpy(rgb).cuda(), [0]),
            (torch.from_numpy(feat.view(np.int16)).cuda().view(torch.bfloat16), [1])]


def test_batched_maps_equal_per_map_oracle(torch):
    B = 24
    c = synth.config4(n_maps=B, n_lo=300, n_hi=9000)
    layers = [dict(channels=3, rule=O.LATEST), dict(channels=16, rule=O.GAUSS, dtype=O.BF16)]
    g, _ = make_pair(c["W"], c["res"], layers, n_maps=B)
    oracles = [O.OracleMap(
        O.Params(W=c["W"], res=c["res"], layers=[O.Layer(3, O.LATEST), O.Layer(16, O.GAUSS, store=O.BF16)]))
        for _ in range(B)]
    xyz, rgb, feat, _, T = synth.concat_clouds(c["clouds"])
    for rnd in range(2):
        for b, cl in enumerate(c["clouds"]):
            xy = cl.T[:2, 3] + 0.3 * rnd
            oracles[b].move(xy)
            g.move(xy, map_index=b)
            if rnd:
                upload_state(g, oracles[b], map_index=b)
        for b, cl in enumerate(c["clouds"]):
            oracles[b].fuse_points(cl.xyz, cl.T, [(cl.rgb, [0]), ((cl.feat,), [1])])
        g.fuse_pointcloud_batch(c["offsets"], torch.from_numpy(xyz).cuda(), T, _batch_sources(torch, rgb, feat))
        g.check()
        for b in range(B):
            assert g.origin(b) == oracles[b].origin
            compare_states(gpu_state(g, b), oracles[b], what=f"round {rnd} map {b}")


def test_batched_with_empty_maps(torch):
    B = 6
    c = synth.config4(n_maps=B, n_lo=100, n_hi=3000)
    # maps 1 and 4 receive no points
    clouds = list(c["clouds"])
    for b in (1, 4):
        clouds[b] = synth.Cloud(clouds[b].xyz[:0], clouds[b].T, clouds[b].rgb[:0], None, clouds[b].feat[:0])
    offsets = np.zeros(B + 1, np.int64)
    offsets[1:] = np.cumsum([cl.n for cl in clouds])
    layers = [dict(channels=3, rule=O.LATEST), dict(channels=16, rule=O.GAUSS, dtype=O.BF16)]
    g, _ = make_pair(c["W"], c["res"], layers, n_maps=B)
    xyz, rgb, feat, _, T = synth.concat_clouds(clouds)
    g.fuse_pointcloud_batch(offsets, torch.from_numpy(xyz).cuda(), T, _batch_sources(torch, rgb, feat))
    g.check()
    for b, cl in enumerate(clouds):
        o = O.OracleMap(O.Params(W=c["W"], res=c["res"], layers=[O.Layer(3, O.LATEST), O.Layer(16, O.GAUSS, store=O.BF16)]))
        o.fuse_points(cl.xyz, cl.T, [(cl.rgb, [0]), ((cl.feat,), [1])])
        compare_states(gpu_state(g, b), o, what=f"map {b}")


@pytest.mark.parametrize("radix_bits", [8, 9])
def test_batched_full_size_equals_per_map_oracle(torch, radix_bits):
    """The bench's own batched workload at full size -- 512 maps of 200 x 200, 10.85 M points
    (log-uniform 5k-60k per map), RGB average + 16-d BF16 Gaussian features, 25-bit keys -- in
    one batched call with 3 or 4 radix passes; every map compared with its own oracle map
    (integers bit-exact, floats at 1e-5, BF16 at one storage ulp)."""
    B = 512
    c = synth.config4(n_maps=B)
    xyz, rgb, feat, _, T = synth.concat_clouds(c["clouds"])
    assert int(c["offsets"][-1]) > 10_000_000
    layers = [dict(channels=3, rule=O.LATEST), dict(channels=16, rule=O.GAUSS, dtype=O.BF16)]
    g, _ = make_pair(c["W"], c["res"], layers, n_maps=B, max_points=int(c["offsets"][-1]) + 4096)
    g.set_tuning(radix_bits, 4, 1 if radix_bits == 8 else 0)  # both fuse kernels at full size
    assert g.get_tuning()["passes"] == (4 if radix_bits == 8 else 3)
    g.fuse_pointcloud_batch(c["offsets"], torch.from_numpy(xyz).cuda(), T, _batch_sources(torch, rgb, feat))
    g.check()
    for b, cl in enumerate(c["clouds"]):
        o = O.OracleMap(O.Params(W=c["W"], res=c["res"],
                                 layers=[O.Layer(3, O.LATEST), O.Layer(16, O.GAUSS, store=O.BF16)]))
        o.fuse_points(cl.xyz, cl.T, [(cl.rgb, [0]), ((cl.feat,), [1])])
        compare_states(gpu_state(g, b), o, what=f"map {b}")
