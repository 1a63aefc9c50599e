"""CUDA top-k class input (Sec. III-C: class probabilities given as the top k classes) against
the oracle, element by element, through the C ABI: point clouds (device and host buffers) and
camera images whose class rows are (class id, probability) pairs."""
import numpy as np
import pytest

import oracle as O
from paper_2309_16818_gb300 import synth

from helpers import compare_states, cuda_xyz, gpu_state, make_pair, multimodal_layers, upload_state

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.mark.parametrize("k,host", [(3, False), (1, False), (5, True)])
def test_topk_cloud_sequence(torch, k, host):
    """Multi-modal poses whose 20-class probabilities arrive as their top k classes, into the
    Dirichlet, class-max and exponential-average layers (colour average as before)."""
    from paper_2309_16818_gb300 import mem as M
    c = synth.config2(n_poses=3, scale=0.25)
    g, o = make_pair(c["W"], c["res"], multimodal_layers())
    for j, scan in enumerate(c["scans"]):
        pairs = synth.topk_pairs(scan.probs, k)
        upload_state(g, o)
        o.move(c["poses"][j][:2])
        g.move(c["poses"][j][:2])
        o.fuse_points(scan.xyz, scan.T, [(scan.rgb, [0]), (O.TopK(pairs, 20), [1, 2, 3])])
        if host:
            g.fuse_pointcloud_host(torch.from_numpy(scan.xyz).pin_memory(), scan.T,
                                   [(torch.from_numpy(scan.rgb).pin_memory(), [0]),
                                    (M.TopK(torch.from_numpy(pairs).pin_memory(), 20), [1, 2, 3])])
        else:
            g.fuse_pointcloud(cuda_xyz(scan), scan.T, [(torch.from_numpy(scan.rgb).cuda(), [0]),
                                                       (M.TopK(torch.from_numpy(pairs).cuda(), 20), [1, 2, 3])])
        g.check()
        compare_states(gpu_state(g), o, what=f"top-{k} pose {j}")
    assert o.valid.sum() > 2000


def test_topk_image(torch):
    """A camera's 20-class segmentation as top-2 pairs per pixel into Dirichlet + class max."""
    from paper_2309_16818_gb300 import mem as M
    c = synth.config2(n_poses=1, scale=0.25)
    layers = [dict(channels=20, rule=O.DIRICHLET), dict(channels=20, rule=O.CLASSMAX)]
    g, o = make_pair(c["W"], c["res"], layers)
    scan = c["scans"][0]
    o.move(c["poses"][0][:2])
    g.move(c["poses"][0][:2])
    o.fuse_points(scan.xyz, scan.T)
    g.fuse_pointcloud(cuda_xyz(scan), scan.T)
    cam = synth.cameras_around(5, c["poses"][0], c["terrain"], H=96, Wi=170, n_feat=4)[0]
    pairs = synth.topk_pairs(cam.seg.reshape(-1, 20), 2)
    upload_state(g, o)
    r = o.fuse_image(cam.H, cam.Wi, [(O.TopK(pairs, 20), [0, 1])], cam.K, cam.T)
    vis = torch.empty(c["W"] ** 2, dtype=torch.uint8, device="cuda")
    g.fuse_image(cam.H, cam.Wi, cam.K, cam.T,
                 [(M.TopK(torch.from_numpy(pairs.reshape(cam.H, cam.Wi, 4)).cuda(), 20), [0, 1])], vis=vis)
    g.check()
    assert r["n_visible"] > 100
    assert np.array_equal(vis.cpu().numpy(), r["vis"])
    compare_states(gpu_state(g), o, what="top-2 image")


def test_topk_arguments_checked_on_the_host(torch):
    from paper_2309_16818_gb300 import mem as M
    g = M.Map(16, 0.1, [M.Layer(5, M.DIRICHLET)])
    xyz = torch.zeros((4, 3), device="cuda")
    bad = torch.zeros((4, 40), dtype=torch.float32, device="cuda")   # 20 pairs > MEM_MAX_TOPK
    with pytest.raises(M.MemError) as ei:
        g.fuse_pointcloud(xyz, np.eye(4), [(M.TopK(bad, 5), [0])])
    assert ei.value.status == M.ERR_ARG
    with pytest.raises(M.MemError):
        g.fuse_pointcloud(xyz, np.eye(4), [(M.TopK(torch.zeros((4, 4), dtype=torch.float16, device="cuda"), 5), [0])])
