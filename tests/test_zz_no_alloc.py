"""The allocation-free height fuse (mem_fuse_pointcloud_noalloc) gives the same layers as the
regular map object, over two calls in a row.

It exists for callers that cannot call cudaMalloc (another framework owns the device memory
pool, or a real-time loop forbids allocation after start-up): they hand in their own layer
buffers and the library works in a fixed device array instead of allocating scratch. This
file is collected last so that a failure here never hides another test's result."""
import numpy as np
import pytest

from paper_2309_16818_gb300 import synth

from helpers import REL, close

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def test_noalloc_matches_map_object_on_two_calls(torch):
    from paper_2309_16818_gb300 import mem as M
    c = synth.config2(n_poses=2, scale=0.5)
    W, res = c["W"], c["res"]
    scans = c["scans"]
    assert max(s.n for s in scans) <= M.NOALLOC_MAX_POINTS
    ref = M.Map(W, res, [])
    dev = "cuda"
    h = torch.zeros(W * W, dtype=torch.float32, device=dev)
    var = torch.zeros_like(h)
    valid = torch.zeros(W * W, dtype=torch.int32, device=dev)
    n_acc = torch.zeros_like(valid)
    n_rej = torch.zeros_like(valid)
    for k, s in enumerate(scans):
        xyz = torch.from_numpy(s.xyz).to(dev)
        ref.fuse_pointcloud(xyz, s.T)
        M.fuse_pointcloud_noalloc(W, res, xyz, s.T, h, var, valid, n_acc, n_rej, origin=(0.0, 0.0))
        torch.cuda.synchronize()
        rv = ref.get_layer(M.LAYER_VALID).cpu().numpy().astype(np.int64)
        gv = valid.cpu().numpy().astype(np.int64)
        assert rv.sum() > 1000
        assert np.array_equal(gv, rv), f"call {k}: valid"
        for lay, mine, scale in ((M.LAYER_NACC, n_acc, None), (M.LAYER_NREJ, n_rej, None),
                                 (M.LAYER_HEIGHT, h, 1.0), (M.LAYER_VARIANCE, var, 0.0)):
            r = ref.get_layer(lay).cpu().numpy()
            g = mine.cpu().numpy()
            if scale is None:
                assert np.array_equal(g.view(np.uint32), r.view(np.uint32)), f"call {k}: counts {lay}"
            else:
                v = rv == 1
                assert not close(g[v], r[v], scale, REL).any(), f"call {k}: layer {lay}"
    assert int(n_rej.sum()) > 0


def test_noalloc_rejects_too_many_points(torch):
    from paper_2309_16818_gb300 import mem as M
    W = 8
    n = M.NOALLOC_MAX_POINTS + 1
    xyz = torch.zeros((n, 3), dtype=torch.float32, device="cuda")
    buf = [torch.zeros(W * W, dtype=t, device="cuda") for t in
           (torch.float32, torch.float32, torch.int32, torch.int32, torch.int32)]
    with pytest.raises(M.MemError) as ei:
        M.fuse_pointcloud_noalloc(W, 0.5, xyz, np.eye(4), *buf)
    assert ei.value.status == M.ERR_ARG and "limit" in str(ei.value)
