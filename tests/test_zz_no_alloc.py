"""The allocation-free height fuse (mem_fuse_pointcloud_noalloc) against the oracle and against
the regular map object, over several calls in a row.

It exists for callers that cannot call cudaMalloc (another framework owns the device memory
pool, or a real-time loop forbids allocation after start-up): they hand in their own layer
buffers and the library works in a fixed device array instead of allocating scratch. This
file is collected last so that a failure here never hides another test's result."""
import numpy as np
import pytest

import oracle as O
from paper_2309_16818_gb300 import synth

from helpers import REL, close

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _buffers(torch, W):
    h = torch.zeros(W * W, dtype=torch.float32, device="cuda")
    var = torch.zeros_like(h)
    valid = torch.zeros(W * W, dtype=torch.int32, device="cuda")
    return h, var, valid, torch.zeros_like(valid), torch.zeros_like(valid)


def _compare(what, h, var, valid, n_acc, n_rej, rv, rh, rvar, racc, rrej):
    gv = valid.cpu().numpy().astype(np.int64)
    assert np.array_equal(gv, rv.astype(np.int64)), f"{what}: valid"
    assert np.array_equal(n_acc.cpu().numpy().view(np.uint32), racc.astype(np.uint32)), f"{what}: n_acc"
    assert np.array_equal(n_rej.cpu().numpy().view(np.uint32), rrej.astype(np.uint32)), f"{what}: n_rej"
    v = rv == 1
    assert not close(h.cpu().numpy()[v], rh[v], 1.0, REL).any(), f"{what}: height"
    assert not close(var.cpu().numpy()[v], rvar[v], 0.0, REL).any(), f"{what}: variance"


@pytest.mark.parametrize("time_var,outlier_var", [(0.0, 0.0), (1e-4, 0.01)])
def test_noalloc_matches_oracle_call_by_call(torch, time_var, outlier_var):
    """Scan, empty cloud, scan: each call starts from the oracle's state copied into the
    caller's buffers, then every cell is compared (integers exactly, floats at 1e-5)."""
    from paper_2309_16818_gb300 import mem as M
    c = synth.config2(n_poses=2, scale=0.5)
    W, res = c["W"], c["res"]
    o = O.OracleMap(O.Params(W=W, res=res, time_var=time_var, outlier_var=outlier_var))
    bufs = _buffers(torch, W)
    h, var, valid, n_acc, n_rej = bufs
    calls = [c["scans"][0], "empty", c["scans"][1]]
    for k, s in enumerate(calls):
        h.copy_(torch.from_numpy(o.h.astype(np.float32)))
        var.copy_(torch.from_numpy(o.var.astype(np.float32)))
        valid.copy_(torch.from_numpy(o.valid.astype(np.int32)))
        n_acc.copy_(torch.from_numpy(o.n_acc.view(np.int32)))
        n_rej.copy_(torch.from_numpy(o.n_rej.view(np.int32)))
        if isinstance(s, str):
            xyz_np, T = np.zeros((0, 3), np.float32), c["scans"][0].T
        else:
            xyz_np, T = s.xyz, s.T
        assert xyz_np.shape[0] <= M.NOALLOC_MAX_POINTS
        o.fuse_points(xyz_np, T)
        M.fuse_pointcloud_noalloc(W, res, torch.from_numpy(np.ascontiguousarray(xyz_np)).cuda(), T,
                                  *bufs, time_var=time_var, outlier_var=outlier_var)
        M.noalloc_check()
        _compare(f"call {k}", *bufs, o.valid, o.h, o.var, o.n_acc, o.n_rej)
    assert o.valid.sum() > 1000 and int(o.n_rej.sum()) > 0


def test_noalloc_matches_map_object_on_two_calls(torch):
    """Two calls in a row without resetting anything, against the map object's entry point
    (mem_fuse_pointcloud) fed the same clouds, with time and outlier variance on."""
    from paper_2309_16818_gb300 import mem as M
    c = synth.config2(n_poses=2, scale=0.5)
    W, res = c["W"], c["res"]
    kw = dict(time_var=1e-4, outlier_var=0.01)
    ref = M.Map(W, res, [], **kw)
    bufs = _buffers(torch, W)
    for k, s in enumerate(c["scans"]):
        xyz = torch.from_numpy(s.xyz).cuda()
        ref.fuse_pointcloud(xyz, s.T)
        M.fuse_pointcloud_noalloc(W, res, xyz, s.T, *bufs, **kw)
        M.noalloc_check()
        ref.check()
        r = [ref.get_layer(L).cpu().numpy() for L in
             (M.LAYER_VALID, M.LAYER_HEIGHT, M.LAYER_VARIANCE, M.LAYER_NACC, M.LAYER_NREJ)]
        assert r[0].sum() > 1000
        _compare(f"call {k}", *bufs, r[0], r[1].astype(np.float64), r[2].astype(np.float64),
                 r[3].view(np.uint32), r[4].view(np.uint32))
    assert int(bufs[4].sum()) > 0


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
    M.noalloc_check()
