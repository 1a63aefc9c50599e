"""CUDA point-cloud path (transform, radix binning, height update, fusion rules, move)
against the oracle, element by element, through the C ABI."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2309_16818_gb300 import synth

from helpers import (cloud_sources_gpu, cloud_sources_np, compare_states, cuda_xyz, gpu_state,
                     make_pair, multimodal_layers, upload_state)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def test_config1_height_and_colour(torch):
    c = synth.config1()
    cl = c["cloud"]
    layers = [dict(channels=3, rule=O.LATEST)]
    g, o = make_pair(c["W"], c["res"], layers)
    o.fuse_points(cl.xyz, cl.T, [(cl.rgb, [0])])
    g.fuse_pointcloud(cuda_xyz(cl), cl.T, [(torch.from_numpy(cl.rgb).cuda(), [0])])
    g.check()
    gs = gpu_state(g)
    assert o.valid.sum() > 10000
    compare_states(gs, o, what="config 1")


@pytest.mark.parametrize("radix_bits,bps,fuse_kernel", [(8, 4, 0), (9, 1, 1), (10, 2, 0), (9, 8, 1), (9, 4, 0)])
def test_multimodal_scan_sequence(torch, radix_bits, bps, fuse_kernel):
    """Several poses of the multi-modal workload (reduced sensors), each step starting both
    sides from the same (oracle) state: move, then fuse, then compare. Both fuse kernels
    (register sums, shared-memory column walks) under several sort schedules."""
    c = synth.config2(n_poses=3, scale=0.25)
    g, o = make_pair(c["W"], c["res"], multimodal_layers(), max_points=1 << 16)
    g.set_tuning(radix_bits, bps, fuse_kernel)
    assert g.get_tuning()["fuse_kernel"] == fuse_kernel
    for k, scan in enumerate(c["scans"]):
        upload_state(g, o)
        xy = c["poses"][k][:2]
        o.move(xy)
        g.move(xy)
        assert g.origin() == o.origin
        o.fuse_points(scan.xyz, scan.T, cloud_sources_np(scan))
        g.fuse_pointcloud(cuda_xyz(scan), scan.T, cloud_sources_gpu(scan))
        g.check()
        compare_states(gpu_state(g), o, what=f"pose {k}")
    assert o.valid.sum() > 2000 and o.n_rej.sum() > 0


@pytest.mark.parametrize("order", ["pair_in_round", "pair_after_its_channels"])
def test_columns_over_several_rounds(torch, order):
    """More summed columns than one round holds (4 height sums + 3 colour + 24 features +
    20 classes + the arg-max pair = 53): the tile kernel takes them in rounds. With the
    features first, the class source's channels begin in the first round and its arg-max pair
    falls in the second, which recomputes the per-point arg-max there."""
    c = synth.config2(n_poses=2, scale=0.25)
    layers = [dict(channels=3, rule=O.LATEST), dict(channels=20, rule=O.DIRICHLET, alpha0=1.0),
              dict(channels=20, rule=O.CLASSMAX), dict(channels=24, rule=O.GAUSS, var_meas=0.3),
              dict(channels=24, rule=O.EXPAVG, w=0.2)]
    g, o = make_pair(c["W"], c["res"], layers, max_points=1 << 16)
    rng = np.random.default_rng(11)
    for k, scan in enumerate(c["scans"]):
        feat = rng.normal(0.0, 1.0, (scan.n, 24)).astype(np.float32)
        src_np = [(scan.rgb, [0]), (scan.probs, [1, 2]), (feat, [3, 4])]
        if order == "pair_after_its_channels":
            src_np = [src_np[0], src_np[2], src_np[1]]
        src_gpu = [(torch.from_numpy(np.ascontiguousarray(a)).cuda(), ls) for a, ls in src_np]
        upload_state(g, o)
        o.fuse_points(scan.xyz, scan.T, src_np)
        g.fuse_pointcloud(cuda_xyz(scan), scan.T, src_gpu)
        g.check()
        compare_states(gpu_state(g), o, what=f"{order} pose {k}")


def test_full_size_multimodal_pose(torch):
    """One full-size pose (128-beam LiDAR + 640x480 depth camera, 500x500 map), all cells."""
    c = synth.config2(n_poses=2, scale=1.0)
    g, o = make_pair(c["W"], c["res"], multimodal_layers())
    for k, scan in enumerate(c["scans"]):
        upload_state(g, o)
        o.move(c["poses"][k][:2])
        g.move(c["poses"][k][:2])
        o.fuse_points(scan.xyz, scan.T, cloud_sources_np(scan))
        g.fuse_pointcloud(cuda_xyz(scan), scan.T, cloud_sources_gpu(scan))
        g.check()
        compare_states(gpu_state(g), o, what=f"full pose {k}")


def test_free_running_sequence_with_moves(torch):
    """The CUDA map runs on its own over 4 poses (no state upload); integer results must match
    except in cells where a gate decision sits within 1e-3 of its threshold."""
    c = synth.config2(n_poses=4, scale=0.25)
    g, o = make_pair(c["W"], c["res"], multimodal_layers())
    W = c["W"]
    near_cells = np.zeros(W * W, bool)
    for k, scan in enumerate(c["scans"]):
        o0 = o.origin
        o.move(c["poses"][k][:2])
        g.move(c["poses"][k][:2])
        # the mask moves with the map: new cell (ix, iy) was old (ix + sx, iy + sy)
        sx = round((o.origin[0] - o0[0]) / c["res"])
        sy = round((o.origin[1] - o0[1]) / c["res"])
        old = near_cells.reshape(W, W)
        new = np.zeros_like(old)
        ys, xs = np.mgrid[0:W, 0:W]
        ok = (xs + sx >= 0) & (xs + sx < W) & (ys + sy >= 0) & (ys + sy < W)
        new[ok] = old[(ys + sy)[ok], (xs + sx)[ok]]
        near_cells = new.ravel()
        r = o.fuse_points(scan.xyz, scan.T, cloud_sources_np(scan), want_cells=True, want_near=True)
        near_cells[r["cells"][r["near"].astype(bool)]] = True
        g.fuse_pointcloud(cuda_xyz(scan), scan.T, cloud_sources_gpu(scan))
    g.check()
    gs = gpu_state(g)
    keep = ~near_cells
    assert keep.sum() > 0.99 * keep.size
    compare_states(gs, o, mask=keep, what="free running", )


def test_deterministic_rerun(torch):
    c = synth.config2(n_poses=1, scale=0.5)
    scan = c["scans"][0]
    outs = []
    for _ in range(2):
        g, _o = make_pair(c["W"], c["res"], multimodal_layers())
        for _k in range(2):
            g.fuse_pointcloud(cuda_xyz(scan), scan.T, cloud_sources_gpu(scan))
        s = gpu_state(g)
        outs.append(np.concatenate([s["h"], s["var"]] + [x.ravel() for x in s["layers"]]))
    assert np.array_equal(outs[0].view(np.uint64), outs[1].view(np.uint64))


def test_edge_cases(torch):
    W, res = 50, 0.1   # W not a multiple of the 16-cell tiles
    layers = [dict(channels=3, rule=O.LATEST), dict(channels=5, rule=O.GAUSS, var_meas=0.3)]
    g, o = make_pair(W, res, layers)
    T = np.eye(4)
    T[2, 3] = 1.0
    # empty cloud
    g.fuse_pointcloud(torch.empty((0, 3), device="cuda"), T, [])
    # all points dropped: NaN, out of range, out of map
    bad = np.array([[np.nan, 0, -1], [0, np.inf, -1], [0.01, 0.0, 0.0], [10.0, 0.0, -1.0],
                    [0.0, -2.51, -1.0]], np.float32)
    rgb = np.zeros((5, 3), np.uint8)
    f = np.zeros((5, 5), np.float32)
    o.fuse_points(bad, T, [(rgb, [0]), (f, [1])])
    g.fuse_pointcloud(torch.from_numpy(bad).cuda(), T,
                      [(torch.from_numpy(rgb).cuda(), [0]), (torch.from_numpy(f).cuda(), [1])])
    # one long run: 5000 points in one cell, points exactly on cell edges, ragged tail
    rng = np.random.default_rng(0)
    one = np.tile(np.array([[0.05, 0.05, -1.0]], np.float32), (5000, 1))
    one[:, 2] += rng.normal(0, 0.01, 5000).astype(np.float32)
    edges = (rng.integers(-25, 25, size=(3001, 2)) * 0.1).astype(np.float32)
    edges = np.column_stack([edges, np.full(3001, -1.0, np.float32)])
    pts = np.concatenate([one, edges, rng.uniform(-3, 3, size=(777, 3)).astype(np.float32)])
    rgb = rng.integers(0, 256, size=(len(pts), 3), dtype=np.uint8)
    f = rng.normal(size=(len(pts), 5)).astype(np.float32)
    upload_state(g, o)
    o.fuse_points(pts, T, [(rgb, [0]), (f, [1])])
    g.fuse_pointcloud(torch.from_numpy(pts).cuda(), T,
                      [(torch.from_numpy(rgb).cuda(), [0]), (torch.from_numpy(f).cuda(), [1])])
    g.check()
    compare_states(gpu_state(g), o, what="edge cases")
    assert o.n_acc.max() + o.n_rej.max() >= 5000


def test_time_and_outlier_variance(torch):
    c = synth.config2(n_poses=2, scale=0.2)
    g, o = make_pair(c["W"], c["res"], multimodal_layers(), outlier_var=0.01, time_var=1e-4)
    for k, scan in enumerate(c["scans"]):
        upload_state(g, o)
        o.fuse_points(scan.xyz, scan.T, cloud_sources_np(scan))
        g.fuse_pointcloud(cuda_xyz(scan), scan.T, cloud_sources_gpu(scan))
        compare_states(gpu_state(g), o, what=f"variance growth pose {k}")


def test_time_variance_on_empty_clouds_and_untouched_cells(torch):
    """time_var ages every valid cell once per call, touched or not: a full scan, an empty
    cloud (device and host-buffer entry points), a few points that leave almost every valid
    cell untouched, and an empty batched call over three maps; each call starts both sides
    from the oracle's state and compares every cell."""
    c = synth.config2(n_poses=2, scale=0.2)
    g, o = make_pair(c["W"], c["res"], multimodal_layers(), outlier_var=0.01, time_var=1e-4)
    s0, s1 = c["scans"]
    few = slice(0, 40)
    empty_np = np.zeros((0, 3), np.float32)
    steps = [("scan", s0.xyz, s0.T, cloud_sources_np(s0), False),
             ("empty", empty_np, s0.T, [], False),
             ("empty host", empty_np, s0.T, [], True),
             ("few points", s1.xyz[few], s1.T, [(s1.rgb[few], [0]), (s1.probs[few], [1, 2, 3])], False)]
    for what, xyz, T, src, host in steps:
        upload_state(g, o)
        o.fuse_points(xyz, T, src)
        if host:
            g.fuse_pointcloud_host(torch.from_numpy(np.ascontiguousarray(xyz)).pin_memory(), T,
                                   [(torch.from_numpy(np.ascontiguousarray(a)).pin_memory(), L) for a, L in src])
        else:
            g.fuse_pointcloud(torch.from_numpy(np.ascontiguousarray(xyz)).cuda(), T,
                              [(torch.from_numpy(np.ascontiguousarray(a)).cuda(), L) for a, L in src])
        g.check()
        compare_states(gpu_state(g), o, what=what)
    assert o.valid.sum() > 1000
    # batched: three maps, one cloud for map 0 then an all-empty call
    B = 3
    gb, _ = make_pair(c["W"], c["res"], [], n_maps=B, time_var=1e-4)
    ob = [O.OracleMap(O.Params(W=c["W"], res=c["res"], time_var=1e-4)) for _ in range(B)]
    for rnd in range(2):
        n0 = s0.n if rnd == 0 else 0
        offsets = np.array([0, n0, n0, n0], np.int64)
        xyz = s0.xyz[:n0]
        ob[0].fuse_points(xyz, s0.T)
        for b in (1, 2):
            ob[b].fuse_points(empty_np, s0.T)
        gb.fuse_pointcloud_batch(offsets, torch.from_numpy(np.ascontiguousarray(xyz)).cuda(),
                                 np.stack([s0.T] * B))
        gb.check()
        for b in range(B):
            compare_states(gpu_state(gb, b), ob[b], what=f"batched round {rnd} map {b}")
    assert ob[0].valid.sum() > 1000


def test_bf16_and_f16_feature_storage(torch):
    """Gaussian feature layers stored in BF16 / F16 / F32, fed BF16 point features."""
    c = synth.config4(n_maps=1, n_lo=40_000, n_hi=40_001)
    cl = c["clouds"][0]
    layers = [dict(channels=16, rule=O.GAUSS, var_meas=1.0, dtype=O.BF16),
              dict(channels=16, rule=O.GAUSS, var_meas=1.0, dtype=O.F16),
              dict(channels=16, rule=O.GAUSS, var_meas=1.0, dtype=O.F32),
              dict(channels=3, rule=O.LATEST)]
    g, o = make_pair(c["W"], c["res"], layers)
    feat_t = torch.from_numpy(cl.feat.view(np.int16)).cuda().view(torch.bfloat16)
    for k in range(3):
        upload_state(g, o)
        o.fuse_points(cl.xyz, cl.T, [((cl.feat,), [0, 1, 2]), (cl.rgb, [3])])
        g.fuse_pointcloud(cuda_xyz(cl), cl.T, [(feat_t, [0, 1, 2]), (torch.from_numpy(cl.rgb).cuda(), [3])])
        compare_states(gpu_state(g), o, what=f"bf16 scan {k}", bf16_rel=2.0 ** -7)


def test_graph_replay_on_a_side_stream_equals_eager(torch):
    """On a stream of its own the point path is captured once and replayed from a CUDA graph;
    the layers must be bit-identical to eager launches on the default stream, pose after pose."""
    from paper_2309_16818_gb300 import mem as M
    c = synth.config2(n_poses=3, scale=0.25)
    layers = [M.Layer(3, M.LATEST), M.Layer(20, M.DIRICHLET), M.Layer(20, M.CLASSMAX),
              M.Layer(20, M.EXPAVG, w=0.1)]
    eager = M.Map(c["W"], c["res"], layers, max_points=1 << 16)
    replay = M.Map(c["W"], c["res"], layers, max_points=1 << 16)
    side = torch.cuda.Stream()
    for k, scan in enumerate(c["scans"]):
        srcs = [(torch.from_numpy(scan.rgb).cuda(), [0]), (torch.from_numpy(scan.probs).cuda(), [1, 2, 3])]
        xyz = cuda_xyz(scan)
        eager.move(c["poses"][k][:2])
        eager.fuse_pointcloud(xyz, scan.T, srcs)
        torch.cuda.synchronize()
        with torch.cuda.stream(side):
            replay.move(c["poses"][k][:2])
            replay.fuse_pointcloud(xyz, scan.T, srcs)
        side.synchronize()
        eager.check()
        replay.check()
        for layer in (M.LAYER_HEIGHT, M.LAYER_VARIANCE, M.LAYER_VALID, M.LAYER_NACC, M.LAYER_NREJ, 0, 1, 2, 3):
            a = eager.get_layer(layer).cpu().numpy()
            b = replay.get_layer(layer).cpu().numpy()
            assert np.array_equal(a.view(np.uint8), b.view(np.uint8)), (k, layer)


@pytest.mark.parametrize("fuse_kernel", [0, 1])
def test_run_to_run_identical_with_moves(torch, fuse_kernel):
    """Every sum is taken in a fixed order, so the same pose sequence (with map moves, which
    wrap the ring-buffer keys) on fresh maps must give bit-identical layers, repeatedly."""
    from paper_2309_16818_gb300 import mem as M
    c = synth.config2(n_poses=4, scale=1.0)
    layers = [M.Layer(3, M.LATEST), M.Layer(20, M.DIRICHLET), M.Layer(20, M.CLASSMAX),
              M.Layer(20, M.EXPAVG, w=0.1)]
    data = [(cuda_xyz(s), torch.from_numpy(s.rgb).cuda(), torch.from_numpy(s.probs).cuda()) for s in c["scans"]]
    ref = None
    for trial in range(4):
        g = M.Map(c["W"], c["res"], layers, max_points=1 << 20)
        g.set_tuning(9, 8 if trial % 2 else 4, fuse_kernel)
        out = []
        for k, s in enumerate(c["scans"]):
            g.move(c["poses"][k][:2])
            x, r, p = data[k]
            g.fuse_pointcloud(x, s.T, [(r, [0]), (p, [1, 2, 3])])
            g.check()
            valid = g.get_layer(M.LAYER_VALID).cpu().numpy().astype(bool)
            for lay in (M.LAYER_HEIGHT, M.LAYER_VARIANCE, M.LAYER_NACC, M.LAYER_NREJ):
                out.append(np.where(valid, g.get_layer(lay).cpu().numpy(), 0).tobytes())
            out.append(valid.tobytes())
            for lay in (0, 1, 2, 3):
                out.append(g.get_layer(lay).cpu().numpy().tobytes())
        if ref is None:
            ref = out
        else:
            for j, (a, b) in enumerate(zip(ref, out)):
                assert a == b, (trial, j)


def test_host_buffer_fuse_equals_device_fuse(torch):
    """mem_fuse_pointcloud_host (pinned host inputs, library staging buffers used in turn on a
    copy stream) gives the same layers as the device-pointer call, pose after pose."""
    from paper_2309_16818_gb300 import mem as M
    c = synth.config2(n_poses=4, scale=0.5)
    layers = [M.Layer(3, M.LATEST), M.Layer(20, M.DIRICHLET), M.Layer(20, M.CLASSMAX),
              M.Layer(20, M.EXPAVG, w=0.1)]
    dev = M.Map(c["W"], c["res"], layers, max_points=1 << 20)
    host = M.Map(c["W"], c["res"], layers, max_points=1 << 20)
    side = torch.cuda.Stream()
    pinned = []
    for k, s in enumerate(c["scans"]):
        hx = torch.from_numpy(s.xyz).pin_memory()
        hr = torch.from_numpy(s.rgb).pin_memory()
        hp = torch.from_numpy(s.probs).pin_memory()
        pinned.append((hx, hr, hp))  # alive until the stream is synchronized
        dev.move(c["poses"][k][:2])
        dev.fuse_pointcloud(hx.cuda(), s.T, [(hr.cuda(), [0]), (hp.cuda(), [1, 2, 3])])
        with torch.cuda.stream(side):
            host.move(c["poses"][k][:2])
            host.fuse_pointcloud_host(hx, s.T, [(hr, [0]), (hp, [1, 2, 3])])
    torch.cuda.synchronize()
    side.synchronize()
    dev.check()
    host.check()
    for lay in (M.LAYER_HEIGHT, M.LAYER_VARIANCE, M.LAYER_VALID, M.LAYER_NACC, M.LAYER_NREJ, 0, 1, 2, 3):
        a = dev.get_layer(lay).cpu().numpy()
        b = host.get_layer(lay).cpu().numpy()
        assert np.array_equal(a.view(np.uint8), b.view(np.uint8)), lay


def test_injected_sort_wait_timeout_reports_and_changes_nothing(torch):
    """Fault injection from the host: the radix sort's look-back waits are made to run out. The
    call must come back (bounded waits, no trap, no hang), mem_check must report MEM_ERR_TIMEOUT,
    the map must be left exactly as before the call, and after the fault is cleared the same call
    must give the oracle's result."""
    import time
    from paper_2309_16818_gb300 import mem as M
    c = synth.config1()
    cl = c["cloud"]
    layers = [dict(channels=3, rule=O.LATEST)]
    g, o = make_pair(c["W"], c["res"], layers)
    src = [(torch.from_numpy(cl.rgb).cuda(), [0])]
    o.fuse_points(cl.xyz, cl.T, [(cl.rgb, [0])])
    g.fuse_pointcloud(cuda_xyz(cl), cl.T, src)
    g.check()
    before = gpu_state(g)
    g.inject_fault(M.FAULT_SORT_WAIT)
    t0 = time.time()
    g.fuse_pointcloud(cuda_xyz(cl), cl.T, src)
    with pytest.raises(M.MemError) as e:
        g.check()
    assert e.value.status == M.ERR_TIMEOUT
    assert time.time() - t0 < 60
    after = gpu_state(g)
    for k in ("h", "var", "valid", "n_acc", "n_rej"):
        assert np.array_equal(after[k], before[k]), k
    assert np.array_equal(after["layers"][0], before["layers"][0])
    g.inject_fault(M.FAULT_NONE)
    g.check()  # the error word was cleared by the failed check
    o.fuse_points(cl.xyz, cl.T, [(cl.rgb, [0])])
    g.fuse_pointcloud(cuda_xyz(cl), cl.T, src)
    g.check()
    compare_states(gpu_state(g), o, what="after the injected fault")
