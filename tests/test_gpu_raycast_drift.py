"""CUDA drift compensation and ray-cast clean-up (Table I rows "drift compensation" and "height
update & ray cast") against the oracle, element by element, through the C ABI.

The synthetic poses are exact, so drift is injected: the sensor pose given to the fuse is
lifted by a few centimetres (an odometry error in z). Stale obstacles are injected too: random
valid cells of the state both sides start from are raised by half a metre, so the clean-up has
phantom obstacles to remove."""
import numpy as np
import pytest

import oracle as O
from paper_2309_16818_gb300 import synth

from helpers import (cloud_sources_gpu, cloud_sources_np, compare_states, cuda_xyz, gpu_state,
                     make_pair, multimodal_layers, upload_state)

pytestmark = pytest.mark.gpu

KW = dict(drift_alpha=1.0, drift_min_points=100, ray_cleanup=True, ray_margin=0.1)


@pytest.fixture(scope="module")
def torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def lifted(T, dz):
    T = np.array(T, dtype=np.float64)
    T[2, 3] += dz
    return T


def phantoms(o, rng, n):
    """Raise n random valid cells of the oracle state by 0.5 m (stale obstacles)."""
    idx = np.nonzero(o.valid)[0]
    pick = rng.choice(idx, size=min(n, len(idx)), replace=False)
    o.h[pick] += 0.5
    return pick


def check_drift(g, r, what, map_index=0):
    d = g.get_drift(map_index)
    assert d["drift_points"] == r["drift_points"], f"{what}: drift points {d} vs {r}"
    assert abs(d["drift"] - r["drift"]) <= 2.0 ** -23 * max(abs(r["drift"]), 1e-30), f"{what}: drift {d} vs {r}"
    return d


@pytest.mark.parametrize("scale", [0.25, 1.0])
def test_drift_and_cleanup_sequence(torch, scale):
    """Multi-modal poses (reduced and full-size sensors) with 0 / +4 / -3 cm of z drift and
    phantom obstacles; every step starts both sides from the oracle's state."""
    c = synth.config2(n_poses=3, scale=scale)
    g, o = make_pair(c["W"], c["res"], multimodal_layers(), **KW)
    rng = np.random.default_rng(3)
    cleared_total = 0
    for k, (scan, dz) in enumerate(zip(c["scans"], (0.0, 0.04, -0.03))):
        if k:
            phantoms(o, rng, 400)
        upload_state(g, o)
        xy = c["poses"][k][:2]
        o.move(xy)
        g.move(xy)
        T = lifted(scan.T, dz)
        r = o.fuse_points(scan.xyz, T, cloud_sources_np(scan))
        g.fuse_pointcloud(cuda_xyz(scan), T, cloud_sources_gpu(scan))
        g.check()
        d = check_drift(g, r, f"pose {k}")
        assert d["cleared"] == r["cleared"], f"pose {k}: cleared {d['cleared']} vs {r['cleared']}"
        compare_states(gpu_state(g), o, what=f"pose {k}")
        if k:  # the gate keeps only errors within its bound, so the shift has dz's sign, not its size
            assert r["drift"] * dz > 0 and abs(r["drift"]) < abs(dz) and r["drift_points"] > 1000
        cleared_total += r["cleared"]
    assert cleared_total > 50


def test_cleanup_only_and_drift_only(torch):
    """Each step alone (the other off) on the same scene."""
    c = synth.config2(n_poses=2, scale=0.25)
    rng = np.random.default_rng(4)
    for kw in (dict(ray_cleanup=True, ray_margin=0.05), dict(drift_alpha=0.5, drift_min_points=10)):
        g, o = make_pair(c["W"], c["res"], multimodal_layers(), **kw)
        for k, scan in enumerate(c["scans"]):
            if k:
                phantoms(o, rng, 300)
            upload_state(g, o)
            T = lifted(scan.T, 0.02 * k)
            r = o.fuse_points(scan.xyz, T, cloud_sources_np(scan))
            g.fuse_pointcloud(cuda_xyz(scan), T, cloud_sources_gpu(scan))
            g.check()
            d = check_drift(g, r, f"{kw} pose {k}")
            assert d["cleared"] == r["cleared"]
            compare_states(gpu_state(g), o, what=f"{kw} pose {k}")


def test_batched_maps_drift_per_map(torch):
    """Each map of a batched call takes its own mean error and shift; maps with too few
    points (or none) are not shifted."""
    B = 6
    c = synth.config4(n_maps=B, n_lo=50, n_hi=6000)
    clouds = list(c["clouds"])
    clouds[2] = synth.Cloud(clouds[2].xyz[:0], clouds[2].T, clouds[2].rgb[:0], None, clouds[2].feat[:0])
    offsets = np.zeros(B + 1, np.int64)
    offsets[1:] = np.cumsum([cl.n for cl in clouds])
    kw = dict(drift_alpha=1.0, drift_min_points=200, ray_cleanup=True, ray_margin=0.1)
    g, _ = make_pair(c["W"], c["res"], [dict(channels=3, rule=O.LATEST)], n_maps=B, **kw)
    oracles = [O.OracleMap(O.Params(W=c["W"], res=c["res"], layers=[O.Layer(3, O.LATEST)], **kw)) for _ in range(B)]
    xyz, rgb, _, _, _ = synth.concat_clouds(clouds)
    rng = np.random.default_rng(6)
    for rnd in range(2):
        Ts = np.stack([lifted(cl.T, 0.03 * rnd * (b % 3 - 1)) for b, cl in enumerate(clouds)])
        res = []
        for b, cl in enumerate(clouds):
            if rnd:
                phantoms(oracles[b], rng, 100)
                upload_state(g, oracles[b], map_index=b)
            res.append(oracles[b].fuse_points(cl.xyz, Ts[b], [(cl.rgb, [0])]))
        g.fuse_pointcloud_batch(offsets, torch.from_numpy(xyz).cuda(), Ts,
                                [(torch.from_numpy(rgb).cuda(), [0])])
        g.check()
        assert g.get_drift(0)["cleared"] == sum(r["cleared"] for r in res)
        for b in range(B):
            check_drift(g, res[b], f"round {rnd} map {b}", map_index=b)
            compare_states(gpu_state(g, b), oracles[b], what=f"round {rnd} map {b}")
    assert any(r["drift"] != 0.0 for r in res) and any(r["cleared"] > 0 for r in res)


def test_empty_cloud_reports_no_drift(torch):
    c = synth.config2(n_poses=1, scale=0.25)
    scan = c["scans"][0]
    g, o = make_pair(c["W"], c["res"], [], **KW)
    g.fuse_pointcloud(cuda_xyz(scan), lifted(scan.T, 0.05), [])
    g.fuse_pointcloud(torch.empty((0, 3), device="cuda"), scan.T, [])
    d = g.get_drift()
    assert d == dict(drift=0.0, drift_points=0, cleared=0)
