"""The seeded input generators follow the recipe the workloads are described by: point counts
per pose, misses kept as NaN, probability rows that sum to one, the log-uniform cloud sizes of the
batched workload, the hidden fraction of the inpainting crops, the terrain formula and
round-to-nearest-even bfloat16 conversion. CPU only."""
import math

import numpy as np
import pytest

from paper_2309_16818_gb300 import synth


def test_terrain_formula():
    t = synth.Terrain(phi=0.3, psi=1.1)
    for x, y in [(0.0, 0.0), (1.7, -2.2), (-3.1, 0.4)]:
        s = math.sin(2 * math.pi * (x * math.cos(0.3) + y * math.sin(0.3)) / 2.5 + 1.1)
        exp = 0.3 * math.sin(0.7 * x) * math.cos(0.5 * y) + 0.2 * (s > 0)
        assert float(t.height(x, y)) == pytest.approx(exp, abs=1e-15)


def test_multimodal_pose_shapes_and_payload():
    c = synth.config2(n_poses=1, scale=1.0)
    cl = c["scans"][0]
    n = 128 * 2048 + 640 * 480
    assert cl.xyz.shape == (n, 3) and cl.xyz.dtype == np.float32 and n == 569_344
    assert cl.rgb.shape == (n, 3) and cl.rgb.dtype == np.uint8
    assert cl.probs.shape == (n, 20) and cl.probs.dtype == np.float32
    np.testing.assert_allclose(cl.probs.astype(np.float64).sum(axis=1), 1.0, atol=1e-5)
    nan = ~np.isfinite(cl.xyz).all(axis=1)
    assert 0 < nan.sum() < n  # misses are kept, as NaN rows
    R = cl.T[:3, :3]
    np.testing.assert_allclose(R @ R.T, np.eye(3), atol=1e-12)
    assert c["W"] == 500 and c["res"] == 0.04


def test_batched_cloud_sizes_are_log_uniform_in_range():
    c = synth.config4(n_maps=12, n_lo=5_000, n_hi=60_000)
    sizes = np.diff(c["offsets"])
    assert np.all((sizes >= 5_000) & (sizes <= 60_000))
    assert c["offsets"][0] == 0 and c["offsets"][-1] == sum(cl.n for cl in c["clouds"])
    # the same draw as the generator: floor(exp(U(log lo, log hi))) from the map's own seed
    for b, n in enumerate(sizes):
        rng = np.random.default_rng(10_000 + b)
        assert n == int(math.floor(math.exp(rng.uniform(math.log(5_000), math.log(60_000)))))


def test_inpainting_crops_hide_the_stated_fraction():
    gt, kn = synth.inpaint_crops(4, size=48, seed=3, lo=0.15, hi=0.6)
    assert gt.shape == kn.shape == (4, 48, 48) and gt.dtype == np.float32 and kn.dtype == np.uint8
    hidden = 1.0 - kn.reshape(4, -1).mean(axis=1)
    assert np.all((hidden >= 0.15) & (hidden <= 0.6))


def test_dirichlet_rows_sum_to_one():
    p = synth.dirichlet_probs(np.random.default_rng(0), 1000, 20, 0.3)
    np.testing.assert_allclose(p.astype(np.float64).sum(axis=1), 1.0, atol=1e-5)
    assert p.min() >= 0.0


def test_bf16_conversion_rounds_to_nearest_even():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(1)
    a = np.concatenate([rng.normal(size=10_000).astype(np.float32) * np.float32(1e3),
                        np.array([1.0, -2.5, 0.0, 1e-40, 65504.0, 3.0e38], np.float32)])
    bits = synth.f32_to_bf16_bits(a)
    ref = torch.from_numpy(a).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    np.testing.assert_array_equal(bits, ref)
    back = synth.bf16_bits_to_f32(bits)
    np.testing.assert_array_equal(back, torch.from_numpy(a).to(torch.bfloat16).float().numpy())
