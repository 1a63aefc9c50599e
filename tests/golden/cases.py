"""Inputs of the stored-value fixtures in this folder: seeded point clouds, a move and a camera
image for a 12 x 12 map at 0.5 m. Input generation only (no fusion arithmetic); the oracle
(make_golden.py) and the library (tests/test_golden.py) consume the same arrays."""
import numpy as np

W, RES = 12, 0.5


def sensor_pose(t):
    T = np.eye(4)
    T[:3, 3] = t
    return T


def cloud(seed, n, n_outliers, t):
    """Points on a smooth surface seen from a sensor at world position t (no rotation), with
    colours, 4-class probabilities and 3-d features; the last n_outliers points are lifted 2 m."""
    rng = np.random.default_rng(seed)
    xy = rng.uniform(-2.8, 2.8, size=(n, 2)) + np.asarray(t[:2])
    z = 0.3 * np.sin(xy[:, 0]) + 0.2 * np.cos(xy[:, 1]) + rng.normal(0.0, 0.01, size=n)
    z[n - n_outliers:] += 2.0
    world = np.column_stack([xy, z])
    xyz = (world - np.asarray(t)).astype(np.float32)
    rgb = rng.integers(0, 256, size=(n, 3), dtype=np.uint8)
    p = rng.random((n, 4)).astype(np.float32) + np.float32(0.05)
    probs = (p / p.sum(axis=1, keepdims=True)).astype(np.float32)
    feat = rng.normal(0.0, 1.0, size=(n, 3)).astype(np.float32)
    return xyz, rgb, probs, feat, sensor_pose(t)


def camera(seed):
    """A 32 x 24 camera 2 m up at x = -3 m looking along +x, 26.6 degrees down (optical frame:
    x right, y down, z forward), with a 3-d feature image and a 4-class segmentation image."""
    f = np.array([1.0, 0.0, -0.5]) / np.sqrt(1.25)
    r = np.array([0.0, -1.0, 0.0])
    d = np.cross(f, r)
    T = np.eye(4)
    T[:3, 0], T[:3, 1], T[:3, 2] = r, d, f
    T[:3, 3] = (-3.0, 0.0, 2.0)
    H, Wi = 24, 32
    K = np.array([20.0, 20.0, 16.0, 12.0])
    rng = np.random.default_rng(seed)
    feat = rng.normal(0.0, 1.0, size=(H * Wi, 3)).astype(np.float32)
    s = rng.random((H * Wi, 4)).astype(np.float32) + np.float32(0.05)
    seg = (s / s.sum(axis=1, keepdims=True)).astype(np.float32)
    return H, Wi, K, T, feat, seg


STEPS = [("points", dict(seed=1, n=400, n_outliers=0, t=(0.0, 0.0, 1.0))),
         ("move", dict(xy=(1.0, 0.5))),
         ("points", dict(seed=2, n=400, n_outliers=20, t=(1.0, 0.5, 1.0))),
         ("image", dict(seed=3))]
