"""Seeded synthetic inputs for the map-update path.

This module simulates sensors over procedural terrain; it holds none of the
mapping method's arithmetic (no binning, no fusion, no projection of cells).
Both the CUDA path and the CPU oracle are fed from here, so everything is
returned as plain numpy arrays (float32 points in the SENSOR frame, uint8
colours, float32 class probabilities, bfloat16 features as uint16 bit
patterns) plus float64 4x4 poses ``T_map_sensor`` (sensor -> world).

The paper's own sensor data (ZED 2i stereo clouds, VLP-16 scans, RealSense
depth clouds, ANYmal camera images; Table II) is not available, so these
generators stand in for it with the same shapes:

* terrain  z = 0.3 sin(0.7x) cos(0.5y) + 0.2 [sin(2 pi (x cos phi + y sin phi)/2.5 + psi) > 0]
* range noise sigma = 0.01 + 0.002 r along each ray
* LiDAR: B beams x A azimuths, elevations uniform in [-25, +15] deg, 0.5..40 m,
  rays cast against the terrain, misses become NaN (and stay in the cloud)
* depth camera: 640x480, fx=fy=385, 0.3..6 m, pitched 30 deg down
* camera images: smooth Gaussian random fields (sigma = 8 px), unit variance
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

# ----------------------------------------------------------------------------
# terrain


@dataclass(frozen=True)
class Terrain:
    phi: float
    psi: float

    @staticmethod
    def from_seed(seed: int) -> "Terrain":
        rng = np.random.default_rng(seed)
        return Terrain(float(rng.uniform(0, 2 * math.pi)), float(rng.uniform(0, 2 * math.pi)))

    def height(self, x, y):
        x = np.asarray(x, dtype=np.float64)
        y = np.asarray(y, dtype=np.float64)
        base = 0.3 * np.sin(0.7 * x) * np.cos(0.5 * y)
        s = np.sin(2 * math.pi * (x * math.cos(self.phi) + y * math.sin(self.phi)) / 2.5 + self.psi)
        return base + 0.2 * (s > 0)


def rot_z(yaw: float) -> np.ndarray:
    c, s = math.cos(yaw), math.sin(yaw)
    return np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])


def rot_y(a: float) -> np.ndarray:
    c, s = math.cos(a), math.sin(a)
    return np.array([[c, 0.0, s], [0.0, 1.0, 0.0], [-s, 0.0, c]])


def pose(R: np.ndarray, t) -> np.ndarray:
    T = np.eye(4)
    T[:3, :3] = R
    T[:3, 3] = np.asarray(t, dtype=np.float64)
    return T


# optical camera frame (x right, y down, z forward) expressed in a body frame
# (x forward, y left, z up)
R_BODY_OPTICAL = np.array([[0.0, 0.0, 1.0], [-1.0, 0.0, 0.0], [0.0, -1.0, 0.0]])


def to_sensor_frame(T_ws: np.ndarray, p_w: np.ndarray) -> np.ndarray:
    """World points -> sensor frame (float32); NaN rows stay NaN."""
    R = T_ws[:3, :3]
    t = T_ws[:3, 3]
    return ((p_w - t) @ R).astype(np.float32)


# ----------------------------------------------------------------------------
# ray casting against the terrain (simulation of the sensors, float64)


def raycast(terrain: Terrain, origin, dirs, tmin: float, tmax: float, n_coarse: int = 96,
            n_bisect: int = 26) -> np.ndarray:
    """First hit distance along unit rays ``dirs`` (M,3) from ``origin``; NaN if none."""
    o = np.asarray(origin, dtype=np.float64)
    d = np.asarray(dirs, dtype=np.float64)
    M = d.shape[0]
    out = np.full(M, np.nan)
    ts = tmin * (tmax / tmin) ** (np.arange(n_coarse) / (n_coarse - 1))
    chunk = 65536
    for a in range(0, M, chunk):
        dd = d[a:a + chunk]
        px = o[0] + ts[None, :] * dd[:, 0:1]
        py = o[1] + ts[None, :] * dd[:, 1:2]
        pz = o[2] + ts[None, :] * dd[:, 2:3]
        below = pz <= terrain.height(px, py)
        hit = below.any(axis=1)
        k = np.argmax(below, axis=1)
        rows = np.nonzero(hit & (k > 0))[0]
        lo = ts[k[rows] - 1].copy()
        hi = ts[k[rows]].copy()
        dr = dd[rows]
        for _ in range(n_bisect):
            mid = 0.5 * (lo + hi)
            q = o[None, :] + mid[:, None] * dr
            under = q[:, 2] <= terrain.height(q[:, 0], q[:, 1])
            hi = np.where(under, mid, hi)
            lo = np.where(under, lo, mid)
        res = np.full(dd.shape[0], np.nan)
        res[rows] = 0.5 * (lo + hi)
        out[a:a + chunk] = res
    return out


def _noisy_points(rng, origin, dirs, t):
    """Gaussian range noise sigma = 0.01 + 0.002 r along each ray."""
    sig = 0.01 + 0.002 * np.nan_to_num(t, nan=0.0)
    tn = t + rng.standard_normal(t.shape) * sig
    return origin[None, :] + tn[:, None] * dirs


def _colour(terrain: Terrain, p_w: np.ndarray, rng) -> np.ndarray:
    x = np.nan_to_num(p_w[:, 0])
    y = np.nan_to_num(p_w[:, 1])
    step = terrain.height(x, y) - 0.3 * np.sin(0.7 * x) * np.cos(0.5 * y)
    base = np.stack([90 + 60 * np.sin(0.9 * x), 110 + 50 * np.cos(0.8 * y), 70 + 300 * step], axis=1)
    base += rng.normal(0, 12, size=base.shape)
    return np.clip(np.rint(base), 0, 255).astype(np.uint8)


def dirichlet_probs(rng, n: int, k: int, alpha: float) -> np.ndarray:
    g = rng.standard_gamma(alpha, size=(n, k))
    g = np.maximum(g, 1e-30)
    return (g / g.sum(axis=1, keepdims=True)).astype(np.float32)


def topk_pairs(probs: np.ndarray, k: int) -> np.ndarray:
    """A segmentation output reduced to its k most probable classes per row: float32 [N, 2k] of
    (class id, probability), largest first, the smaller class first on equal probabilities."""
    p = np.asarray(probs, np.float32)
    order = np.argsort(-p, axis=1, kind="stable")[:, :k]
    out = np.empty((p.shape[0], 2 * k), np.float32)
    out[:, 0::2] = order.astype(np.float32)
    out[:, 1::2] = np.take_along_axis(p, order, axis=1)
    return out


def f32_to_bf16_bits(a: np.ndarray) -> np.ndarray:
    """float32 -> bfloat16 bit patterns (round to nearest even), as uint16."""
    b = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = (b + 0x7FFF + ((b >> 16) & 1)) >> 16
    return r.astype(np.uint16)


def bf16_bits_to_f32(b: np.ndarray) -> np.ndarray:
    return (np.asarray(b, dtype=np.uint16).astype(np.uint32) << 16).view(np.float32)


# ----------------------------------------------------------------------------
# configuration 1: one 20k-point cloud, 200x200 map at 0.04 m


@dataclass
class Cloud:
    xyz: np.ndarray            # float32 [N,3], sensor frame, NaN rows allowed
    T: np.ndarray              # float64 [4,4] sensor -> world
    rgb: np.ndarray | None = None     # uint8 [N,3]
    probs: np.ndarray | None = None   # float32 [N,K]
    feat: np.ndarray | None = None    # uint16 (bf16 bits) or float32 [N,d]

    @property
    def n(self) -> int:
        return int(self.xyz.shape[0])


def uniform_ground_cloud(seed: int, n: int, extent: float, terrain: Terrain, *,
                         sensor_xy=(0.0, 0.0), height: float = 0.6, yaw: float | None = None,
                         n_feat: int = 0) -> Cloud:
    """Points uniform in xy over a square ``extent`` wide around ``sensor_xy`` on the terrain,
    observed from a sensor ``height`` above the terrain with range noise, in the sensor frame."""
    rng = np.random.default_rng(seed)
    if yaw is None:
        yaw = float(rng.uniform(-math.pi, math.pi))
    sx, sy = sensor_xy
    s = np.array([sx, sy, float(terrain.height(sx, sy)) + height])
    xy = rng.uniform(-extent / 2, extent / 2, size=(n, 2)) + np.array([sx, sy])
    g = np.column_stack([xy, terrain.height(xy[:, 0], xy[:, 1])])
    v = g - s
    r = np.linalg.norm(v, axis=1)
    d = v / r[:, None]
    p_w = _noisy_points(rng, s, d, r)
    T = pose(rot_z(yaw), s)
    cl = Cloud(to_sensor_frame(T, p_w), T, rgb=_colour(terrain, p_w, rng))
    if n_feat:
        cl.feat = f32_to_bf16_bits(smooth_features(rng, p_w, n_feat))
    return cl


def smooth_features(rng, p_w: np.ndarray, d: int) -> np.ndarray:
    """d-dim features: random Fourier features of position plus noise, ~unit variance."""
    w = rng.normal(0, 1.2, size=(2, d))
    b = rng.uniform(0, 2 * math.pi, size=d)
    f = math.sqrt(2.0) * np.cos(p_w[:, :2] @ w + b) * 0.9
    f += rng.normal(0, 0.3, size=f.shape)
    return f.astype(np.float32)


def config1(seed: int = 0):
    """One 20k-point cloud; map 200x200 at 0.04 m (8 m x 8 m)."""
    ter = Terrain.from_seed(seed)
    cl = uniform_ground_cloud(seed + 1, 20_000, 8.0, ter)
    return dict(W=200, res=0.04, terrain=ter, cloud=cl)


# ----------------------------------------------------------------------------
# configuration 2: LiDAR (128 x 2048) + depth camera (640 x 480), 20-class probs


def lidar_dirs(n_beams: int, n_az: int, yaw: float) -> np.ndarray:
    el = np.deg2rad(np.linspace(-25.0, 15.0, n_beams))
    az = np.linspace(0, 2 * math.pi, n_az, endpoint=False) + yaw
    E, A = np.meshgrid(el, az, indexing="ij")
    return np.stack([np.cos(E) * np.cos(A), np.cos(E) * np.sin(A), np.sin(E)], axis=-1).reshape(-1, 3)


def depth_dirs(width: int, height: int, f: float, R_wc: np.ndarray) -> np.ndarray:
    u, v = np.meshgrid(np.arange(width) + 0.5, np.arange(height) + 0.5)
    d = np.stack([(u - width / 2) / f, (v - height / 2) / f, np.ones_like(u)], axis=-1).reshape(-1, 3)
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return d @ R_wc.T


def path_poses(seed: int, n_poses: int, step: float = 0.3):
    """Robot xy and yaw along a seeded path: 0.3 m steps, heading changes within +-15 deg."""
    rng = np.random.default_rng(seed)
    x, y, yaw = 0.0, 0.0, float(rng.uniform(-math.pi, math.pi))
    out = []
    for _ in range(n_poses):
        out.append((x, y, yaw))
        yaw += math.radians(float(rng.uniform(-15, 15)))
        x += step * math.cos(yaw)
        y += step * math.sin(yaw)
    return out


def multimodal_scan(seed: int, terrain: Terrain, robot, *, n_beams=128, n_az=2048,
                    depth_w=640, depth_h=480, n_classes=20, dir_alpha=0.3):
    """LiDAR + depth-camera clouds from one robot pose, concatenated into one cloud in the
    LiDAR frame; per point RGB and Dirichlet(alpha) class probabilities."""
    rng = np.random.default_rng(seed)
    x, y, yaw = robot
    base = np.array([x, y, float(terrain.height(x, y)) + 0.6])
    T_lidar = pose(rot_z(yaw), base)
    d_l = lidar_dirs(n_beams, n_az, yaw)
    t_l = raycast(terrain, base, d_l, 0.5, 40.0)
    p_l = _noisy_points(rng, base, d_l, t_l)
    # depth camera: 0.2 m ahead of the LiDAR, pitched 30 deg down
    R_wc = rot_z(yaw) @ rot_y(math.radians(30.0)) @ R_BODY_OPTICAL
    cam = base + rot_z(yaw) @ np.array([0.2, 0.0, -0.1])
    f = 385.0 * depth_w / 640.0
    d_c = depth_dirs(depth_w, depth_h, f, R_wc)
    t_c = raycast(terrain, cam, d_c, 0.3, 6.0, n_coarse=48)
    p_c = _noisy_points(rng, cam, d_c, t_c)
    p_w = np.concatenate([p_l, p_c], axis=0)
    n = p_w.shape[0]
    cl = Cloud(to_sensor_frame(T_lidar, p_w), T_lidar)
    cl.rgb = _colour(terrain, p_w, rng)
    cl.probs = dirichlet_probs(rng, n, n_classes, dir_alpha)
    return cl


def config2(seed: int = 0, n_poses: int = 10, scale: float = 1.0):
    """Multi-modal clouds along a 10-pose path over a 500x500 map at 0.04 m.
    ``scale`` < 1 shrinks the sensors (beams, azimuths, depth resolution) for small tests."""
    ter = Terrain.from_seed(seed)
    poses = path_poses(seed + 7, n_poses)
    nb = max(8, int(round(128 * scale)))
    na = max(64, int(round(2048 * scale)))
    dw = max(32, int(round(640 * scale)))
    dh = max(24, int(round(480 * scale)))
    scans = [multimodal_scan(1000 + k, ter, poses[k], n_beams=nb, n_az=na, depth_w=dw, depth_h=dh)
             for k in range(n_poses)]
    return dict(W=500, res=0.04, terrain=ter, poses=poses, scans=scans, n_classes=20)


# ----------------------------------------------------------------------------
# configuration 3: 4 pinhole cameras 848x480, 64-channel features + 20-class seg


def gaussian_field(rng, h: int, w: int, c: int, sigma: float) -> np.ndarray:
    """Smooth Gaussian random field (H,W,C) with unit variance per channel (FFT blur)."""
    noise = rng.standard_normal((c, h, w)).astype(np.float32)
    fy = np.fft.fftfreq(h)[:, None]
    fx = np.fft.rfftfreq(w)[None, :]
    g = np.exp(-2 * (math.pi * sigma) ** 2 * (fx ** 2 + fy ** 2)).astype(np.float32)
    out = np.fft.irfft2(np.fft.rfft2(noise) * g[None], s=(h, w)).astype(np.float32)
    out -= out.mean(axis=(1, 2), keepdims=True)
    out /= out.std(axis=(1, 2), keepdims=True) + 1e-12
    return np.ascontiguousarray(out.transpose(1, 2, 0))


def softmax_field(rng, h: int, w: int, k: int, sigma: float, temp: float = 2.0) -> np.ndarray:
    z = gaussian_field(rng, h, w, k, sigma) * temp
    z -= z.max(axis=2, keepdims=True)
    e = np.exp(z)
    return (e / e.sum(axis=2, keepdims=True)).astype(np.float32)


@dataclass
class Camera:
    T: np.ndarray          # float64 [4,4] optical camera -> world
    K: tuple               # fx, fy, cx, cy
    H: int
    Wi: int
    feat: np.ndarray | None = None   # float32 [H,W,C]
    seg: np.ndarray | None = None    # float32 [H,W,K]


def cameras_around(seed: int, robot, terrain: Terrain, *, n_cams=4, H=480, Wi=848, f=420.0,
                   n_feat=64, n_classes=20, sigma_px=8.0, images=True):
    """Pinhole cameras mounted +-0.3 m around the robot at 0.6 m, yaw 0/90/180/270 +-10 deg,
    pitch -20 +- 5 deg (looking down)."""
    rng = np.random.default_rng(seed)
    x, y, yaw = robot
    zc = float(terrain.height(x, y)) + 0.6
    cams = []
    scale = Wi / 848.0
    for c in range(n_cams):
        a = yaw + c * math.pi / 2 + math.radians(float(rng.uniform(-10, 10)))
        pitch = math.radians(20.0 + float(rng.uniform(-5, 5)))
        R = rot_z(a) @ rot_y(pitch) @ R_BODY_OPTICAL
        pos = np.array([x + 0.3 * math.cos(a), y + 0.3 * math.sin(a), zc])
        cam = Camera(pose(R, pos), (f * scale, f * scale, Wi / 2.0, H / 2.0), H, Wi)
        if images:
            cam.feat = gaussian_field(rng, H, Wi, n_feat, sigma_px * scale)
            cam.seg = softmax_field(rng, H, Wi, n_classes, sigma_px * scale)
        cams.append(cam)
    return cams


def config3(seed: int = 0, scale: float = 1.0, n_feat: int = 64):
    """Map 500x500 at 0.04 m pre-filled from one multi-modal scan, 4 cameras."""
    c2 = config2(seed, n_poses=1, scale=scale)
    cams = cameras_around(seed + 3, c2["poses"][0], c2["terrain"], H=max(24, int(480 * scale)),
                          Wi=max(32, int(848 * scale)), n_feat=n_feat)
    return dict(W=500, res=0.04, terrain=c2["terrain"], robot=c2["poses"][0], prefill=c2["scans"][0],
                cameras=cams)


# ----------------------------------------------------------------------------
# configuration 4: 512 independent maps, log-uniform 5k..60k points, RGB + 16-d bf16 features


def config4_cloud(b: int, seed_base: int = 10_000, n_lo: int = 5_000, n_hi: int = 60_000,
                  W: int = 200, res: float = 0.05, n_feat: int = 16):
    """The cloud of map b of the batched workload (its own terrain, pose and size)."""
    rng = np.random.default_rng(seed_base + b)
    n = int(math.floor(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
    ter = Terrain.from_seed(seed_base + b)
    sxy = tuple(rng.uniform(-1.0, 1.0, size=2))
    return uniform_ground_cloud(seed_base + b + 500_000, n, W * res, ter, sensor_xy=sxy, n_feat=n_feat)


def config4(n_maps: int = 512, seed_base: int = 10_000, n_lo: int = 5_000, n_hi: int = 60_000,
            W: int = 200, res: float = 0.05, n_feat: int = 16):
    clouds = [config4_cloud(b, seed_base, n_lo, n_hi, W, res, n_feat) for b in range(n_maps)]
    offsets = np.zeros(n_maps + 1, dtype=np.int64)
    offsets[1:] = np.cumsum([c.n for c in clouds])
    return dict(W=W, res=res, clouds=clouds, offsets=offsets)


# ----------------------------------------------------------------------------
# configuration 5: crops of height maps with occlusion holes


def line_of_sight(terrain: Terrain, sensor, X, Y, Z, n_steps: int = 96) -> np.ndarray:
    """True where the straight segment from the sensor to (X, Y, Z) stays above the continuous
    terrain (dense float64 march; a sensor simulation, not a map computation)."""
    s = np.asarray(sensor, dtype=np.float64)
    t = (np.arange(1, n_steps) / n_steps)[:, None, None]
    px = s[0] + t * (X[None] - s[0])
    py = s[1] + t * (Y[None] - s[1])
    pz = s[2] + t * (Z[None] - s[2])
    return np.all(pz > terrain.height(px, py) + 1e-9, axis=0)


def inpaint_crops(n: int, size: int = 256, res: float = 0.05, seed: int = 0, lo: float = 0.10,
                  hi: float = 0.60, sensor_height=(0.3, 1.2)):
    """n crops (size x size cells) of terrain heights with the cells hidden from a random sensor
    pose removed (occlusion holes); the hidden fraction is rejection-sampled into [lo, hi].
    Returns heights float32 [n,S,S] (the full, ground-truth field) and known uint8 [n,S,S]."""
    rng = np.random.default_rng(seed)
    hs, ks = [], []
    ext = size * res
    xs = (np.arange(size) - size / 2 + 0.5) * res
    X, Y = np.meshgrid(xs, xs)
    while len(hs) < n:
        ter = Terrain.from_seed(int(rng.integers(0, 2**31)))
        Z = ter.height(X, Y)
        sx, sy = rng.uniform(-ext / 2, ext / 2, size=2)
        sz = float(ter.height(sx, sy)) + float(rng.uniform(*sensor_height))
        vis = line_of_sight(ter, (sx, sy, sz), X, Y, Z)
        frac = 1.0 - vis.mean()
        if not (lo <= frac <= hi):
            continue
        hs.append(Z.astype(np.float32))
        ks.append(vis.astype(np.uint8))
    return np.stack(hs), np.stack(ks)


def concat_clouds(clouds):
    xyz = np.concatenate([c.xyz for c in clouds], axis=0)
    rgb = np.concatenate([c.rgb for c in clouds], axis=0) if clouds[0].rgb is not None else None
    feat = np.concatenate([c.feat for c in clouds], axis=0) if clouds[0].feat is not None else None
    probs = np.concatenate([c.probs for c in clouds], axis=0) if clouds[0].probs is not None else None
    T = np.stack([c.T for c in clouds], axis=0)
    return xyz, rgb, feat, probs, T
