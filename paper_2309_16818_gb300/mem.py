"""Python binding of ``libmem.so`` (include/mem.h): argument marshalling only.

Device memory and streams come from PyTorch; every step of the map update runs
in the library's CUDA kernels. Importing this module does not need a GPU, but
loading the library does need it built (``paper_2309_16818_gb300.build``); a
missing library raises instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmem.so")

MAX_LAYERS, MAX_SOURCES, MAX_SOURCE_LAYERS = 16, 8, 8
OK, ERR_ARG, ERR_CUDA, ERR_OOM, ERR_TIMEOUT, ERR_STATE = range(6)
FAULT_NONE, FAULT_SORT_WAIT = 0, 1
LATEST, EXPAVG, GAUSS, DIRICHLET, CLASSMAX = range(5)
F32, BF16, F16, U8 = range(4)
LAYER_HEIGHT, LAYER_VARIANCE, LAYER_VALID, LAYER_NACC, LAYER_NREJ = -1, -2, -3, -4, -5
PART_VALUE, PART_THETA, PART_VAR, PART_OBSERVED = range(4)

EXPORTS = ["mem_create_map", "mem_destroy_map", "mem_move_map", "mem_fuse_pointcloud",
           "mem_fuse_pointcloud_host", "mem_fuse_pointcloud_batch", "mem_fuse_image", "mem_get_layer", "mem_set_layer",
           "mem_get_origin", "mem_check", "mem_last_error", "mem_set_tuning", "mem_get_tuning",
           "mem_set_profiling", "mem_get_profile", "mem_get_stats", "mem_fuse_pointcloud_noalloc",
           "mem_autotune_batch", "mem_inpaint_diffusion", "mem_unet_create", "mem_unet_destroy",
           "mem_unet_param_count", "mem_unet_set_params", "mem_unet_get_params", "mem_unet_forward",
           "mem_unet_gradients", "mem_unet_train_step", "mem_unet_check", "mem_inject_fault",
           "mem_noalloc_check", "mem_get_drift", "mem_unet_prepare", "mem_compute_normals",
           "mem_pca_layer"]
NOALLOC_MAX_POINTS = 1 << 18
PROFILE_SLOTS = ["key", "digit_scan", "radix_sort", "unused3", "fuse_tiles", "fuse_cross",
                 "time_var", "image", "move", "drift", "raycast"]


class LayerDesc(C.Structure):
    _fields_ = [("channels", C.c_int32), ("dtype", C.c_int32), ("rule", C.c_int32),
                ("w", C.c_float), ("var_meas", C.c_float), ("alpha0", C.c_float)]


class MapConfig(C.Structure):
    _fields_ = [("W", C.c_int32), ("n_maps", C.c_int32), ("res", C.c_double),
                ("n_layers", C.c_int32), ("layers", LayerDesc * MAX_LAYERS),
                ("sigma0", C.c_float), ("sigma1", C.c_float), ("gate_lambda", C.c_float),
                ("outlier_var", C.c_float), ("time_var", C.c_float), ("range_min", C.c_float),
                ("range_max", C.c_float), ("z_near", C.c_float), ("max_points", C.c_int64),
                ("drift_alpha", C.c_double), ("drift_min_points", C.c_int32),
                ("ray_cleanup", C.c_int32), ("ray_margin", C.c_float)]


class Source(C.Structure):
    _fields_ = [("data", C.c_void_p), ("dtype", C.c_int32), ("channels", C.c_int32),
                ("n_layers", C.c_int32), ("layers", C.c_int32 * MAX_SOURCE_LAYERS), ("topk", C.c_int32)]


@dataclass
class TopK:
    """Top-k class input (mem_source.topk): ``pairs`` a float32 tensor [N, 2k] (or [H, Wi, 2k])
    of (class id, probability), ``K`` the class count of the layers it feeds."""
    pairs: object
    K: int


class MemError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"status {status}: {msg}")
        self.status = status


_lib = None


def lib():
    """Load ``libmem.so``; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -m paper_2309_16818_gb300.build`")
        L = C.CDLL(LIB_PATH)
        P, I32, I64 = C.c_void_p, C.c_int32, C.c_int64
        sig = {
            "mem_create_map": [P, P], "mem_destroy_map": [P],
            "mem_move_map": [P, I32, P, P],
            "mem_fuse_pointcloud": [P, I64, P, I32, P, P, P],
            "mem_fuse_pointcloud_host": [P, I64, P, I32, P, P, P],
            "mem_fuse_pointcloud_batch": [P, P, P, I32, P, P, P],
            "mem_fuse_image": [P, I32, I32, I32, I32, P, P, P, P, P, P],
            "mem_get_layer": [P, I32, I32, I32, P, P], "mem_set_layer": [P, I32, I32, I32, P, P],
            "mem_get_origin": [P, I32, P], "mem_check": [P, P], "mem_last_error": [],
            "mem_set_tuning": [P, I32, I32, I32], "mem_get_tuning": [P, P],
            "mem_set_profiling": [P, I32], "mem_get_profile": [P, P, P], "mem_get_stats": [P, P, P],
            "mem_fuse_pointcloud_noalloc": [P, P, I64, P, P, P, P, P, P, P, P],
            "mem_autotune_batch": [P, P, P, I32, P, P, I32, P, P, P],
            "mem_inpaint_diffusion": [I32, I32, I32, P, P, P, C.c_float, I32, P, P],
            "mem_unet_create": [I32, P, P], "mem_unet_destroy": [P], "mem_unet_param_count": [P, P],
            "mem_unet_set_params": [P, P, P], "mem_unet_get_params": [P, P, P],
            "mem_unet_forward": [P, I32, I32, I32, P, P, P, P],
            "mem_unet_gradients": [P, I32, I32, I32, P, P, P, P, I64, P, P, P],
            "mem_unet_train_step": [P, I32, I32, I32, P, P, P, P, I64, C.c_float, P, P],
            "mem_unet_check": [P, P], "mem_inject_fault": [P, I32],
            "mem_noalloc_check": [P], "mem_get_drift": [P, I32, P, P],
            "mem_unet_prepare": [I32, I32, I32, P, P, P, P, P, P, P],
            "mem_compute_normals": [P, I32, P, P, P], "mem_pca_layer": [P, I32, I32, I32, P, P, P],
        }
        for name, args in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = C.c_char_p if name == "mem_last_error" else C.c_int
        _lib = L
    return _lib


def _ck(status):
    if status != OK:
        raise MemError(status, lib().mem_last_error().decode())


def _torch():
    import torch
    return torch


def _dtype_code(t) -> int:
    torch = _torch()
    m = {torch.float32: F32, torch.bfloat16: BF16, torch.float16: F16, torch.uint8: U8}
    if t.dtype not in m:
        raise TypeError(f"unsupported dtype {t.dtype}")
    return m[t.dtype]


def _stream(stream):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _pose(T, n=1):
    a = np.ascontiguousarray(np.asarray(T, dtype=np.float64).reshape(n * 16))
    return a


def fuse_pointcloud_noalloc(W, res, xyz, T, h, var, valid, n_acc, n_rej, origin=(0.0, 0.0),
                            stream=None, **params):
    """Allocation-free height fuse into caller-owned tensors (mem_fuse_pointcloud_noalloc):
    h, var float32 [W*W]; valid, n_acc, n_rej int32 [W*W] (uint32 bit patterns)."""
    cfg = MapConfig()
    cfg.W, cfg.n_maps, cfg.res, cfg.n_layers = W, 1, res, 0
    d = dict(sigma0=0.01, sigma1=0.002, gate_lambda=2.0, outlier_var=0.0, time_var=0.0,
             range_min=0.1, range_max=50.0, z_near=0.05)
    d.update(params)
    for k, v in d.items():
        setattr(cfg, k, v)
    o = np.ascontiguousarray(origin, dtype=np.float64)
    n = int(xyz.shape[0])
    for t in (h, var, valid, n_acc, n_rej):
        assert t.is_cuda and t.is_contiguous() and t.numel() == W * W and t.element_size() == 4
    _ck(lib().mem_fuse_pointcloud_noalloc(C.byref(cfg), o.ctypes.data, n,
                                          C.c_void_p(xyz.data_ptr() if n else 0), _pose(T).ctypes.data,
                                          C.c_void_p(h.data_ptr()), C.c_void_p(var.data_ptr()),
                                          C.c_void_p(valid.data_ptr()), C.c_void_p(n_acc.data_ptr()),
                                          C.c_void_p(n_rej.data_ptr()), _stream(stream)))


def noalloc_check(stream=None):
    """Synchronise and raise MemError (ERR_TIMEOUT) if an allocation-free fuse on the current
    device timed out in a bounded device wait since the previous check (mem_noalloc_check)."""
    _ck(lib().mem_noalloc_check(_stream(stream)))


def inpaint_diffusion(h, known, tol=1e-6, max_iters=20000, out=None, stream=None):
    """Harmonic fill of unknown cells: h float32 [B,H,W] cuda, known uint8 [B,H,W] cuda.
    Returns (filled float32 [B,H,W], sweeps used int32 [B])."""
    torch = _torch()
    assert h.is_cuda and h.dtype == torch.float32 and h.is_contiguous() and h.dim() == 3
    assert known.is_cuda and known.dtype == torch.uint8 and known.shape == h.shape and known.is_contiguous()
    B, H, W = h.shape
    if out is None:
        out = torch.empty_like(h)
    its = torch.zeros(B, dtype=torch.int32, device=h.device)
    _ck(lib().mem_inpaint_diffusion(B, H, W, C.c_void_p(h.data_ptr()), C.c_void_p(known.data_ptr()),
                                    C.c_void_p(out.data_ptr()), tol, max_iters,
                                    C.c_void_p(its.data_ptr()), _stream(stream)))
    return out, its


def unet_prepare(h, known, fill, stream=None):
    """Network inputs of a batch of crops (mem_unet_prepare): h, fill float32 [B,H,W] cuda,
    known uint8 [B,H,W] cuda. Returns (x3 float32 [B,H,W,3], hidden uint8 [B,H,W],
    mean of the known heights float32 [B])."""
    torch = _torch()
    for t in (h, known, fill):
        assert t.is_cuda and t.is_contiguous() and t.shape == h.shape and t.dim() == 3
    assert h.dtype == torch.float32 and fill.dtype == torch.float32 and known.dtype == torch.uint8
    B, H, W = h.shape
    x3 = torch.empty((B, H, W, 3), dtype=torch.float32, device=h.device)
    hidden = torch.empty((B, H, W), dtype=torch.uint8, device=h.device)
    mean = torch.empty(B, dtype=torch.float32, device=h.device)
    _ck(lib().mem_unet_prepare(B, H, W, C.c_void_p(h.data_ptr()), C.c_void_p(known.data_ptr()),
                               C.c_void_p(fill.data_ptr()), C.c_void_p(x3.data_ptr()),
                               C.c_void_p(hidden.data_ptr()), C.c_void_p(mean.data_ptr()), _stream(stream)))
    return x3, hidden, mean


@dataclass
class Layer:
    channels: int
    rule: int
    dtype: int = F32
    w: float = 0.1
    var_meas: float = 1.0
    alpha0: float = 1.0

    @property
    def stored(self) -> int:
        return 2 if self.rule == CLASSMAX else self.channels


class Map:
    """A set of ``n_maps`` robot-centric W x W maps with the given multi-modal layers."""

    def __init__(self, W: int, res: float, layers=(), n_maps: int = 1, sigma0: float = 0.01,
                 sigma1: float = 0.002, gate_lambda: float = 2.0, outlier_var: float = 0.0,
                 time_var: float = 0.0, range_min: float = 0.1, range_max: float = 50.0,
                 z_near: float = 0.05, max_points: int = 1 << 20, drift_alpha: float = 0.0,
                 drift_min_points: int = 1, ray_cleanup: bool = False, ray_margin: float = 0.1):
        cfg = MapConfig()
        cfg.W, cfg.n_maps, cfg.res = W, n_maps, res
        self.layers = list(layers)
        cfg.n_layers = len(self.layers)
        for i, L in enumerate(self.layers):
            d = cfg.layers[i]
            d.channels, d.dtype, d.rule = L.channels, L.dtype, L.rule
            d.w, d.var_meas, d.alpha0 = L.w, L.var_meas, L.alpha0
        cfg.sigma0, cfg.sigma1, cfg.gate_lambda = sigma0, sigma1, gate_lambda
        cfg.outlier_var, cfg.time_var = outlier_var, time_var
        cfg.range_min, cfg.range_max, cfg.z_near = range_min, range_max, z_near
        cfg.max_points = max_points
        cfg.drift_alpha, cfg.drift_min_points = drift_alpha, drift_min_points
        cfg.ray_cleanup, cfg.ray_margin = int(bool(ray_cleanup)), ray_margin
        self.cfg = cfg
        self.W, self.n_maps, self.res = W, n_maps, res
        self._h = C.c_void_p()
        _ck(lib().mem_create_map(C.byref(cfg), C.byref(self._h)))

    def close(self):
        if self._h:
            lib().mem_destroy_map(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- inputs -------------------------------------------------------------------
    def _sources(self, sources, keep, on_host=False):
        arr = (Source * MAX_SOURCES)()
        for i, (t, layers) in enumerate(sources):
            K = None
            if isinstance(t, TopK):
                t, K = t.pairs, t.K
            assert t.is_cuda != on_host and t.is_contiguous()
            keep.append(t)
            arr[i].data = t.data_ptr()
            arr[i].dtype = _dtype_code(t)
            arr[i].channels = t.shape[-1] if K is None else K
            arr[i].topk = 0 if K is None else t.shape[-1] // 2
            arr[i].n_layers = len(layers)
            for k, l in enumerate(layers):
                arr[i].layers[k] = l
        return arr

    def fuse_pointcloud(self, xyz, T, sources=(), stream=None):
        """xyz: cuda float32 [N,3] (sensor frame); sources: [(cuda [N,C] tensor, [layer ids])];
        T: 4x4 sensor -> world (float64 host)."""
        keep = []
        src = self._sources(list(sources), keep)
        n = int(xyz.shape[0])
        _ck(lib().mem_fuse_pointcloud(self._h, n, C.c_void_p(xyz.data_ptr() if n else 0),
                                      len(sources), src, _pose(T).ctypes.data, _stream(stream)))

    def fuse_pointcloud_host(self, xyz, T, sources=(), stream=None):
        """As fuse_pointcloud with CPU tensors (pinned for an asynchronous upload): the library
        copies them to device staging buffers of its own, overlapping the previous call's
        kernels. The tensors must stay unchanged until the call's work on `stream` is done."""
        keep = []
        src = self._sources(list(sources), keep, on_host=True)
        assert not xyz.is_cuda and xyz.is_contiguous()
        n = int(xyz.shape[0])
        _ck(lib().mem_fuse_pointcloud_host(self._h, n, C.c_void_p(xyz.data_ptr() if n else 0),
                                           len(sources), src, _pose(T).ctypes.data, _stream(stream)))

    def fuse_pointcloud_batch(self, offsets, xyz, T, sources=(), stream=None):
        keep = []
        src = self._sources(list(sources), keep)
        off = np.ascontiguousarray(offsets, dtype=np.int64)
        Tb = _pose(T, self.n_maps)
        _ck(lib().mem_fuse_pointcloud_batch(self._h, off.ctypes.data,
                                            C.c_void_p(xyz.data_ptr() if xyz.numel() else 0),
                                            len(sources), src, Tb.ctypes.data, _stream(stream)))

    def fuse_image(self, H, Wi, K, T, sources=(), map_index=0, vis=None, pix=None, stream=None):
        keep = []
        src = self._sources(list(sources), keep)
        Kd = np.ascontiguousarray(K, dtype=np.float64)
        _ck(lib().mem_fuse_image(self._h, map_index, H, Wi, len(sources), src, Kd.ctypes.data,
                                 _pose(T).ctypes.data,
                                 C.c_void_p(vis.data_ptr() if vis is not None else 0),
                                 C.c_void_p(pix.data_ptr() if pix is not None else 0),
                                 _stream(stream)))

    def move(self, robot_xy, map_index=0, stream=None):
        xy = np.ascontiguousarray(robot_xy, dtype=np.float64)
        _ck(lib().mem_move_map(self._h, map_index, xy.ctypes.data, _stream(stream)))

    # -- state ----------------------------------------------------------------------
    def _layer_shape(self, layer, part):
        torch = _torch()
        W2 = self.W * self.W
        if layer < 0:
            dt = {LAYER_HEIGHT: torch.float32, LAYER_VARIANCE: torch.float32,
                  LAYER_VALID: torch.uint8, LAYER_NACC: torch.int32, LAYER_NREJ: torch.int32}[layer]
            return (W2,), dt
        L = self.layers[layer]
        if part == PART_VALUE:
            dt = {F32: torch.float32, BF16: torch.bfloat16, F16: torch.float16}[L.dtype]
            return (W2, L.stored), dt
        if part == PART_THETA:
            return (W2, L.channels), torch.float32
        if part == PART_VAR:
            return (W2,), torch.float32
        return (W2,), torch.uint8

    def get_layer(self, layer, part=PART_VALUE, map_index=0, out=None, stream=None):
        torch = _torch()
        shape, dt = self._layer_shape(layer, part)
        if out is None:
            out = torch.empty(shape, dtype=dt, device="cuda")
        _ck(lib().mem_get_layer(self._h, map_index, layer, part, C.c_void_p(out.data_ptr()),
                                _stream(stream)))
        return out

    def set_layer(self, layer, src, part=PART_VALUE, map_index=0, stream=None):
        shape, dt = self._layer_shape(layer, part)
        assert src.is_cuda and src.is_contiguous() and src.dtype == dt and src.numel() == int(np.prod(shape))
        _ck(lib().mem_set_layer(self._h, map_index, layer, part, C.c_void_p(src.data_ptr()),
                                _stream(stream)))

    def origin(self, map_index=0):
        o = np.zeros(2)
        _ck(lib().mem_get_origin(self._h, map_index, o.ctypes.data))
        return float(o[0]), float(o[1])

    def check(self, stream=None):
        _ck(lib().mem_check(self._h, _stream(stream)))

    def inject_fault(self, kind):
        """Tests only: FAULT_SORT_WAIT makes the sort's bounded waits run out; FAULT_NONE clears."""
        _ck(lib().mem_inject_fault(self._h, kind))

    def set_tuning(self, radix_bits, blocks_per_sm, fuse_kernel=0):
        """fuse_kernel 0: per-cell sums in registers where the call's columns fit one round;
        1: the shared-memory tile kernel always."""
        _ck(lib().mem_set_tuning(self._h, radix_bits, blocks_per_sm, fuse_kernel))

    def get_tuning(self):
        out = np.zeros(4, np.int32)
        _ck(lib().mem_get_tuning(self._h, out.ctypes.data))
        return dict(radix_bits=int(out[0]), blocks_per_sm=int(out[1]), passes=int(out[2]),
                    fuse_kernel=int(out[3]))

    def autotune_batch(self, offsets, xyz, T, sources=(), reps=3, stream=None):
        """Pick the fastest schedule for this batched call; the map state is left unchanged.
        Returns (chosen tuning, list of candidate times in ms)."""
        keep = []
        src = self._sources(list(sources), keep)
        off = np.ascontiguousarray(offsets, dtype=np.int64)
        Tb = _pose(T, self.n_maps)
        ms = np.zeros(32, np.float32)
        n = C.c_int32(32)
        _ck(lib().mem_autotune_batch(self._h, off.ctypes.data,
                                     C.c_void_p(xyz.data_ptr() if xyz.numel() else 0), len(sources),
                                     src, Tb.ctypes.data, reps, _stream(stream), ms.ctypes.data,
                                     C.byref(n)))
        return self.get_tuning(), [float(x) for x in ms[:n.value]]

    def set_profiling(self, on: bool):
        _ck(lib().mem_set_profiling(self._h, int(on)))

    def get_profile(self):
        """{slot name: (total ms, launch groups)} since the previous read."""
        ms = np.zeros(16, np.float64)
        calls = np.zeros(16, np.int64)
        _ck(lib().mem_get_profile(self._h, ms.ctypes.data, calls.ctypes.data))
        return {k: (float(ms[i]), int(calls[i])) for i, k in enumerate(PROFILE_SLOTS)}

    def normals(self, map_index=0, stream=None):
        """Surface normals of the elevation layer: (float32 [W*W, 3], uint8 ok [W*W]) cuda."""
        torch = _torch()
        out = torch.empty((self.W * self.W, 3), dtype=torch.float32, device="cuda")
        ok = torch.empty(self.W * self.W, dtype=torch.uint8, device="cuda")
        _ck(lib().mem_compute_normals(self._h, map_index, C.c_void_p(out.data_ptr()), C.c_void_p(ok.data_ptr()),
                                      _stream(stream)))
        return out, ok

    def pca(self, layer, n_comp=3, map_index=0, stream=None):
        """PCA layer of a feature layer: (projections float32 [W*W, n_comp], eigenvalues
        [n_comp], vectors [n_comp, C], mean [C]) cuda."""
        torch = _torch()
        Cc = self.layers[layer].channels
        proj = torch.empty((self.W * self.W, n_comp), dtype=torch.float32, device="cuda")
        info = torch.empty(n_comp + n_comp * Cc + Cc, dtype=torch.float32, device="cuda")
        _ck(lib().mem_pca_layer(self._h, map_index, layer, n_comp, C.c_void_p(proj.data_ptr()),
                                C.c_void_p(info.data_ptr()), _stream(stream)))
        return proj, info[:n_comp], info[n_comp:n_comp + n_comp * Cc].view(n_comp, Cc), info[n_comp + n_comp * Cc:]

    def get_drift(self, map_index=0, stream=None):
        """{drift: shift applied by the last point fuse, drift_points: points in its mean,
        cleared: cells invalidated by the last call's ray-cast clean-up}."""
        out = np.zeros(3, np.float64)
        _ck(lib().mem_get_drift(self._h, map_index, _stream(stream), out.ctypes.data))
        return dict(drift=float(out[0]), drift_points=int(out[1]), cleared=int(out[2]))

    def get_stats(self, stream=None):
        out = np.zeros(4, np.int64)
        _ck(lib().mem_get_stats(self._h, _stream(stream), out.ctypes.data))
        return dict(crossing_cells=int(out[0]), cells=int(out[1]), kept=int(out[2]),
                    passes=int(out[3]))


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else C.c_void_p(0)


class UNet:
    """Inpainting U-Net on the library's BF16 tensor-core kernels (mem_unet_*)."""

    def __init__(self, cin=3, widths=(32, 64, 128, 128)):
        self.cin, self.widths = cin, tuple(widths)
        w = (C.c_int32 * 4)(*widths)
        self._h = C.c_void_p()
        _ck(lib().mem_unet_create(cin, w, C.byref(self._h)))
        n = C.c_int64()
        _ck(lib().mem_unet_param_count(self._h, C.byref(n)))
        self.n_params = n.value

    def close(self):
        if self._h:
            lib().mem_unet_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, flat, stream=None):
        torch = _torch()
        assert flat.is_cuda and flat.dtype == torch.float32 and flat.numel() == self.n_params
        _ck(lib().mem_unet_set_params(self._h, _ptr(flat.contiguous()), _stream(stream)))

    def get_params(self, stream=None):
        torch = _torch()
        out = torch.empty(self.n_params, dtype=torch.float32, device="cuda")
        _ck(lib().mem_unet_get_params(self._h, _ptr(out), _stream(stream)))
        return out

    def forward(self, x3, fill, out=None, stream=None):
        torch = _torch()
        n, H, W, _ = x3.shape
        if out is None:
            out = torch.empty((n, H, W), dtype=torch.float32, device="cuda")
        _ck(lib().mem_unet_forward(self._h, n, H, W, _ptr(x3), _ptr(fill), _ptr(out), _stream(stream)))
        return out

    def gradients(self, x3, fill, target, hidden, stream=None):
        torch = _torch()
        n, H, W, _ = x3.shape
        g = torch.empty(self.n_params, dtype=torch.float32, device="cuda")
        loss = torch.zeros(1, dtype=torch.float32, device="cuda")
        nh = int(hidden.sum().item())
        _ck(lib().mem_unet_gradients(self._h, n, H, W, _ptr(x3), _ptr(fill), _ptr(target), _ptr(hidden), nh,
                                     _ptr(g), _ptr(loss), _stream(stream)))
        return g, loss

    def train_step(self, x3, fill, target, hidden, lr, n_hidden=None, loss=None, stream=None):
        torch = _torch()
        n, H, W, _ = x3.shape
        if loss is None:
            loss = torch.zeros(1, dtype=torch.float32, device="cuda")
        nh = int(hidden.sum().item()) if n_hidden is None else int(n_hidden)
        _ck(lib().mem_unet_train_step(self._h, n, H, W, _ptr(x3), _ptr(fill), _ptr(target), _ptr(hidden), nh,
                                      lr, _ptr(loss), _stream(stream)))
        return loss

    def check(self, stream=None):
        """Synchronise and raise MemError if a bounded device wait ran out."""
        _ck(lib().mem_unet_check(self._h, _stream(stream)))
