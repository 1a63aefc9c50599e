"""CPU oracle of MEM's map-update path (arXiv 2309.16818), plain C behind ctypes.

TEST INFRASTRUCTURE ONLY. The test suite, the smoke check and the benchmark's
CPU-baseline leg are the only users; the CUDA library never imports, links or
calls anything here, and nothing here calls the CUDA library.

Parity status of each function (what pins it in ``tests/test_oracle_*.py``):

* ``fuse_points``  transform / key (hand-computed cells, 90-degree yaw, brute force on W=8),
  height update (k equal-variance readings closed form, flat plane, sequential == batch,
  gate at lambda +- eps), rules (closed forms of Eqs. 1, 2, 6-7, 12; sums to one; one-hot counts;
  permutation invariance; brute force of the class max)
* ``fuse_image``   known cell -> known pixel, flat map all visible, wall-shadow interval,
  Bresenham path properties in all 8 octants, dense float64 ray march on small maps
* ``move``         shift + inverse shift, fuse-then-move == move-then-fuse
* ``harmonic_fill`` linear fields and constants reproduced, maximum principle

``tests/test_oracle_mutants.py`` builds copies of this oracle (and of ``unet.py``) with one
planted mistake each -- a dropped term, a wrong sign, a transposed index, swapped weights, an
off-by-one limit -- and
requires the pins above to fail on every one. ``tests/golden/make_golden.py`` writes the stored
expected values of ``tests/golden/fusion_w12.json`` from this oracle alone.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liboracle.so")
SRC = [os.path.join(HERE, "mem_oracle.c")]

LATEST, EXPAVG, GAUSS, DIRICHLET, CLASSMAX = range(5)
F32, BF16, F16, U8 = range(4)
MAX_LAYERS = 16
MAX_SRC_LAYERS = 8


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no contraction of a*b+c, no fast-math). MEM_ORACLE_LIB names
    an already built copy to load instead (the planted-mistake tests build altered copies)."""
    if os.environ.get("MEM_ORACLE_LIB"):
        return os.environ["MEM_ORACLE_LIB"]
    newest = max(os.path.getmtime(p) for p in SRC + [os.path.join(HERE, "mem_oracle.h")])
    if force or not os.path.exists(LIB_PATH) or os.path.getmtime(LIB_PATH) < newest:
        tmp = LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
                               "-shared", "-o", tmp] + SRC + ["-lm"])
        os.replace(tmp, LIB_PATH)
    return LIB_PATH


class Cfg(C.Structure):
    _fields_ = [("W", C.c_int32), ("n_layers", C.c_int32), ("res", C.c_double),
                ("sigma0", C.c_float), ("sigma1", C.c_float), ("gate_lambda", C.c_float),
                ("outlier_var", C.c_float), ("time_var", C.c_float), ("range_min", C.c_float),
                ("range_max", C.c_float), ("z_near", C.c_float), ("round_store", C.c_int32),
                ("channels", C.c_int32 * MAX_LAYERS), ("rule", C.c_int32 * MAX_LAYERS),
                ("store", C.c_int32 * MAX_LAYERS), ("w", C.c_double * MAX_LAYERS),
                ("var_meas", C.c_double * MAX_LAYERS), ("alpha0", C.c_double * MAX_LAYERS),
                ("drift_alpha", C.c_double), ("drift_min_points", C.c_int32),
                ("ray_cleanup", C.c_int32), ("ray_margin", C.c_float)]


class State(C.Structure):
    _fields_ = [("h", C.c_void_p), ("var", C.c_void_p), ("valid", C.c_void_p),
                ("n_acc", C.c_void_p), ("n_rej", C.c_void_p),
                ("layer", C.c_void_p * MAX_LAYERS), ("lvar", C.c_void_p * MAX_LAYERS),
                ("obs", C.c_void_p * MAX_LAYERS), ("origin", C.c_double * 2)]


class Src(C.Structure):
    _fields_ = [("data", C.c_void_p), ("dtype", C.c_int32), ("channels", C.c_int32),
                ("n_layers", C.c_int32), ("layers", C.c_int32 * MAX_SRC_LAYERS), ("topk", C.c_int32)]


@dataclass
class TopK:
    """Class probabilities given as the top k classes (Sec. III-C): ``pairs`` float32 [N, 2k] of
    (class id, probability) per row, ``K`` the class count of the layers the source feeds."""
    pairs: np.ndarray
    K: int


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        P = C.c_void_p
        L.orc_init_state.argtypes = [P, P]
        L.orc_pose_rel.argtypes = [P, P, P]
        L.orc_point_cell.argtypes = [P, P, P, P, P, P]
        L.orc_point_cell.restype = C.c_int
        L.orc_fuse_points.argtypes = [P, P, C.c_int64, P, C.c_int32, P, P, P, P]
        L.orc_fuse_points.restype = C.c_int64
        L.orc_move.argtypes = [P, P, P]
        L.orc_bresenham.argtypes = [C.c_int32] * 4 + [P, C.c_int32]
        L.orc_bresenham.restype = C.c_int32
        L.orc_fuse_image.argtypes = [P, P, C.c_int32, C.c_int32, C.c_int32, P, P, P, P, P]
        L.orc_fuse_image.restype = C.c_int64
        L.orc_harmonic_fill.argtypes = [C.c_int32, C.c_int32, P, P, C.c_double, C.c_int32, P]
        L.orc_harmonic_fill.restype = C.c_int32
        L.orc_last_fuse_info.argtypes = [P, P, P]
        L.orc_normals.argtypes = [P, P, P, P]
        _lib = L
    return _lib


def _p(a: np.ndarray) -> int:
    assert a.flags.c_contiguous
    return a.ctypes.data


@dataclass
class Layer:
    """A multi-modal layer: ``channels`` = K classes or d feature dimensions."""
    channels: int
    rule: int
    store: int = F32
    w: float = 0.1
    var_meas: float = 1.0
    alpha0: float = 1.0

    @property
    def stored(self) -> int:
        return 2 if self.rule == CLASSMAX else self.channels


@dataclass
class Params:
    W: int
    res: float
    layers: list = field(default_factory=list)
    sigma0: float = 0.01
    sigma1: float = 0.002
    gate_lambda: float = 2.0
    outlier_var: float = 0.0
    time_var: float = 0.0
    range_min: float = 0.1
    range_max: float = 50.0
    z_near: float = 0.05
    drift_alpha: float = 0.0
    drift_min_points: int = 1
    ray_cleanup: bool = False
    ray_margin: float = 0.1


def _dtype_code(a: np.ndarray, bf16: bool = False) -> int:
    if a.dtype == np.float32:
        return F32
    if a.dtype == np.uint8:
        return U8
    if a.dtype == np.uint16 and bf16:
        return BF16
    if a.dtype == np.float16:
        return F16
    raise TypeError(f"unsupported source dtype {a.dtype}")


class OracleMap:
    """Map state held in float64 numpy arrays. ``round_store`` rounds stored values to their
    storage precision after each update (float32 geometric layers, per-layer format)."""

    def __init__(self, p: Params, round_store: bool = True):
        self.p = p
        W2 = p.W * p.W
        c = Cfg()
        c.W = p.W
        c.n_layers = len(p.layers)
        c.res = p.res
        for k in ("sigma0", "sigma1", "gate_lambda", "outlier_var", "time_var", "range_min",
                  "range_max", "z_near", "drift_alpha", "drift_min_points", "ray_margin"):
            setattr(c, k, getattr(p, k))
        c.ray_cleanup = int(bool(p.ray_cleanup))
        c.round_store = int(round_store)
        for i, L in enumerate(p.layers):
            c.channels[i] = L.channels
            c.rule[i] = L.rule
            c.store[i] = L.store
            c.w[i] = L.w
            c.var_meas[i] = L.var_meas
            c.alpha0[i] = L.alpha0
        self.cfg = c
        self.h = np.zeros(W2)
        self.var = np.zeros(W2)
        self.valid = np.zeros(W2, np.uint8)
        self.n_acc = np.zeros(W2, np.uint32)
        self.n_rej = np.zeros(W2, np.uint32)
        self.layer = [np.zeros(W2 * L.stored) for L in p.layers]
        self.lvar = [np.zeros(W2 * L.channels) if L.rule == GAUSS else np.zeros(1) for L in p.layers]
        self.obs = [np.zeros(W2, np.uint8) for _ in p.layers]
        st = State()
        st.h, st.var, st.valid = _p(self.h), _p(self.var), _p(self.valid)
        st.n_acc, st.n_rej = _p(self.n_acc), _p(self.n_rej)
        for i in range(len(p.layers)):
            st.layer[i] = _p(self.layer[i])
            st.lvar[i] = _p(self.lvar[i])
            st.obs[i] = _p(self.obs[i])
        st.origin[0] = 0.0
        st.origin[1] = 0.0
        self.st = st
        lib().orc_init_state(C.byref(c), C.byref(st))

    # -- state views ---------------------------------------------------------------
    @property
    def origin(self):
        return (self.st.origin[0], self.st.origin[1])

    def layer_values(self, l: int) -> np.ndarray:
        L = self.p.layers[l]
        return self.layer[l].reshape(self.p.W * self.p.W, L.stored)

    def theta(self, l: int) -> np.ndarray:
        """Dirichlet layer: posterior mean alpha / sum(alpha) (Eq. 11)."""
        a = self.layer_values(l)
        return a / a.sum(axis=1, keepdims=True)

    def gauss_var(self, l: int) -> np.ndarray:
        return self.lvar[l].reshape(self.p.W * self.p.W, self.p.layers[l].channels)

    # -- operations ----------------------------------------------------------------
    def _sources(self, sources, keep):
        arr = (Src * max(1, len(sources)))()
        for i, (data, layers) in enumerate(sources):
            if isinstance(data, TopK):
                a = np.ascontiguousarray(data.pairs, dtype=np.float32)
                keep.append(a)
                arr[i].data = _p(a)
                arr[i].dtype = F32
                arr[i].channels = data.K
                arr[i].topk = a.shape[-1] // 2
                arr[i].n_layers = len(layers)
                for k, l in enumerate(layers):
                    arr[i].layers[k] = l
                continue
            bf16 = isinstance(data, tuple)
            a = np.ascontiguousarray(data[0] if bf16 else data)
            keep.append(a)
            arr[i].data = _p(a)
            arr[i].dtype = _dtype_code(a, bf16)
            arr[i].channels = a.shape[1] if a.ndim == 2 else a.shape[-1]
            arr[i].n_layers = len(layers)
            for k, l in enumerate(layers):
                arr[i].layers[k] = l
        return arr

    def fuse_points(self, xyz: np.ndarray, T: np.ndarray, sources=(), want_cells=False,
                    want_near=False):
        """sources: list of (array [N,C], (uint16 bf16 bits array,) or TopK, [layer ids])."""
        xyz = np.ascontiguousarray(xyz, dtype=np.float32)
        n = xyz.shape[0]
        keep = []
        src = self._sources(list(sources), keep)
        T = np.ascontiguousarray(T, dtype=np.float64)
        cells = np.empty(n, np.int32) if want_cells else None
        near = np.empty(n, np.uint8) if want_near else None
        kept = lib().orc_fuse_points(C.byref(self.cfg), C.byref(self.st), n, _p(xyz), len(sources),
                                     C.cast(src, C.c_void_p), _p(T),
                                     _p(near) if near is not None else None,
                                     _p(cells) if cells is not None else None)
        drift, dn, cleared = C.c_double(), C.c_int64(), C.c_int64()
        lib().orc_last_fuse_info(C.byref(drift), C.byref(dn), C.byref(cleared))
        return dict(kept=kept, cells=cells, near=near, drift=drift.value, drift_points=dn.value,
                    cleared=cleared.value)

    def fuse_image(self, H: int, Wi: int, sources, K, T):
        keep = []
        src = self._sources(list(sources), keep)
        Kd = np.ascontiguousarray(K, dtype=np.float64)
        T = np.ascontiguousarray(T, dtype=np.float64)
        W2 = self.p.W * self.p.W
        vis = np.empty(W2, np.uint8)
        pix = np.empty(W2, np.int32)
        nv = lib().orc_fuse_image(C.byref(self.cfg), C.byref(self.st), H, Wi, len(sources),
                                  C.cast(src, C.c_void_p), _p(Kd), _p(T), _p(vis), _p(pix))
        return dict(n_visible=nv, vis=vis, pix=pix)

    def normals(self):
        """Surface normals of the elevation layer: (normals float32 [W*W, 3], ok uint8 [W*W])."""
        W2 = self.p.W * self.p.W
        out = np.zeros((W2, 3), np.float32)
        ok = np.zeros(W2, np.uint8)
        lib().orc_normals(C.byref(self.cfg), C.byref(self.st), _p(out), _p(ok))
        return out, ok

    def pca(self, l: int, n_comp: int = 3):
        """PCA of a feature layer over its observed cells (see pca_of_features)."""
        from .plugins import pca_of_features
        obs = self.obs[l].astype(bool)
        return pca_of_features(self.layer_values(l), obs, n_comp)

    def move(self, robot_xy):
        xy = np.ascontiguousarray(robot_xy, dtype=np.float64)
        lib().orc_move(C.byref(self.cfg), C.byref(self.st), _p(xy))


def point_cell(p: Params, T: np.ndarray, pts: np.ndarray, origin=(0.0, 0.0)):
    """Cell index (or -1), map-frame z and measurement variance of each point."""
    m = OracleMap(Params(p.W, p.res, [], p.sigma0, p.sigma1, p.gate_lambda, p.outlier_var,
                         p.time_var, p.range_min, p.range_max, p.z_near, p.drift_alpha,
                         p.drift_min_points, p.ray_cleanup, p.ray_margin))
    Rt = np.empty(12, np.float32)
    o = np.array(origin, dtype=np.float64)
    T = np.ascontiguousarray(T, dtype=np.float64)
    lib().orc_pose_rel(_p(T), _p(o), _p(Rt))
    out = []
    for q in np.ascontiguousarray(pts, dtype=np.float32):
        q = np.ascontiguousarray(q)
        cell = np.zeros(1, np.int32)
        z = np.zeros(1, np.float32)
        vm = np.zeros(1, np.float32)
        ok = lib().orc_point_cell(C.byref(m.cfg), _p(Rt), _p(q), _p(cell), _p(z), _p(vm))
        out.append((int(cell[0]) if ok else -1, float(z[0]), float(vm[0])))
    return out


def bresenham(sx: int, sy: int, ex: int, ey: int) -> np.ndarray:
    cap = 2 * (abs(ex - sx) + abs(ey - sy)) + 4
    buf = np.zeros(2 * cap, np.int32)
    n = lib().orc_bresenham(sx, sy, ex, ey, _p(buf), cap)
    return buf[:2 * n].reshape(n, 2)


def harmonic_fill_exact(h: np.ndarray, known: np.ndarray) -> np.ndarray:
    """The harmonic fill as its definition: for every unknown cell, (number of in-grid
    4-neighbours) * x_j - sum of unknown neighbours = sum of known neighbours; solved directly
    in float64 (sparse LU). Unknown cells with no known cell in their connected group keep the
    mean of the known cells (the starting value of the iterative solvers)."""
    import scipy.ndimage as ndi
    import scipy.sparse as sp
    import scipy.sparse.linalg as spl
    h = np.asarray(h, dtype=np.float64)
    kn = np.asarray(known).astype(bool)
    H, W = h.shape
    out = h.copy()
    mean = h[kn].mean() if kn.any() else 0.0
    unk = ~kn
    if not unk.any():
        return out
    lab, nlab = ndi.label(unk)  # 4-connected groups of unknown cells
    touch = np.zeros(nlab + 1, bool)
    grow = ndi.binary_dilation(kn)  # unknown cells next to a known cell
    touch[np.unique(lab[unk & grow])] = True
    solve = unk & touch[lab]
    out[unk & ~solve] = mean
    n = int(solve.sum())
    if n == 0:
        return out
    idx = -np.ones((H, W), np.int64)
    idx[solve] = np.arange(n)
    deg = np.zeros((H, W))
    b = np.zeros((H, W))
    rows, cols = [], []
    for dy, dx in ((0, 1), (0, -1), (1, 0), (-1, 0)):
        ys, xs = np.nonzero(solve)
        ny, nx = ys + dy, xs + dx
        ok = (ny >= 0) & (ny < H) & (nx >= 0) & (nx < W)
        ys, xs, ny, nx = ys[ok], xs[ok], ny[ok], nx[ok]
        np.add.at(deg, (ys, xs), 1.0)
        nk = kn[ny, nx]
        np.add.at(b, (ys[nk], xs[nk]), h[ny[nk], nx[nk]])
        nu = ~nk
        rows.append(idx[ys[nu], xs[nu]])
        cols.append(idx[ny[nu], nx[nu]])
    r = np.concatenate(rows)
    c = np.concatenate(cols)
    A = sp.csr_matrix((-np.ones(len(r)), (r, c)), shape=(n, n)) + sp.diags(deg[solve])
    out[solve] = spl.spsolve(A.tocsc(), b[solve])
    return out


def harmonic_fill(h: np.ndarray, known: np.ndarray, tol: float = 1e-10, max_sweeps: int = 200000):
    h = np.ascontiguousarray(h, dtype=np.float64).copy()
    k = np.ascontiguousarray(known, dtype=np.uint8)
    r = np.zeros(1)
    it = lib().orc_harmonic_fill(h.shape[0], h.shape[1], _p(h), _p(k), tol, max_sweeps, _p(r))
    return h, int(it), float(r[0])
