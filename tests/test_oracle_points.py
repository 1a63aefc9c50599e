"""Pins of the oracle's point-cloud path (Sec. III-B association, the height update it
inherits, and the fusion rules of Sec. III-C) against closed forms, invariants and brute
force. CPU only."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2309_16818_gb300 import synth


def ident(t=(0.0, 0.0, 0.0)):
    T = np.eye(4)
    T[:3, 3] = t
    return T


def mk(W=8, res=0.5, layers=(), **kw):
    return O.Params(W=W, res=res, layers=list(layers), **kw)


# --------------------------------------------------------------------------- transform / key

def test_identity_pose_cells_by_hand():
    p = mk(W=8, res=0.5)
    pts = np.array([
        [0.25, 0.25, 0.0],    # floor(0.5)=0 -> ix=4, iy=4 -> 36
        [-0.01, 0.74, 0.0],   # floor(-0.02)=-1 -> 3 ; floor(1.48)=1 -> 5 -> 5*8+3 = 43
        [0.5, -0.5, 0.0],     # edge: floor(1.0)=1 -> 5 ; floor(-1.0)=-1 -> 3 -> 29
        [-2.0, -2.0, 0.3],    # lower corner cell -> 0
        [1.99, 1.99, 0.0],    # floor(3.98)=3 -> 7 -> 63
        [2.0, 0.1, 0.0],      # x = +W/2 res is outside
        [np.nan, 0.1, 0.0],   # non-finite
        [0.01, 0.01, 0.0],    # range 0.014 < range_min 0.1
    ], dtype=np.float32)
    got = [c for c, _, _ in O.point_cell(p, ident(), pts)]
    assert got == [36, 43, 29, 0, 63, -1, -1, -1]


def test_translation_and_origin():
    p = mk(W=8, res=0.5)
    # sensor 1 m up and 0.5 m along x; map centre at x = 0.5 -> same cells as identity
    got = O.point_cell(p, ident((0.5, 0.0, 1.0)), np.array([[0.25, 0.25, -1.0]], np.float32),
                       origin=(0.5, 0.0))
    assert got[0][0] == 36 and got[0][1] == 0.0


def test_yaw_90_swaps_axes_exactly():
    p = mk(W=16, res=0.25)
    T = ident()
    T[:3, :3] = [[0, -1, 0], [1, 0, 0], [0, 0, 1]]
    rng = np.random.default_rng(1)
    pts = (rng.integers(-30, 30, size=(200, 3)) * 0.0625 + 0.03125).astype(np.float32)
    got = O.point_cell(p, T, pts)
    for (xs, ys, zs), (c, z, _) in zip(pts, got):
        x, y = -ys, xs
        ix, iy = math.floor(x / 0.25) + 8, math.floor(y / 0.25) + 8
        exp = iy * 16 + ix if (0 <= ix < 16 and 0 <= iy < 16) else -1
        assert c == exp
        if c >= 0:
            assert z == zs


def test_transform_matches_float64_within_ulps():
    p = mk(W=2000, res=0.01, range_max=1e9)
    rng = np.random.default_rng(2)
    yaw, pitch = 0.7, 0.2
    T = ident((1.3, -0.4, 0.6))
    T[:3, :3] = synth.rot_z(yaw) @ synth.rot_y(pitch)
    pts = rng.uniform(-5, 5, size=(300, 3)).astype(np.float32)
    got = O.point_cell(p, T, pts)
    for q, (c, z, vm) in zip(pts, got):
        zd = T[2, :3] @ q.astype(np.float64) + T[2, 3]
        assert abs(z - zd) <= 8 * np.spacing(np.float32(abs(zd) + 1))
        rng_ = float(np.linalg.norm(q.astype(np.float64)))
        assert abs(vm - (0.01 + 0.002 * rng_) ** 2) <= 1e-6 * vm


def test_brute_force_cells_w8():
    p = mk(W=8, res=0.5)
    rng = np.random.default_rng(3)
    pts = rng.uniform(-2.6, 2.6, size=(2000, 3)).astype(np.float32)
    got = O.point_cell(p, ident(), pts)
    n_in = 0
    for q, (c, _, _) in zip(pts, got):
        x, y = float(q[0]), float(q[1])
        if min(abs(x / 0.5 - round(x / 0.5)), abs(y / 0.5 - round(y / 0.5))) < 1e-5:
            continue  # too close to an edge for a float64 reference to be decisive
        ix, iy = math.floor(x / 0.5) + 4, math.floor(y / 0.5) + 4
        r = math.sqrt(sum(float(v) ** 2 for v in q))
        ok = 0 <= ix < 8 and 0 <= iy < 8 and 0.1 <= r <= 50
        assert c == (iy * 8 + ix if ok else -1)
        n_in += ok
    assert n_in > 500


# --------------------------------------------------------------------------- height update

# sensor-frame points with exactly equal range 9/8 (Pythagorean quadruples over 8), all
# inside cell (4, 4) of an 8 x 8 map at 1 m: their float32 ranges, and so their
# measurement variances, are identical
EQUAL_RANGE_PTS = np.array([[1, 4, -8], [4, 1, -8], [4, 4, -7], [0, 0, -9], [4, 7, -4],
                            [7, 4, -4]], np.float32) / 8


def equal_range_points(k, rng):
    return EQUAL_RANGE_PTS[rng.integers(0, len(EQUAL_RANGE_PTS), size=k)]


def test_k_equal_variance_readings_closed_form():
    """k readings of equal variance s^2 into a prior sigma0^2 give s^2 / (k + s^2/sigma0^2);
    into an empty cell s^2 / k; the mean is the precision-weighted mean."""
    rng = np.random.default_rng(4)
    p = mk(W=8, res=1.0, gate_lambda=1e6)
    m = O.OracleMap(p, round_store=False)
    k1, k2 = 7, 12
    a = equal_range_points(k1, rng)
    b = equal_range_points(k2, rng)
    j = 4 * 8 + 4
    s = np.float32(np.float32(0.002) * np.float32(9 / 8) + np.float32(0.01))
    s2 = float(s * s)
    r = m.fuse_points(a, ident(), want_cells=True)
    assert np.all(r["cells"] == j)
    assert m.var[j] == pytest.approx(s2 / k1, rel=1e-14)
    assert m.h[j] == pytest.approx(a[:, 2].astype(np.float64).mean(), abs=1e-14)
    h0, v0 = m.h[j], m.var[j]
    m.fuse_points(b, ident())
    pw = s2 / v0
    assert pw == pytest.approx(k1, rel=1e-14)
    assert m.var[j] == pytest.approx(s2 / (k2 + pw), rel=1e-14)
    assert m.h[j] == pytest.approx((h0 * pw + b[:, 2].astype(np.float64).sum()) / (k2 + pw),
                                   abs=1e-14)
    assert m.n_acc[j] == k1 + k2 and m.n_rej[j] == 0


def test_flat_plane_reproduces_height():
    rng = np.random.default_rng(5)
    p = mk(W=32, res=0.1, gate_lambda=3.0)
    m = O.OracleMap(p)
    c = 0.375  # exactly representable
    xy = rng.uniform(-1.5, 1.5, size=(5000, 2))
    pts = np.column_stack([xy, np.full(len(xy), c - 0.6)]).astype(np.float32)
    for _ in range(3):
        m.fuse_points(pts, ident((0, 0, 0.6)))
    v = m.valid.astype(bool)
    assert v.sum() > 800
    assert np.all(np.abs(m.h[v] - c) <= 1e-6)


def test_sequential_equals_batch():
    rng = np.random.default_rng(6)
    p = mk(W=8, res=0.5, gate_lambda=1e6)
    pts = rng.uniform(-1.9, 1.9, size=(64, 3)).astype(np.float32)
    pts[:, 2] = rng.uniform(-1.2, -0.8, size=64)
    a = O.OracleMap(p, round_store=False)
    a.fuse_points(pts, ident())
    b = O.OracleMap(p, round_store=False)
    for q in pts:
        b.fuse_points(q[None], ident())
    v = a.valid.astype(bool)
    assert np.array_equal(v, b.valid.astype(bool))
    np.testing.assert_allclose(b.h[v], a.h[v], rtol=0, atol=1e-12)
    np.testing.assert_allclose(b.var[v], a.var[v], rtol=1e-12)


@pytest.mark.parametrize("lam", [1.0, 2.0, 3.5])
def test_gate_boundary(lam):
    p = mk(W=8, res=0.5, gate_lambda=lam)
    m = O.OracleMap(p, round_store=False)
    j = 4 * 8 + 4
    # seed the cell: many equal points at z = 0 -> valid, h = 0
    base = np.array([[0.2, 0.2, -1.0]], np.float32)
    m.fuse_points(np.repeat(base, 4, 0), ident((0, 0, 1.0)))
    h0, v0 = m.h[j], m.var[j]
    assert m.valid[j] == 1
    for eps, rej in ((+1e-3, 1), (-1e-3, 0)):
        mm = O.OracleMap(p, round_store=False)
        mm.fuse_points(np.repeat(base, 4, 0), ident((0, 0, 1.0)))
        # a point (0.2, 0.2, -v) below the sensor: range sqrt(0.08 + v^2), map z = 1 - v;
        # find v with (z - h0)^2 = (lam + eps)^2 (v0 + vm) by bisection in float64
        lo, hi = 0.5, 1.0
        for _ in range(200):
            v = 0.5 * (lo + hi)
            d = (1.0 - v) - h0
            vm = (0.01 + 0.002 * math.sqrt(0.08 + v * v)) ** 2
            if d * d > (lam + eps) ** 2 * (v0 + vm):
                lo = v
            else:
                hi = v
        q = np.array([[0.2, 0.2, -v]], np.float32)
        mm.fuse_points(q, ident((0, 0, 1.0)))
        assert mm.n_rej[j] == rej and mm.n_acc[j] == 4 + (1 - rej)


def test_outlier_and_time_variance():
    p = mk(W=8, res=0.5, gate_lambda=2.0, outlier_var=0.5, time_var=0.25)
    m = O.OracleMap(p, round_store=False)
    j = 4 * 8 + 4
    m.fuse_points(np.array([[0.2, 0.2, -1.0]] * 3, np.float32), ident((0, 0, 1.0)))
    v1 = m.var[j]
    # first scan: v = s^2/3 + time_var
    m.fuse_points(np.array([[0.2, 0.2, 2.0]] * 2, np.float32), ident((0, 0, 1.0)))
    assert m.n_rej[j] == 2
    assert m.var[j] == pytest.approx(v1 + 2 * 0.5 + 0.25, rel=1e-12)
    assert m.valid.sum() == 1


def test_time_variance_ages_untouched_valid_cells():
    """time_var is added to EVERY valid cell once per call, touched or not (the height
    update's process noise; the paper defers the model to its predecessor, this is the reading
    stated in the design notes). Two valid cells; later calls touch only one of them, and an
    empty cloud touches none: the other cell's variance grows by exactly time_var per call."""
    p = mk(W=8, res=0.5, time_var=0.25)
    m = O.OracleMap(p, round_store=False)
    j, k = 4 * 8 + 4, 6 * 8 + 6
    # first call: three readings in j and two in k (points below a sensor at height 1)
    pts = np.array([[0.2, 0.2, -1.0]] * 3 + [[1.2, 1.2, -1.0]] * 2, np.float32)
    m.fuse_points(pts, ident((0, 0, 1.0)))
    assert m.valid[j] == 1 and m.valid[k] == 1 and m.valid.sum() == 2
    s2 = lambda r: (0.01 + 0.002 * r) ** 2
    vk = s2(math.sqrt(1.2 ** 2 * 2 + 1.0)) / 2 + 0.25      # fresh cell: s^2 / 2, then aged once
    assert m.var[k] == pytest.approx(vk, rel=1e-6)   # float32 measurement variance
    vk = m.var[k]
    for call in range(3):
        m.fuse_points(np.array([[0.2, 0.2, -1.0]], np.float32), ident((0, 0, 1.0)))
        vk += 0.25
        assert m.var[k] == pytest.approx(vk, rel=1e-12), f"untouched cell, call {call}"
        assert m.n_acc[k] == 2
    # an empty cloud ages both valid cells and nothing else
    vj = m.var[j]
    m.fuse_points(np.zeros((0, 3), np.float32), ident((0, 0, 1.0)))
    assert m.var[k] == pytest.approx(vk + 0.25, rel=1e-12)
    assert m.var[j] == pytest.approx(vj + 0.25, rel=1e-12)
    assert m.valid.sum() == 2 and np.all(m.var[m.valid == 0] == 0)


# --------------------------------------------------------------------------- fusion rules

def cell_groups(cells):
    g = {}
    for i, c in enumerate(cells):
        if c >= 0:
            g.setdefault(int(c), []).append(i)
    return g


def test_latest_average_brute_force_and_sum_to_one():
    rng = np.random.default_rng(7)
    p = mk(W=8, res=0.5, layers=[O.Layer(3, O.LATEST), O.Layer(5, O.LATEST)])
    m = O.OracleMap(p, round_store=False)
    n = 300
    pts = rng.uniform(-2.2, 2.2, size=(n, 3)).astype(np.float32)
    rgb = rng.integers(0, 256, size=(n, 3), dtype=np.uint8)
    probs = synth.dirichlet_probs(rng, n, 5, 0.5)
    r = m.fuse_points(pts, ident(), [(rgb, [0]), (probs, [1])], want_cells=True)
    g = cell_groups(r["cells"])
    for c, idx in g.items():
        exp = [sum(float(rgb[i, k]) for i in idx) / len(idx) for k in range(3)]
        assert list(m.layer_values(0)[c]) == pytest.approx(exp, abs=1e-12)
        assert m.layer_values(1)[c].sum() == pytest.approx(1.0, abs=5 * 2 ** -23)
    untouched = np.setdiff1d(np.arange(64), list(g))
    assert np.all(m.layer_values(0)[untouched] == 0) and np.all(m.obs[0][untouched] == 0)


def test_permutation_invariance():
    rng = np.random.default_rng(8)
    L = [O.Layer(3, O.LATEST), O.Layer(4, O.DIRICHLET), O.Layer(4, O.CLASSMAX),
         O.Layer(4, O.EXPAVG, w=0.3), O.Layer(4, O.GAUSS, var_meas=0.5)]
    p = mk(W=8, res=0.5, layers=L)
    n = 400
    pts = rng.uniform(-2, 2, size=(n, 3)).astype(np.float32)
    pts[:, 2] = rng.normal(-1, 0.02, n)
    rgb = rng.integers(0, 256, size=(n, 3), dtype=np.uint8)
    pr = synth.dirichlet_probs(rng, n, 4, 0.3)
    perm = rng.permutation(n)
    out = []
    for order in (np.arange(n), perm):
        m = O.OracleMap(p, round_store=False)
        for _ in range(2):
            m.fuse_points(pts[order], ident((0, 0, 0.0)),
                          [(rgb[order], [0]), (pr[order], [1, 2, 3, 4])])
        out.append(m)
    a, b = out
    np.testing.assert_allclose(a.h, b.h, atol=1e-12)
    np.testing.assert_array_equal(a.n_acc, b.n_acc)
    for l in range(len(L)):
        np.testing.assert_allclose(a.layer[l], b.layer[l], atol=1e-12)


def test_expavg_closed_form():
    w, T = 0.2, 9
    p = mk(W=8, res=0.5, layers=[O.Layer(2, O.EXPAVG, w=w)])
    m = O.OracleMap(p, round_store=False)
    q = np.array([[0.2, 0.2, -1.0]], np.float32)
    a0, a = np.array([[0.9, 0.1]], np.float32), np.array([[0.25, 0.75]], np.float32)
    m.fuse_points(q, ident(), [(a0, [0])])
    for _ in range(T):
        m.fuse_points(q, ident(), [(a, [0])])
    j = 36
    exp = a.astype(np.float64)[0] + (1 - w) ** T * (a0.astype(np.float64)[0] - a.astype(np.float64)[0])
    np.testing.assert_allclose(m.layer_values(0)[j], exp, atol=1e-12)


def test_fig3_expavg_forgets_faster_than_dirichlet():
    """Fig. 3: after a class switch exponential averaging loses confidence in the old class
    geometrically, (1-w)^n, while the Dirichlet posterior mean decays like 1/n."""
    K, w, a0, n0 = 3, 0.1, 1.0, 10
    p = mk(W=8, res=0.5, layers=[O.Layer(K, O.EXPAVG, w=w), O.Layer(K, O.DIRICHLET, alpha0=a0)])
    m = O.OracleMap(p, round_store=False)
    q = np.array([[0.2, 0.2, -1.0]], np.float32)
    one = lambda k: np.eye(K, dtype=np.float32)[k][None]
    for _ in range(n0):
        m.fuse_points(q, ident(), [(one(0), [0, 1])])
    j = 36
    for n in range(1, 61):
        m.fuse_points(q, ident(), [(one(1), [0, 1])])
        e = m.layer_values(0)[j][0]
        d = m.theta(1)[j][0]
        assert e == pytest.approx((1 - w) ** n, rel=1e-12)
        assert d == pytest.approx((a0 + n0) / (K * a0 + n0 + n), rel=1e-12)
        if n >= 12:
            assert e < d


def test_gaussian_closed_forms():
    sf2 = 0.7
    p = mk(W=8, res=0.5, layers=[O.Layer(3, O.GAUSS, var_meas=sf2)], gate_lambda=1e6)
    rng = np.random.default_rng(9)
    m = O.OracleMap(p, round_store=False)
    q = np.array([[0.2, 0.2, -1.0]], np.float32)
    j = 36
    f1 = rng.normal(size=(5, 3)).astype(np.float32)
    m.fuse_points(np.repeat(q, 5, 0), ident(), [(f1, [0])])
    mu1 = m.layer_values(0)[j].copy()
    # first observation: infinitely wide prior -> mu = mu_ML in [min f, max f], var = sf2 / N
    np.testing.assert_allclose(mu1, f1.astype(np.float64).mean(0), atol=1e-12)
    assert np.all(mu1 >= f1.min(0)) and np.all(mu1 <= f1.max(0))
    np.testing.assert_allclose(m.gauss_var(0)[j], sf2 / 5, rtol=1e-12)
    # equal readings: variance sf2 / (k + sf2 / var0) and all dimensions share it
    f2 = rng.normal(size=(8, 3)).astype(np.float32)
    m.fuse_points(np.repeat(q, 8, 0), ident(), [(f2, [0])])
    v = m.gauss_var(0)[j]
    assert np.all(v == v[0])
    assert v[0] == pytest.approx(sf2 / (8 + sf2 / (sf2 / 5)), rel=1e-12)
    # sequential == batch: 13 readings at once from an empty cell
    b = O.OracleMap(p, round_store=False)
    b.fuse_points(np.repeat(q, 13, 0), ident(), [(np.concatenate([f1, f2]), [0])])
    np.testing.assert_allclose(b.layer_values(0)[j], m.layer_values(0)[j], atol=1e-12)
    np.testing.assert_allclose(b.gauss_var(0)[j], m.gauss_var(0)[j], rtol=1e-12)


def test_dirichlet_one_hot_votes_exact():
    K, a0 = 20, 1.0
    p = mk(W=8, res=0.5, layers=[O.Layer(K, O.DIRICHLET, alpha0=a0)])
    m = O.OracleMap(p)
    q = np.array([[0.2, 0.2, -1.0]], np.float32)
    N, c = 37, 11
    oh = np.zeros((N, K), np.float32)
    oh[:, c] = 1
    m.fuse_points(np.repeat(q, N, 0), ident(), [(oh, [0])])
    j = 36
    alpha = m.layer_values(0)[j]
    assert alpha[c] == a0 + N and np.all(np.delete(alpha, c) == a0)
    th = m.theta(0)[j]
    assert th[c] == (a0 + N) / (K * a0 + N)
    assert th.sum() == pytest.approx(1.0, abs=K * 2 ** -52)


def test_classmax_brute_force():
    rng = np.random.default_rng(10)
    K = 6
    p = mk(W=8, res=0.5, layers=[O.Layer(K, O.CLASSMAX)])
    m = O.OracleMap(p)
    n = 500
    pts = rng.uniform(-2, 2, size=(n, 3)).astype(np.float32)
    pr = synth.dirichlet_probs(rng, n, K, 0.3)
    pr[5, :] = 0.5  # ties: smallest class index must win
    r = m.fuse_points(pts, ident(), [(pr, [0])], want_cells=True)
    g = cell_groups(r["cells"])
    for c, idx in g.items():
        best, bid = -1.0, -1
        for k in range(K):
            for i in idx:
                if pr[i, k] > best:
                    best, bid = float(pr[i, k]), k
        assert m.layer_values(0)[c][0] == bid and m.layer_values(0)[c][1] == best
    assert np.all(m.layer_values(0)[np.setdiff1d(np.arange(64), list(g))][:, 0] == -1)


def test_bf16_storage_rounding():
    p = mk(W=8, res=0.5, layers=[O.Layer(2, O.LATEST, store=O.BF16)])
    m = O.OracleMap(p)
    q = np.array([[0.2, 0.2, -1.0]], np.float32)
    v = np.array([[1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8]], np.float32)  # both ties -> even
    m.fuse_points(q, ident(), [(v, [0])])
    assert list(m.layer_values(0)[36]) == [1.0, 1.0 + 2 ** -6]


def test_time_variance_ages_only_valid_cells():
    """time_var inflates the variance of every valid cell once per call (Sec. III-B reading);
    cells never observed stay at zero variance and invalid."""
    p = mk(W=8, res=0.5, time_var=0.25)
    m = O.OracleMap(p, round_store=False)
    for _ in range(3):
        m.fuse_points(np.array([[0.2, 0.2, -1.0]] * 3, np.float32), ident((0, 0, 1.0)))
    assert m.valid.sum() == 1
    assert np.all(m.var[m.valid == 0] == 0) and np.all(m.h[m.valid == 0] == 0)


def test_classmax_ties_take_the_smallest_class():
    p = mk(W=8, res=0.5, layers=[O.Layer(4, O.CLASSMAX)])
    m = O.OracleMap(p, round_store=False)
    a = np.float32(0.3)
    pts = np.array([[0.2, 0.2, -1.0], [1.2, 1.2, -1.0], [1.3, 1.3, -1.0]], np.float32)
    pr = np.array([[a, a, a, np.float32(0.1)],         # one point, three equal maxima
                   [0.6, 0.4, 0.0, 0.0], [0.4, 0.6, 0.0, 0.0]], np.float32)  # equal maxima across points
    r = m.fuse_points(pts, ident(), [(pr, [0])], want_cells=True)
    c0, c1 = int(r["cells"][0]), int(r["cells"][1])
    assert r["cells"][1] == r["cells"][2]
    assert m.layer_values(0)[c0][0] == 0 and m.layer_values(0)[c0][1] == pytest.approx(float(a))
    assert m.layer_values(0)[c1][0] == 0 and m.layer_values(0)[c1][1] == pytest.approx(0.6)


def test_range_limits_are_inclusive():
    """A point is kept iff range_min <= |p_s| <= range_max (Sec. III-B filter); points on the
    optical axis have exactly representable ranges here."""
    p = mk(W=8, res=0.5, range_min=0.5, range_max=2.0)
    pts = np.array([[0, 0, -2.0], [0, 0, -2.0001], [0, 0, -0.5], [0, 0, -0.4999], [0, 0, -1.0]], np.float32)
    got = [c for c, _, _ in O.point_cell(p, ident(), pts)]
    j = 4 * 8 + 4
    assert got == [j, -1, j, -1, j]
