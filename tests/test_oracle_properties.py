"""Property tests of the oracle over random small inputs (hypothesis): permutation invariance of a
call's result (Sec. III-B/III-C define per-cell sums, so the order of points cannot matter beyond
floating-point reassociation), the Dirichlet update adds exactly the per-cell probability sums
(Eq. 12) and its posterior mean sums to one, the class max is the per-cell arg-max with the
smallest index on ties, the height of a fresh cell is the precision-weighted mean of its readings
with variance 1 / sum of precisions, and a move commutes with a fuse on the cells both frames
share. CPU only."""
import math

import numpy as np
import pytest

import oracle as O

hyp = pytest.importorskip("hypothesis")
from hypothesis import given, settings  # noqa: E402
from hypothesis import strategies as st  # noqa: E402

SETTINGS = dict(max_examples=25, deadline=None, derandomize=True)


def ident():
    return np.eye(4)


def cloud(seed, n, W, res, k):
    rng = np.random.default_rng(seed)
    half = W * res / 2
    pts = np.column_stack([rng.uniform(-half + 1e-3, half - 1e-3, size=(n, 2)),
                           rng.normal(-1.0, 0.05, size=n)]).astype(np.float32)
    p = rng.random((n, k)).astype(np.float32) + np.float32(0.01)
    probs = (p / p.sum(axis=1, keepdims=True)).astype(np.float32)
    rgb = rng.integers(0, 256, size=(n, 3), dtype=np.uint8)
    return rng, pts, probs, rgb


def groups(cells):
    g = {}
    for i, c in enumerate(cells):
        if c >= 0:
            g.setdefault(int(c), []).append(i)
    return g


@settings(**SETTINGS)
@given(seed=st.integers(0, 2 ** 31 - 1), n=st.integers(1, 300), k=st.integers(2, 6))
def test_result_does_not_depend_on_point_order(seed, n, k):
    rng, pts, probs, rgb = cloud(seed, n, 8, 0.5, k)
    L = [O.Layer(3, O.LATEST), O.Layer(k, O.DIRICHLET), O.Layer(k, O.CLASSMAX), O.Layer(k, O.EXPAVG, w=0.3),
         O.Layer(k, O.GAUSS, var_meas=0.5)]
    perm = rng.permutation(n)
    maps = []
    for order in (np.arange(n), perm):
        m = O.OracleMap(O.Params(W=8, res=0.5, layers=L), round_store=False)
        for _ in range(2):
            m.fuse_points(pts[order], ident(), [(rgb[order], [0]), (probs[order], [1, 2, 3, 4])])
        maps.append(m)
    a, b = maps
    np.testing.assert_array_equal(a.valid, b.valid)
    np.testing.assert_array_equal(a.n_acc, b.n_acc)
    np.testing.assert_array_equal(a.n_rej, b.n_rej)
    np.testing.assert_allclose(a.h, b.h, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(a.var, b.var, rtol=1e-12, atol=0)
    for l in range(len(L)):
        np.testing.assert_allclose(a.layer[l], b.layer[l], rtol=1e-12, atol=1e-12)


@settings(**SETTINGS)
@given(seed=st.integers(0, 2 ** 31 - 1), n=st.integers(1, 200), k=st.integers(2, 8),
       alpha0=st.sampled_from([0.5, 1.0, 2.0]))
def test_dirichlet_adds_probability_sums_and_class_max_is_the_argmax(seed, n, k, alpha0):
    _, pts, probs, _ = cloud(seed, n, 8, 0.5, k)
    L = [O.Layer(k, O.DIRICHLET, alpha0=alpha0), O.Layer(k, O.CLASSMAX)]
    m = O.OracleMap(O.Params(W=8, res=0.5, layers=L), round_store=False)
    r = m.fuse_points(pts, ident(), [(probs, [0, 1])], want_cells=True)
    g = groups(r["cells"])
    alpha = m.layer_values(0)
    cm = m.layer_values(1)
    for c, idx in g.items():
        s = probs[idx].astype(np.float64).sum(axis=0)
        np.testing.assert_allclose(alpha[c], alpha0 + s, rtol=1e-12)
        assert math.isclose(float(m.theta(0)[c].sum()), 1.0, rel_tol=1e-12)
        mx = probs[idx].astype(np.float64).max(axis=0)
        best = int(np.flatnonzero(mx == mx.max())[0])  # smallest class index among the maxima
        assert int(cm[c, 0]) == best and cm[c, 1] == mx.max()
    untouched = np.setdiff1d(np.arange(64), list(g))
    assert np.all(m.obs[0][untouched] == 0) and np.all(alpha[untouched] == alpha0)


@settings(**SETTINGS)
@given(seed=st.integers(0, 2 ** 31 - 1), n=st.integers(1, 120))
def test_fresh_cell_height_is_the_precision_weighted_mean(seed, n):
    """Identity pose (the transform is exact), gate off: per cell h = sum(z / s^2) / sum(1 / s^2)
    and var = 1 / sum(1 / s^2), s = sigma0 + sigma1 * range (range and s rounded to float32 by the
    oracle, so the closed form is taken at 1e-6)."""
    _, pts, _, _ = cloud(seed, n, 8, 0.5, 2)
    p = O.Params(W=8, res=0.5, gate_lambda=1e6)
    m = O.OracleMap(p, round_store=False)
    r = m.fuse_points(pts, ident(), want_cells=True)
    x = pts.astype(np.float64)
    rng_ = np.sqrt((x ** 2).sum(axis=1))
    s = p.sigma0 + p.sigma1 * rng_
    w = 1.0 / (s * s)
    for c, idx in groups(r["cells"]).items():
        sw = w[idx].sum()
        assert m.var[c] == pytest.approx(1.0 / sw, rel=1e-6)
        assert m.h[c] == pytest.approx((w[idx] * x[idx, 2]).sum() / sw, rel=1e-6, abs=1e-6)
        assert m.n_acc[c] == len(idx) and m.valid[c] == 1


@settings(**SETTINGS)
@given(seed=st.integers(0, 2 ** 31 - 1), n=st.integers(1, 200), sx=st.integers(-3, 3), sy=st.integers(-3, 3))
def test_move_commutes_with_fuse_on_shared_cells(seed, n, sx, sy):
    W, res = 12, 0.5
    _, pts, probs, rgb = cloud(seed, n, W, res, 3)
    L = [O.Layer(3, O.LATEST), O.Layer(3, O.DIRICHLET)]
    xy = (sx * res, sy * res)
    T = ident()
    a = O.OracleMap(O.Params(W=W, res=res, layers=L, gate_lambda=1e6))
    a.fuse_points(pts, T, [(rgb, [0]), (probs, [1])])
    a.move(xy)
    b = O.OracleMap(O.Params(W=W, res=res, layers=L, gate_lambda=1e6))
    b.move(xy)
    b.fuse_points(pts, T, [(rgb, [0]), (probs, [1])])
    # new cell (ix, iy) was old (ix + sx, iy + sy): compare where that old cell existed
    ys, xs = np.mgrid[0:W, 0:W]
    keep = ((xs + sx >= 0) & (xs + sx < W) & (ys + sy >= 0) & (ys + sy < W)).ravel()
    assert np.array_equal(a.valid[keep], b.valid[keep])
    np.testing.assert_array_equal(a.h[keep], b.h[keep])
    np.testing.assert_array_equal(a.layer_values(0)[keep], b.layer_values(0)[keep])
    np.testing.assert_array_equal(a.layer_values(1)[keep], b.layer_values(1)[keep])


# --------------------------------------------------------------------------- image visibility

def _flat(W, res, height=0.0):
    m = O.OracleMap(O.Params(W=W, res=res, range_max=1e6, gate_lambda=1e6))
    xs = (np.arange(W) - W // 2 + 0.5) * res
    X, Y = np.meshgrid(xs, xs)
    pts = np.column_stack([X.ravel(), Y.ravel(), np.full(W * W, height - 100.0)]).astype(np.float32)
    T = np.eye(4)
    T[2, 3] = 100.0
    m.fuse_points(pts, T)
    return m


DOWN = np.array([[1.0, 0, 0], [0, -1.0, 0], [0, 0, -1.0]])  # optical axis = world -z


@settings(**SETTINGS)
@given(cx=st.integers(2, 21), cy=st.integers(2, 21), hc=st.floats(1.0, 3.0), pick=st.integers(0, 10 ** 6),
       pick_q=st.integers(0, 10 ** 6))
def test_an_occluder_on_the_walk_hides_the_cell_and_removing_it_restores_it(cx, cy, hc, pick, pick_q):
    """Visibility (Sec. III-B): a cell is seen iff every valid cell strictly between it and the
    camera's cell on the Bresenham walk lies below the ray. Raising one such cell above the
    camera hides the target; lowering it again shows it."""
    W, res = 24, 0.25
    m = _flat(W, res)
    pos = ((cx - W // 2 + 0.5) * res, (cy - W // 2 + 0.5) * res, hc)
    T = np.eye(4)
    T[:3, :3] = DOWN
    T[:3, 3] = pos
    K = (30.0, 30.0, 100.0, 100.0)
    out = m.fuse_image(200, 200, [], K, T)
    far = [j for j in np.flatnonzero(out["vis"]) if max(abs(j % W - cx), abs(j // W - cy)) >= 2]
    if not far:
        return
    j = far[pick % len(far)]
    path = O.bresenham(cx, cy, int(j % W), int(j // W))
    inner = path[1:-1]
    q = inner[pick_q % len(inner)]
    qi = int(q[1]) * W + int(q[0])
    m.h[qi] = hc + 1.0
    assert m.fuse_image(200, 200, [], K, T)["vis"][j] == 0
    m.h[qi] = 0.0
    assert m.fuse_image(200, 200, [], K, T)["vis"][j] == 1


@settings(**SETTINGS)
@given(seed=st.integers(0, 2 ** 31 - 1), cx=st.integers(0, 23), cy=st.integers(0, 23))
def test_lowering_other_cells_never_hides_a_visible_cell(seed, cx, cy):
    W, res = 24, 0.25
    rng = np.random.default_rng(seed)
    m = _flat(W, res)
    m.h[:] = rng.uniform(0.0, 0.6, size=W * W)
    T = np.eye(4)
    T[:3, :3] = DOWN
    T[:3, 3] = ((cx - W // 2 + 0.5) * res, (cy - W // 2 + 0.5) * res, 1.5)
    K = (30.0, 30.0, 100.0, 100.0)
    before = m.fuse_image(200, 200, [], K, T)
    lowered = rng.random(W * W) < 0.5
    m.h[lowered] -= rng.uniform(0.0, 0.5, size=int(lowered.sum()))
    after = m.fuse_image(200, 200, [], K, T)
    same = ~lowered  # cells whose own height (so projection and ray) did not change
    assert np.all(after["vis"][same] >= before["vis"][same])
    assert np.array_equal(after["pix"][same & (before["vis"] == 1)], before["pix"][same & (before["vis"] == 1)])


@settings(**SETTINGS)
@given(seed=st.integers(0, 2 ** 31 - 1), n1=st.integers(1, 150), n2=st.integers(1, 150),
       var_meas=st.sampled_from([0.1, 0.5, 2.0]))
def test_gaussian_rule_sequential_equals_batch(seed, n1, n2, var_meas):
    """The Gaussian feature update (Eqs. 6-7) is the conjugate update with known variance, so two
    calls in a row give the posterior of one call with both sets of points (and the Dirichlet
    counts add the same way)."""
    _, pts, probs, _ = cloud(seed, n1 + n2, 8, 0.5, 3)
    rng = np.random.default_rng(seed + 1)
    feat = rng.normal(0.0, 1.0, size=(n1 + n2, 3)).astype(np.float32)
    L = [O.Layer(3, O.GAUSS, var_meas=var_meas), O.Layer(3, O.DIRICHLET)]
    a = O.OracleMap(O.Params(W=8, res=0.5, layers=L), round_store=False)
    a.fuse_points(pts[:n1], ident(), [(feat[:n1], [0]), (probs[:n1], [1])])
    a.fuse_points(pts[n1:], ident(), [(feat[n1:], [0]), (probs[n1:], [1])])
    b = O.OracleMap(O.Params(W=8, res=0.5, layers=L), round_store=False)
    b.fuse_points(pts, ident(), [(feat, [0]), (probs, [1])])
    np.testing.assert_array_equal(a.obs[0], b.obs[0])
    seen = a.obs[0] == 1
    np.testing.assert_allclose(a.layer_values(0)[seen], b.layer_values(0)[seen], rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(a.gauss_var(0)[seen], b.gauss_var(0)[seen], rtol=1e-9)
    np.testing.assert_allclose(a.layer_values(1), b.layer_values(1), rtol=1e-12)
