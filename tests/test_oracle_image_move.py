"""Pins of the oracle's image association (Sec. III-B: pinhole projection of cells and the
Bresenham visibility check), the robot-centric map move, and the harmonic fill. CPU only."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2309_16818_gb300 import synth

DOWN = np.array([[1.0, 0, 0], [0, -1.0, 0], [0, 0, -1.0]])  # optical axis = world -z


def cam_pose(R, pos):
    T = np.eye(4)
    T[:3, :3] = R
    T[:3, 3] = pos
    return T


def flat_map(W, res, height=0.0, layers=()):
    """A map whose every cell is valid at `height` (set through the oracle's own update)."""
    m = O.OracleMap(O.Params(W=W, res=res, layers=list(layers), range_max=1e6, gate_lambda=1e6))
    xs = (np.arange(W) - W // 2 + 0.5) * res
    X, Y = np.meshgrid(xs, xs)
    pts = np.column_stack([X.ravel(), Y.ravel(), np.full(W * W, height - 100.0)]).astype(np.float32)
    T = np.eye(4)
    T[2, 3] = 100.0
    m.fuse_points(pts, T)
    assert m.valid.all()
    return m


# --------------------------------------------------------------------------- Bresenham

@pytest.mark.parametrize("e", [(7, 3), (3, 7), (-3, 7), (-7, 3), (-7, -3), (-3, -7), (3, -7),
                               (7, -3), (9, 0), (0, -9), (5, 5), (-6, 6), (0, 0)])
def test_bresenham_path_properties(e):
    sx, sy = 2, -1
    ex, ey = sx + e[0], sy + e[1]
    P = O.bresenham(sx, sy, ex, ey)
    assert tuple(P[0]) == (sx, sy) and tuple(P[-1]) == (ex, ey)
    dx, dy = abs(ex - sx), abs(ey - sy)
    assert len(P) == max(dx, dy) + 1
    steps = np.diff(P, axis=0)
    assert np.all(np.abs(steps) <= 1) and np.all(np.abs(steps).sum(1) >= 1)
    # monotone along both axes and within half a cell of the ideal line in the minor axis
    assert np.all(steps[:, 0] * np.sign(ex - sx) >= 0) and np.all(steps[:, 1] * np.sign(ey - sy) >= 0)
    for x, y in P:
        if dx >= dy and dx > 0:
            yi = sy + (ey - sy) * (x - sx) / (ex - sx)
            assert abs(y - yi) <= 0.5 + 1e-12
        elif dy > 0:
            xi = sx + (ex - sx) * (y - sy) / (ey - sy)
            assert abs(x - xi) <= 0.5 + 1e-12


# --------------------------------------------------------------------------- projection

def test_known_cell_projects_to_known_pixel():
    W, res = 16, 0.25
    m = flat_map(W, res, height=0.5)
    j = 5 * W + 9
    xc = (9 - W // 2 + 0.5) * res
    yc = (5 - W // 2 + 0.5) * res
    K = (300.0, 300.0, 200.0, 120.0)
    T = cam_pose(DOWN, (xc, yc, 3.0))
    out = m.fuse_image(240, 400, [], K, T)
    assert out["vis"][j] == 1 and out["pix"][j] == 120 * 400 + 200
    # a cell offset by d along the camera x axis at depth Z projects to u = cx + fx d / Z
    for di in (-3, -1, 2, 4):
        jj = 5 * W + 9 + di
        u = 200.0 + 300.0 * (di * res) / 2.5
        assert out["pix"][jj] == 120 * 400 + math.floor(u + 0.5)


def test_flat_map_every_in_frustum_cell_visible():
    W, res = 32, 0.1
    m = flat_map(W, res, height=0.0)
    R = synth.rot_z(0.3) @ synth.rot_y(math.radians(35)) @ synth.R_BODY_OPTICAL
    pos = np.array([-1.2, -0.4, 1.1])
    K = (200.0, 200.0, 160.0, 120.0)
    out = m.fuse_image(240, 320, [], K, cam_pose(R, pos))
    n_checked = 0
    for iy in range(W):
        for ix in range(W):
            X = np.array([(ix - W // 2 + 0.5) * res, (iy - W // 2 + 0.5) * res, 0.0])
            Xc = R.T @ (X - pos)
            if Xc[2] <= 0.05:
                exp = 0
            else:
                u = K[0] * Xc[0] / Xc[2] + K[2]
                v = K[1] * Xc[1] / Xc[2] + K[3]
                if min(abs(u + 0.5 - round(u + 0.5)), abs(v + 0.5 - round(v + 0.5))) < 1e-3:
                    continue
                exp = int(0 <= math.floor(u + 0.5) < 320 and 0 <= math.floor(v + 0.5) < 240)
                if exp:
                    assert out["pix"][iy * W + ix] == math.floor(v + 0.5) * 320 + math.floor(u + 0.5)
            assert out["vis"][iy * W + ix] == exp
            n_checked += exp
    assert n_checked > 100


@pytest.mark.parametrize("D,hc,Hw", [(10, 2.0, 1.0), (6, 1.5, 0.5), (8, 3.0, 2.0)])
def test_wall_shadow_closed_form(D, hc, Hw):
    """A wall of height Hw, D cells from a camera at height hc on flat ground, hides the cells
    at distance e with D < e <= D hc / (hc - Hw) along the camera's row."""
    W, res = 64, 0.25
    m = flat_map(W, res, height=0.0)
    sx, sy = 10, 32
    wall = sx + D
    hv = m.h.reshape(W, W)
    hv[:, wall] = Hw
    R = synth.rot_y(math.radians(40)) @ synth.R_BODY_OPTICAL   # looking along +x, pitched down
    pos = np.array([(sx - W // 2 + 0.5) * res, (sy - W // 2 + 0.5) * res, hc])
    out = m.fuse_image(2000, 2000, [], (300.0, 300.0, 1000.0, 1000.0), cam_pose(R, pos))
    edge = D * hc / (hc - Hw)
    for e in range(D + 1, W - sx):
        j = sy * W + sx + e
        assert out["vis"][j] == (0 if e <= edge else 1), (e, edge)
    assert out["vis"][sy * W + wall] == 1  # the wall top itself is seen


def test_image_rules_on_visible_cells():
    W, res = 16, 0.25
    L = [O.Layer(4, O.GAUSS, var_meas=0.5), O.Layer(3, O.DIRICHLET, alpha0=0.5),
         O.Layer(3, O.CLASSMAX), O.Layer(4, O.EXPAVG, w=0.25)]
    m = flat_map(W, res, layers=L)
    rng = np.random.default_rng(0)
    H, Wi = 60, 80
    feat = rng.normal(size=(H * Wi, 4)).astype(np.float32)
    seg = synth.dirichlet_probs(rng, H * Wi, 3, 1.0)
    T = cam_pose(DOWN, (0.1, -0.2, 2.0))
    K = (40.0, 40.0, 40.0, 30.0)
    o1 = m.fuse_image(H, Wi, [(feat, [0, 3]), (seg, [1, 2])], K, T)
    vis = o1["vis"].astype(bool)
    assert vis.sum() > 50
    pix = o1["pix"][vis]
    np.testing.assert_allclose(m.layer_values(0)[vis], feat[pix], atol=1e-6)
    np.testing.assert_allclose(m.gauss_var(0)[vis], 0.5)
    np.testing.assert_allclose(m.layer_values(1)[vis], 0.5 + seg[pix], atol=1e-6)
    assert np.array_equal(m.layer_values(2)[vis][:, 0], np.argmax(seg[pix], axis=1))
    o2 = m.fuse_image(H, Wi, [(feat, [0, 3])], K, T)
    assert np.array_equal(o2["vis"], o1["vis"])
    # second identical observation: Gaussian variance halves, mean unchanged
    np.testing.assert_allclose(m.gauss_var(0)[vis], 0.25, rtol=1e-7)
    np.testing.assert_allclose(m.layer_values(0)[vis], feat[pix], atol=1e-6)
    assert not m.obs[0][~vis].any()


# --------------------------------------------------------------------------- move

def _filled(rng, W=16, res=0.25, layers=()):
    m = O.OracleMap(O.Params(W=W, res=res, layers=list(layers), gate_lambda=1e6))
    n = 2000
    pts = ((rng.integers(-40, 40, size=(n, 3)) + 0.5) * 0.0625).astype(np.float32)
    pts[:, 2] = -1.0 + 0.0625 * rng.integers(-3, 4, size=n)
    srcs = [(synth.dirichlet_probs(rng, n, 3, 0.5), list(range(len(layers))))] if layers else []
    T = np.eye(4)
    T[2, 3] = 1.0
    m.fuse_points(pts, T, srcs)
    return m, pts, srcs, T


def test_move_and_back_restores_interior():
    rng = np.random.default_rng(1)
    L = [O.Layer(3, O.DIRICHLET), O.Layer(3, O.EXPAVG)]
    m, *_ = _filled(rng, layers=L)
    W = 16
    h0, l0, o0 = m.h.copy(), m.layer[0].copy(), m.origin
    m.move((0.5, -0.75))       # shift (2, -3) cells
    assert m.origin == (0.5, -0.75)
    m.move((0.0, 0.0))
    assert m.origin == o0
    # new(ix, iy) = old(ix + 2, iy - 3), then back: cells with ix >= 2 and iy < W - 3 survive
    interior = np.zeros((W, W), bool)
    interior[:W - 3, 2:] = True
    interior = interior.ravel()
    assert np.array_equal(m.h[interior], h0[interior])
    assert np.array_equal(m.layer_values(0)[interior], l0.reshape(-1, 3)[interior])
    # cells that left and re-entered are reset
    assert not m.valid[~interior].any()
    assert np.all(m.layer_values(0)[~interior] == 1.0)


def test_fuse_then_move_equals_move_then_fuse():
    rng = np.random.default_rng(2)
    W = 16
    L = [O.Layer(3, O.LATEST)]
    a, pts, srcs, T = _filled(rng, layers=L)
    a.move((0.75, 0.25))
    b = O.OracleMap(O.Params(W=W, res=0.25, layers=L, gate_lambda=1e6))
    b.move((0.75, 0.25))
    b.fuse_points(pts, T, srcs)
    # cells seen in both frames (new map columns 0..W-4, rows 0..W-2)
    keep = np.zeros((W, W), bool)
    keep[:W - 1, :W - 3] = True
    keep = keep.ravel()
    assert np.array_equal(a.valid[keep], b.valid[keep])
    assert np.array_equal(a.h[keep], b.h[keep])
    assert np.array_equal(a.layer_values(0)[keep], b.layer_values(0)[keep])


# --------------------------------------------------------------------------- harmonic fill

def _hole(H, W, rng, frac=0.4, border=1):
    """Random known cells; with border > 0 the outer `border` rings are known too (border = 0
    leaves unknown cells on the crop border, where the fill is zero-flux)."""
    known = rng.random((H, W)) > frac
    if border > 0:
        known[:border] = known[-border:] = True
        known[:, :border] = known[:, -border:] = True
    return known


def test_harmonic_fill_reproduces_linear_fields():
    rng = np.random.default_rng(3)
    H, W = 24, 20
    y, x = np.mgrid[0:H, 0:W]
    f = 0.3 * x - 0.7 * y + 2.0
    known = _hole(H, W, rng)
    h = np.where(known, f, rng.normal(size=(H, W)))
    out, it, r = O.harmonic_fill(h, known, tol=1e-13)
    assert r <= 1e-13
    np.testing.assert_allclose(out, f, atol=1e-9)


def test_harmonic_fill_constant_and_maximum_principle():
    rng = np.random.default_rng(4)
    H, W = 20, 20
    known = _hole(H, W, rng, frac=0.6, border=0)
    known[0, 0] = True
    assert not known[0].all() and not known.all()  # unknown cells on the border
    c = np.full((H, W), 1.25)
    out, _, _ = O.harmonic_fill(np.where(known, c, 0.0), known, tol=1e-13)
    np.testing.assert_allclose(out, 1.25, atol=1e-10)
    g = rng.normal(size=(H, W))
    out, _, _ = O.harmonic_fill(np.where(known, g, 0.0), known, tol=1e-12)
    assert out.min() >= g[known].min() - 1e-9 and out.max() <= g[known].max() + 1e-9


def test_exact_harmonic_fill_pins():
    """The direct solve reproduces linear fields and constants, obeys the maximum principle and
    agrees with the Gauss-Seidel sweeps of the C oracle."""
    rng = np.random.default_rng(5)
    H, W = 40, 36
    y, x = np.mgrid[0:H, 0:W]
    f = -0.2 * x + 0.45 * y + 1.0
    known = _hole(H, W, rng, frac=0.5)
    out = O.harmonic_fill_exact(np.where(known, f, 7.0), known)
    np.testing.assert_allclose(out, f, atol=1e-10)
    g = rng.normal(size=(H, W))
    known = _hole(H, W, rng, frac=0.6, border=0)
    known[5, 5] = True
    ex = O.harmonic_fill_exact(np.where(known, g, 0.0), known)
    gs, _, r = O.harmonic_fill(np.where(known, g, 0.0), known, tol=1e-13)
    np.testing.assert_allclose(ex, gs, atol=1e-9)
    assert ex.min() >= g[known].min() - 1e-12 and ex.max() <= g[known].max() + 1e-12
    # a group of unknown cells with no known neighbour keeps the mean of the known cells
    kn = np.zeros((8, 8), bool)
    kn[:, :2] = True
    kn[:, 2] = False
    kn[4, 2] = False
    h0 = np.arange(64, dtype=float).reshape(8, 8)
    out = O.harmonic_fill_exact(h0, kn)
    np.testing.assert_allclose(out[kn], h0[kn])


@pytest.mark.parametrize("above,seen", [(0.04, 0), (0.06, 1)])
def test_near_plane_is_strict(above, seen):
    """A cell is projected only when it lies more than z_near (0.05 m) in front of the camera."""
    W, res = 16, 0.25
    m = flat_map(W, res, height=0.5)
    j = 5 * W + 9
    xc = (9 - W // 2 + 0.5) * res
    yc = (5 - W // 2 + 0.5) * res
    out = m.fuse_image(240, 400, [], (300.0, 300.0, 200.0, 120.0), cam_pose(DOWN, (xc, yc, 0.5 + above)))
    assert out["vis"][j] == seen
    if seen:
        assert out["pix"][j] == 120 * 400 + 200


def test_invalid_cells_never_occlude():
    """Only valid cells can hide a cell (an unobserved cell has no height); a tall stale value in an
    invalid cell on the walk changes nothing, the same value in a valid cell hides the target."""
    W, res = 64, 0.25
    m = flat_map(W, res, height=0.0)
    sx, sy, hc = 10, 32, 2.0
    R = synth.rot_y(math.radians(40)) @ synth.R_BODY_OPTICAL   # looking along +x, pitched down
    pos = np.array([(sx - W // 2 + 0.5) * res, (sy - W // 2 + 0.5) * res, hc])
    T = cam_pose(R, pos)
    K = (300.0, 300.0, 1000.0, 1000.0)
    j, q = sy * W + sx + 12, sy * W + sx + 6
    assert m.fuse_image(2000, 2000, [], K, T)["vis"][j] == 1
    m.h[q] = 100.0
    assert m.fuse_image(2000, 2000, [], K, T)["vis"][j] == 0
    m.valid[q] = 0
    assert m.fuse_image(2000, 2000, [], K, T)["vis"][j] == 1


def test_camera_outside_the_map_walks_from_the_clamped_edge_cell():
    """The camera's cell is clamped into the map: a camera beyond the +x edge walks from the edge
    cell, which is an end of every walk and so never occludes, even when it is a wall."""
    W, res = 64, 0.25
    m = flat_map(W, res, height=0.0)
    sy, hc = 32, 2.0
    hv = m.h.reshape(W, W)
    hv[:, W - 1] = 1.0  # a wall along the edge column
    R = synth.rot_z(math.pi) @ synth.rot_y(math.radians(40)) @ synth.R_BODY_OPTICAL  # looking along -x
    pos = np.array([(W // 2) * res + 0.5, (sy - W // 2 + 0.5) * res, hc])
    out = m.fuse_image(2000, 2000, [], (300.0, 300.0, 1000.0, 1000.0), cam_pose(R, pos))
    for x in range(W - 12, W - 1):
        assert out["vis"][sy * W + x] == 1, x


def test_move_rounds_to_the_nearest_cell_and_keeps_counts():
    rng = np.random.default_rng(6)
    L = [O.Layer(3, O.LATEST)]
    m, *_ = _filled(rng, layers=L)
    W, res = 16, 0.25
    a0, r0, h0 = m.n_acc.copy().reshape(W, W), m.n_rej.copy().reshape(W, W), m.h.copy().reshape(W, W)
    m.move((0.7 * res, -0.6 * res))  # 0.7 and -0.6 cells round to (1, -1)
    assert m.origin == (res, -res)
    a, r, h = m.n_acc.reshape(W, W), m.n_rej.reshape(W, W), m.h.reshape(W, W)
    # new (ix, iy) = old (ix + 1, iy - 1)
    assert np.array_equal(a[1:, :W - 1], a0[:W - 1, 1:])
    assert np.array_equal(r[1:, :W - 1], r0[:W - 1, 1:])
    assert np.array_equal(h[1:, :W - 1], h0[:W - 1, 1:])
    assert a0.sum() > 0
