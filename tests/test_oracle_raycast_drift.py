"""Pins of the oracle's drift compensation and ray-cast clean-up (Table I rows "drift
compensation" and "height update & ray cast"; the paper defers both to its predecessor, so
the readings are the ones stated in the design notes) against closed forms, boundary cases
and invariants. CPU only.

Scene used below: W = 16 cells of 0.5 m, sensor 1 m above the map centre (sensor cell (8, 8)),
every cell valid at height 0 with variance 1e-4 unless a test says otherwise."""
import numpy as np
import pytest

import oracle as O

W, RES = 16, 0.5


def ident(t=(0.0, 0.0, 1.0)):
    T = np.eye(4)
    T[:3, 3] = t
    return T


def flat_map(var=1e-4, **kw):
    m = O.OracleMap(O.Params(W=W, res=RES, **kw), round_store=True)
    m.h[:] = 0.0
    m.var[:] = var
    m.valid[:] = 1
    return m


def cell(ix, iy):
    return iy * W + ix


def map_z(z):
    """Map-frame height of a ground_point at height z: one float32 rounding of (z - 1) + 1."""
    return float(np.float32(np.float32(z - 1.0) + np.float32(1.0)))


def ground_point(ix, iy, z=0.0, dx=0.25, dy=0.25):
    """Sensor-frame point at the given map position inside cell (ix, iy) (sensor at (0, 0, 1))."""
    return [(ix - W // 2) * RES + dx, (iy - W // 2) * RES + dy, z - 1.0]


# --------------------------------------------------------------------------- ray-cast clean-up

def test_phantom_obstacle_on_the_ray_is_cleared():
    """A ground point in cell (14, 8) casts its ray from (8, 8) at height 1 down to height 0;
    at cell (11, 8) the ray parameter is t = 18/36 = 1/2, the ray height 0.5. An obstacle of
    0.7 m there (0.2 m above the ray, margin 0.1) is stale and becomes invalid; every other
    cell keeps its state."""
    m = flat_map(ray_cleanup=True, ray_margin=0.1)
    q = cell(11, 8)
    m.h[q] = 0.7
    r = m.fuse_points(np.array([ground_point(14, 8)], np.float32), ident())
    assert r["cleared"] == 1
    assert m.valid[q] == 0
    assert m.valid.sum() == W * W - 1
    assert m.n_acc[cell(14, 8)] == 1


@pytest.mark.parametrize("H,cleared", [(0.601, 1), (0.599, 0), (0.5, 0), (5.0, 1)])
def test_margin_boundary(H, cleared):
    """Cleared iff the cell's height exceeds the ray height (0.5 at t = 1/2) by more than the
    margin (0.1): 0.601 is cleared, 0.599 and the ray height itself are not."""
    m = flat_map(ray_cleanup=True, ray_margin=0.1)
    q = cell(11, 8)
    m.h[q] = H
    r = m.fuse_points(np.array([ground_point(14, 8)], np.float32), ident())
    assert r["cleared"] == cleared and m.valid[q] == 1 - cleared


def test_ray_height_at_other_parameters():
    """Cells (9, 8) .. (13, 8) have t = 1/6 .. 5/6 and ray heights 1 - t: an obstacle 0.15 m
    above the ray height is cleared wherever it stands, one 0.05 m above it nowhere."""
    for k in range(1, 6):
        t = k / 6.0
        for above, exp in ((0.15, 0), (0.05, 1)):
            m = flat_map(ray_cleanup=True, ray_margin=0.1)
            q = cell(8 + k, 8)
            m.h[q] = (1.0 - t) + above
            m.fuse_points(np.array([ground_point(14, 8)], np.float32), ident())
            assert m.valid[q] == exp, (k, above)


def test_ray_ends_at_the_point_not_at_its_cell():
    """The point's cell holds 0.3 m with a wide variance, so the ground point (0 m) is accepted;
    its ray still ends at the point: 0.5 m at t = 1/2 (a ray ending at the cell's 0.3 m would
    be 0.65 m there), so a 0.7 m obstacle is cleared."""
    m = flat_map(ray_cleanup=True, ray_margin=0.1)
    e, q = cell(14, 8), cell(11, 8)
    m.h[e] = 0.3
    m.var[e] = 1.0
    m.h[q] = 0.7
    m.fuse_points(np.array([ground_point(14, 8)], np.float32), ident())
    assert m.n_acc[e] == 1 and m.valid[q] == 0


def test_cell_that_accepts_a_point_is_not_cleared():
    """The stale cell also receives a point: rejected by its gate (0 m against 0.7 m), the
    cell is still cleared; with a wide prior variance the point is accepted and the cell
    keeps its (updated) height."""
    q = cell(11, 8)
    pts = np.array([ground_point(14, 8), ground_point(11, 8)], np.float32)
    m = flat_map(ray_cleanup=True, ray_margin=0.1)
    m.h[q] = 0.7
    m.fuse_points(pts, ident())
    assert m.n_rej[q] == 1 and m.valid[q] == 0
    m = flat_map(ray_cleanup=True, ray_margin=0.1)
    m.h[q] = 0.7
    m.var[q] = 1.0
    m.fuse_points(pts, ident())
    assert m.n_acc[q] == 1 and m.valid[q] == 1 and m.h[q] < 0.7


def test_rejected_points_cast_no_ray():
    """A point 1 m below a valid cell at 0 m is an outlier of its cell: it casts no ray, so
    the obstacle its ray would pass stays."""
    m = flat_map(ray_cleanup=True, ray_margin=0.1)
    q = cell(11, 8)
    m.h[q] = 0.7
    r = m.fuse_points(np.array([ground_point(14, 8, z=-1.0)], np.float32), ident())
    assert m.n_rej[cell(14, 8)] == 1
    assert r["cleared"] == 0 and m.valid[q] == 1


def test_invalid_cells_and_line_ends_are_never_cleared():
    """An invalid cell on the ray stays invalid (nothing to clear); obstacles in the sensor's
    cell and in the point's own cell are not intermediate cells of the walk."""
    m = flat_map(ray_cleanup=True, ray_margin=0.1)
    q = cell(11, 8)
    m.h[q] = 0.7
    m.valid[q] = 0
    m.h[cell(8, 8)] = 5.0
    r = m.fuse_points(np.array([ground_point(14, 8)], np.float32), ident())
    assert r["cleared"] == 0 and m.valid[cell(8, 8)] == 1 and m.valid[q] == 0
    # the endpoint: a cell whose point is rejected is still not its own ray's intermediate cell
    m = flat_map(ray_cleanup=True, ray_margin=0.1)
    e = cell(14, 8)
    m.h[e] = 3.0
    r = m.fuse_points(np.array([ground_point(14, 8)], np.float32), ident())
    assert m.n_rej[e] == 1 and m.valid[e] == 1 and r["cleared"] == 0


def test_cleanup_off_changes_nothing():
    m = flat_map(ray_cleanup=False)
    q = cell(11, 8)
    m.h[q] = 0.7
    r = m.fuse_points(np.array([ground_point(14, 8)], np.float32), ident())
    assert r["cleared"] == 0 and m.valid[q] == 1


def test_diagonal_ray_uses_the_bresenham_cells():
    """Ray from (8, 8) to (12, 11): the error-term walk (dx = 4, dy = -3, err = 1) steps
    diagonally, diagonally, along x, diagonally, so the intermediate cells are (9, 9),
    (10, 10), (11, 10); an obstacle next to the line but not on it is untouched."""
    line = [tuple(int(v) for v in x) for x in O.bresenham(8, 8, 12, 11)]
    assert line == [(8, 8), (9, 9), (10, 10), (11, 10), (12, 11)]
    for ix, iy in line[1:-1] + [(10, 9), (9, 8), (11, 11)]:
        m = flat_map(ray_cleanup=True, ray_margin=0.1)
        m.h[cell(ix, iy)] = 2.0
        m.fuse_points(np.array([ground_point(12, 11)], np.float32), ident())
        on_line = (ix, iy) in line
        assert m.valid[cell(ix, iy)] == (0 if on_line else 1), (ix, iy)


def test_diagonal_ray_parameter_by_hand():
    """Along the ray (8, 8) -> (12, 11) (e - s = (4, 3), |e - s|^2 = 25) the intermediate cells
    (9, 9), (10, 10), (11, 10) have t = 7/25, 14/25, 18/25 and ray heights 1 - t = 0.72, 0.44,
    0.28: an obstacle 0.15 m above that height is cleared, one 0.05 m above it is not."""
    for (ix, iy), t in (((9, 9), 7 / 25), ((10, 10), 14 / 25), ((11, 10), 18 / 25)):
        for above, exp in ((0.15, 0), (0.05, 1)):
            m = flat_map(ray_cleanup=True, ray_margin=0.1)
            m.h[cell(ix, iy)] = (1.0 - t) + above
            m.fuse_points(np.array([ground_point(12, 11)], np.float32), ident())
            assert m.valid[cell(ix, iy)] == exp, ((ix, iy), above)


def test_cleared_cells_do_not_age():
    m = flat_map(ray_cleanup=True, ray_margin=0.1, time_var=0.5)
    q = cell(11, 8)
    m.h[q] = 0.7
    m.fuse_points(np.array([ground_point(14, 8)], np.float32), ident())
    assert m.valid[q] == 0 and m.var[q] == pytest.approx(1e-4)
    assert m.var[cell(2, 2)] == pytest.approx(1e-4 + 0.5)


def test_union_of_rays_and_order_invariance():
    """From the same state, fusing A and B together clears exactly the cells that A alone or
    B alone clears, except cells that accept a point of A or B; permuting the points changes
    nothing."""
    rng = np.random.default_rng(5)
    h0 = rng.uniform(0.0, 0.6, W * W)
    def run(pts):
        m = flat_map(ray_cleanup=True, ray_margin=0.1, gate_lambda=3.0)
        m.h[:] = h0
        m.var[:] = 0.02
        m.fuse_points(pts, ident())
        return m
    def cloud(n):
        xy = rng.uniform(-3.9, 3.9, size=(n, 2))
        z = rng.uniform(-0.2, 0.3, size=(n, 1)) - 1.0
        return np.hstack([xy, z]).astype(np.float32)
    A, B = cloud(60), cloud(60)
    ma, mb, mab = run(A), run(B), run(np.concatenate([A, B]))
    cleared = lambda m: (m.valid == 0)
    accepted = mab.n_acc > 0
    exp = (cleared(ma) | cleared(mb)) & ~accepted
    assert np.array_equal(cleared(mab), exp)
    assert cleared(mab).sum() > 3
    perm = rng.permutation(120)
    mp = run(np.concatenate([A, B])[perm])
    assert np.array_equal(mp.valid, mab.valid) and np.allclose(mp.h, mab.h, rtol=1e-12)


# --------------------------------------------------------------------------- drift compensation

def test_drift_closed_form_flat_plane():
    """Every cell valid at 0 m; 20 points at 0.01 m in 20 cells: the mean error is 0.01, so
    with alpha = 1 the whole map moves up by float32(0.01) before the height update; untouched
    cells end exactly there, touched cells stay at the plane."""
    m = flat_map(drift_alpha=1.0, drift_min_points=1)
    pts = np.array([ground_point(2 + k % 10, 3 + k // 10, z=0.01) for k in range(20)], np.float32)
    r = m.fuse_points(pts, ident())
    assert r["drift_points"] == 20
    assert r["drift"] == map_z(0.01)
    assert m.h[cell(0, 0)] == r["drift"] and m.h[cell(15, 15)] == r["drift"]
    touched = [cell(2 + k % 10, 3 + k // 10) for k in range(20)]
    assert np.allclose(m.h[touched], 0.01, atol=1e-7)


@pytest.mark.parametrize("alpha", [0.5, -1.0])
def test_drift_scales_with_alpha(alpha):
    m = flat_map(drift_alpha=alpha)
    pts = np.array([ground_point(2 + k, 4, z=0.02) for k in range(10)], np.float32)
    r = m.fuse_points(pts, ident())
    e = map_z(0.02)
    assert r["drift"] == float(np.float32(alpha * e))
    assert m.h[cell(0, 0)] == float(np.float32(alpha * e))


def test_drift_ignores_outliers_and_invalid_cells():
    """Points that their cell's gate rejects, and points in invalid cells, do not enter the
    mean error."""
    m = flat_map(drift_alpha=1.0)
    m.valid[cell(12, 12)] = 0
    good = [ground_point(2 + k, 4, z=0.01) for k in range(10)]
    outl = [ground_point(2 + k, 6, z=0.5) for k in range(5)]        # 0.5 m off: rejected
    inval = [ground_point(12, 12, z=0.01)] * 3                       # invalid cell
    r = m.fuse_points(np.array(good + outl + inval, np.float32), ident())
    assert r["drift_points"] == 10
    assert r["drift"] == map_z(0.01)
    assert m.n_rej[cell(3, 6)] == 1


def test_drift_needs_enough_points():
    m = flat_map(drift_alpha=1.0, drift_min_points=11)
    pts = np.array([ground_point(2 + k, 4, z=0.01) for k in range(10)], np.float32)
    r = m.fuse_points(pts, ident())
    assert r["drift"] == 0.0 and m.h[cell(0, 0)] == 0.0 and r["drift_points"] == 10
    m = flat_map(drift_alpha=1.0, drift_min_points=10)
    r = m.fuse_points(pts, ident())
    assert r["drift"] != 0.0 and m.h[cell(0, 0)] == r["drift"]


def test_height_update_gates_against_the_shifted_map():
    """40 points at 0.02 m shift the map by 0.02; a point at 0.045 m in cell (9, 9) (range
    1.45 m, sigma_m 0.0129 m, lambda 3: threshold 9 (1e-6 + 1.67e-4) = 1.5e-3 m^2) is an
    outlier of the unshifted cell (0.045^2 = 2.0e-3) but not of the shifted one
    (0.025^2 = 6.3e-4): rejected without drift compensation, accepted with it."""
    pts = [ground_point(2 + k % 10, 3 + k // 10, z=0.02) for k in range(40)]
    pts.append(ground_point(9, 9, z=0.045))
    pts = np.array(pts, np.float32)
    q = cell(9, 9)
    m0 = flat_map(var=1e-6, gate_lambda=3.0)
    m0.fuse_points(pts, ident())
    assert m0.n_rej[q] == 1
    m1 = flat_map(var=1e-6, gate_lambda=3.0, drift_alpha=1.0)
    r = m1.fuse_points(pts, ident())
    assert r["drift_points"] == 40 and m1.n_acc[q] == 1 and m1.n_rej[q] == 0


def test_drift_off_or_empty_cloud_moves_nothing():
    m = flat_map(drift_alpha=1.0)
    r = m.fuse_points(np.zeros((0, 3), np.float32), ident())
    assert r["drift"] == 0.0 and r["drift_points"] == 0 and np.all(m.h == 0)
    m = flat_map(drift_alpha=0.0)
    r = m.fuse_points(np.array([ground_point(3, 3, z=0.01)], np.float32), ident())
    assert r["drift"] == 0.0 and m.h[cell(0, 0)] == 0.0
