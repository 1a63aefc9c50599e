"""Pins of the oracle's post-processing plugins: surface normals of the elevation layer
(Table I "normal calculation") and the PCA layer of a feature layer (Sec. III-D) against
closed forms and invariants. CPU only."""
import numpy as np
import pytest

import oracle as O
from oracle import plugins as PL

W, RES = 16, 0.25


def plane_map(f, valid=None):
    m = O.OracleMap(O.Params(W=W, res=RES), round_store=True)
    iy, ix = np.mgrid[0:W, 0:W]
    x = (ix - W // 2 + 0.5) * RES
    y = (iy - W // 2 + 0.5) * RES
    m.h[:] = np.float32(f(x, y)).ravel()
    m.valid[:] = 1 if valid is None else valid.ravel()
    return m, x.ravel(), y.ravel()


def test_plane_normals_closed_form():
    """On h = 0.3 x - 0.2 y + 1 every cell, border cells included, has the normal
    (-0.3, 0.2, 1) / sqrt(1.13) (central and one-sided differences are exact on a plane)."""
    m, _, _ = plane_map(lambda x, y: 0.3 * x - 0.2 * y + 1.0)
    n, ok = m.normals()
    assert ok.all()
    exp = np.array([-0.3, 0.2, 1.0]) / np.sqrt(1.13)
    assert np.allclose(n, exp, rtol=0, atol=2e-5)
    assert np.allclose(np.linalg.norm(n, axis=1), 1.0, atol=1e-6)


def test_quadratic_central_and_one_sided_slopes():
    """On h = x^2 the central slope at x is 2x, the forward one 2x + res, the backward one
    2x - res: a missing left neighbour selects the forward difference, a missing right one
    the backward difference."""
    m, x, _ = plane_map(lambda x, y: x * x)
    j = 5 * W + 6
    xj = x[j]
    def gx_of(n):
        return -n[0] / n[2]
    n, ok = m.normals()
    assert ok[j] and gx_of(n[j]) == pytest.approx(2 * xj, abs=1e-4)
    m.valid[j - 1] = 0
    n, ok = m.normals()
    assert gx_of(n[j]) == pytest.approx(2 * xj + RES, abs=1e-4)
    m.valid[j - 1] = 1
    m.valid[j + 1] = 0
    n, ok = m.normals()
    assert gx_of(n[j]) == pytest.approx(2 * xj - RES, abs=1e-4)
    # the map edges use the one-sided differences
    n, ok = plane_map(lambda x, y: x * x)[0].normals()
    assert gx_of(n[3 * W]) == pytest.approx(2 * x[3 * W] + RES, abs=1e-4)
    assert gx_of(n[3 * W + W - 1]) == pytest.approx(2 * x[3 * W + W - 1] - RES, abs=1e-4)


def test_normals_need_a_neighbour_on_each_axis():
    valid = np.zeros((W, W), np.uint8)
    valid[4, 3:8] = 1      # a row: no neighbour along y
    valid[9:12, 9] = 1     # a column: no neighbour along x
    valid[2:4, 12:14] = 1  # a 2x2 block: neighbours both ways
    m, _, _ = plane_map(lambda x, y: 0.1 * x, valid)
    n, ok = m.normals()
    assert ok.reshape(W, W)[4].sum() == 0 and ok.reshape(W, W)[:, 9].sum() == 0
    assert ok.sum() == 4 and np.all(n[ok == 0] == 0)


def _subspace_features(rng, n, d=64, lam=(9.0, 4.0, 1.0)):
    """n points f = mean + A z: A has orthonormal columns, z has zero mean, uncorrelated
    columns and sample variances lam exactly."""
    A, _ = np.linalg.qr(rng.normal(size=(d, 3)))
    z = rng.normal(size=(n, 3))
    z -= z.mean(axis=0)
    q, _ = np.linalg.qr(z)                      # orthonormal, zero-mean columns
    z = q * np.sqrt(np.array(lam) * n)          # sample variance lam_k, uncorrelated
    mean = rng.normal(size=d)
    return mean + z @ A.T, A, z, mean


def test_pca_recovers_a_known_subspace():
    """Features on a 3-D affine subspace with variances 9, 4, 1 along orthonormal axes: the
    eigenvalues are exactly 9, 4, 1, the vectors are the axes up to sign, the projections are
    the subspace coordinates (same sign), the mean is the offset."""
    rng = np.random.default_rng(1)
    f, A, z, mean = _subspace_features(rng, 500)
    obs = np.ones(500, bool)
    proj, w, V, m = PL.pca_of_features(f, obs)
    assert np.allclose(w, [9.0, 4.0, 1.0], rtol=1e-10)
    assert np.allclose(m, mean, atol=1e-12)
    for k in range(3):
        s = np.sign(V[k] @ A[:, k])
        assert np.allclose(V[k], s * A[:, k], atol=1e-10)
        assert np.allclose(proj[:, k], s * z[:, k], atol=1e-9)


def test_pca_sign_convention_and_unobserved_cells():
    rng = np.random.default_rng(2)
    f, _, _, _ = _subspace_features(rng, 300, d=16)
    obs = rng.random(300) < 0.7
    proj, w, V, m = PL.pca_of_features(f, obs)
    for k in range(3):
        i = int(np.argmax(np.abs(V[k])))
        assert V[k, i] > 0
    assert np.all(proj[~obs] == 0)
    # values in unobserved cells change nothing
    g = f.copy()
    g[~obs] = 1e6
    proj2, w2, V2, m2 = PL.pca_of_features(g, obs)
    assert np.array_equal(proj2, proj) and np.array_equal(V2, V)
    # the cells' order does not matter
    perm = rng.permutation(300)
    proj3, w3, V3, _ = PL.pca_of_features(f[perm], obs[perm])
    assert np.allclose(proj3, proj[perm], atol=1e-9) and np.allclose(w3, w, rtol=1e-12)


def test_pca_of_nothing_observed():
    proj, w, V, m = PL.pca_of_features(np.ones((10, 4)), np.zeros(10, bool))
    assert np.all(proj == 0) and np.all(w == 0)
