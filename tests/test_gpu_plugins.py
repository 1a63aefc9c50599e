"""CUDA post-processing plugins against the oracle through the C ABI: surface normals of the
elevation layer (bit-exact: the same float32 sequence) and the PCA layer of a feature layer
(float32 sums and Jacobi sweeps against float64 numpy, at tolerances set by the spectrum)."""
import numpy as np
import pytest

import oracle as O
from oracle import plugins as PL
from paper_2309_16818_gb300 import synth

from helpers import cuda_xyz, make_pair, upload_state

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def test_normals_equal_the_oracle_after_moves(torch):
    """Two fused poses with a move between them (ring-buffer offsets), then normals of every
    cell: vectors and the ok mask bit-exact."""
    c = synth.config2(n_poses=2, scale=0.25)
    g, o = make_pair(c["W"], c["res"], [])
    for k, scan in enumerate(c["scans"]):
        o.move(c["poses"][k][:2])
        g.move(c["poses"][k][:2])
        o.fuse_points(scan.xyz, scan.T)
        upload_state(g, o)
    n, ok = g.normals()
    on, ook = o.normals()
    assert ook.sum() > 5000
    assert np.array_equal(ok.cpu().numpy(), ook)
    assert np.array_equal(n.cpu().numpy().view(np.uint32), on.view(np.uint32))


def _designed_features(rng, cells, C, lam=(9.0, 4.0, 1.0), noise=0.05):
    A, _ = np.linalg.qr(rng.normal(size=(C, 3)))
    z = rng.normal(size=(cells, 3)) * np.sqrt(lam)
    mean = rng.normal(size=C)
    return (mean + z @ A.T + noise * rng.normal(size=(cells, C))).astype(np.float32)


@pytest.mark.parametrize("C,dtype", [(16, O.F32), (64, O.F32), (64, O.BF16), (128, O.F32)])
def test_pca_matches_the_oracle(torch, C, dtype):
    """A feature layer set to features with principal variances 9, 4, 1 (plus small noise) on
    70 % of the cells of a moved 120 x 120 map: eigenvalues within 1e-4 relative, vectors within
    1e-3 after aligning signs (and signed by the same rule), projections within 1e-3 of their
    scale; unobserved cells 0."""
    from paper_2309_16818_gb300 import mem as M
    from helpers import torch_dt
    W = 120
    rng = np.random.default_rng(C)
    g, o = make_pair(W, 0.05, [dict(channels=C, rule=O.GAUSS, dtype=dtype)])
    g.move((0.33, -0.41))
    o.move((0.33, -0.41))
    f = _designed_features(rng, W * W, C)
    obs = (rng.random(W * W) < 0.7).astype(np.uint8)
    fv = torch.from_numpy(f).to(torch_dt(dtype)).cuda()
    g.set_layer(0, fv.contiguous())
    g.set_layer(0, torch.from_numpy(obs).cuda(), part=M.PART_OBSERVED)
    stored = fv.float().cpu().numpy().astype(np.float64)   # the values the layer holds
    proj, vals, vecs, mean = g.pca(0, 3)
    proj, vals, vecs, mean = (t.cpu().numpy().astype(np.float64) for t in (proj, vals, vecs, mean))
    op, ow, oV, om = PL.pca_of_features(stored, obs.astype(bool), 3)
    assert np.allclose(vals, ow, rtol=1e-4)
    assert np.allclose(mean, om, atol=1e-5 * (1 + np.abs(om).max()))
    for k in range(3):
        s = np.sign(vecs[k] @ oV[k])
        assert s > 0, "sign convention"
        assert np.allclose(vecs[k], oV[k], atol=1e-3)
        scale = np.sqrt(ow[k])
        assert np.abs(proj[:, k] - op[:, k]).max() <= 1e-3 * scale * 10
    assert np.all(proj[obs == 0] == 0)


def test_pca_on_fused_camera_features(torch):
    """The PCA of a 64-d feature layer filled by a camera (smooth random features): the top
    eigenvalues within 1e-3 relative of the oracle's on the same layer values, and the
    projections' subspace error bounded by the spectral gap."""
    from paper_2309_16818_gb300 import mem as M
    c = synth.config2(n_poses=1, scale=0.25)
    g, o = make_pair(c["W"], c["res"], [dict(channels=64, rule=O.GAUSS)])
    scan = c["scans"][0]
    o.move(c["poses"][0][:2])
    g.move(c["poses"][0][:2])
    g.fuse_pointcloud(cuda_xyz(scan), scan.T)
    cam = synth.cameras_around(3, c["poses"][0], c["terrain"], H=240, Wi=424, n_feat=64)[0]
    g.fuse_image(cam.H, cam.Wi, cam.K, cam.T, [(torch.from_numpy(cam.feat).cuda(), [0])])
    vals_layer = g.get_layer(0).cpu().numpy().astype(np.float64)
    obs = g.get_layer(0, part=M.PART_OBSERVED).cpu().numpy().astype(bool)
    assert obs.sum() > 1000
    proj, vals, vecs, mean = (t.cpu().numpy().astype(np.float64) for t in g.pca(0, 3))
    op, ow, oV, om = PL.pca_of_features(vals_layer, obs, 3)
    assert np.allclose(vals, ow, rtol=1e-3)
    # each GPU vector lies in the oracle's top subspace up to the gap-limited mixing
    full = np.linalg.eigvalsh(np.cov((vals_layer[obs] - om).T, bias=True))[::-1]
    gap = min(full[k] - full[k + 1] for k in range(3)) / full[0]
    for k in range(3):
        resid = vecs[k] - oV.T @ (oV @ vecs[k])
        assert np.linalg.norm(resid) <= max(1e-3, 1e-5 / gap), (k, gap)
