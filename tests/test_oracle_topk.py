"""Pins of the oracle's top-k class input (Sec. III-C: class probabilities may be given as the
top k classes of each point or pixel, to save memory): a source of (class id, probability)
pairs must fuse exactly as the dense K-vector that holds those probabilities and zeros
elsewhere, under every rule, for point clouds and images. CPU only."""
import numpy as np
import pytest

import oracle as O
from paper_2309_16818_gb300 import synth

K = 7


def dense_of(pairs, K):
    """The dense rows a top-k source stands for, written out directly (no duplicates here)."""
    out = np.zeros((pairs.shape[0], K), np.float32)
    for i, row in enumerate(pairs):
        for j in range(0, len(row), 2):
            out[i, int(row[j])] = row[j + 1]
    return out


def layers():
    return [O.Layer(K, O.LATEST), O.Layer(K, O.EXPAVG, w=0.3), O.Layer(K, O.DIRICHLET, alpha0=0.5),
            O.Layer(K, O.CLASSMAX), O.Layer(K, O.GAUSS, var_meas=0.5)]


def states_equal(a, b):
    assert np.array_equal(a.valid, b.valid) and np.array_equal(a.h, b.h)
    for l in range(len(a.p.layers)):
        assert np.array_equal(a.layer[l], b.layer[l]), l
        assert np.array_equal(a.obs[l], b.obs[l]), l
        assert np.array_equal(a.lvar[l], b.lvar[l]), l


@pytest.mark.parametrize("k", [1, 3, K])
def test_topk_points_equal_the_dense_vector(k):
    rng = np.random.default_rng(k)
    n = 400
    pts = np.column_stack([rng.uniform(-1.9, 1.9, size=(n, 2)), np.full(n, -1.0)]).astype(np.float32)
    probs = synth.dirichlet_probs(rng, n, K, 0.4)
    pairs = synth.topk_pairs(probs, k)
    T = np.eye(4)
    T[2, 3] = 1.0
    a = O.OracleMap(O.Params(W=8, res=0.5, layers=layers()))
    b = O.OracleMap(O.Params(W=8, res=0.5, layers=layers()))
    for rep in range(2):
        a.fuse_points(pts, T, [(O.TopK(pairs, K), [0, 1, 2, 3, 4])])
        b.fuse_points(pts, T, [(dense_of(pairs, K), [0, 1, 2, 3, 4])])
    states_equal(a, b)
    if k == K:  # every class listed: the full probability vector itself
        c = O.OracleMap(O.Params(W=8, res=0.5, layers=layers()))
        for rep in range(2):
            c.fuse_points(pts, T, [(probs, [0, 1, 2, 3, 4])])
        states_equal(a, c)


def test_repeated_ids_add_and_invalid_ids_are_ignored():
    """Row (2, 0.25) (2, 0.5) (-1, 9) (7, 9) (2.5, 9) (nan, 9) (0, 0.125): class 2 gets 0.75,
    class 0 0.125, the rest nothing (ids must be whole numbers in [0, 7))."""
    row = np.array([[2, 0.25, 2, 0.5, -1, 9, 7, 9, 2.5, 9, np.nan, 9, 0, 0.125]], np.float32)
    m = O.OracleMap(O.Params(W=8, res=0.5, layers=[O.Layer(K, O.LATEST)]), round_store=False)
    T = np.eye(4)
    T[2, 3] = 1.0
    m.fuse_points(np.array([[0.2, 0.2, -1.0]], np.float32), T, [(O.TopK(row, K), [0])])
    v = m.layer_values(0)[36]
    assert list(v) == [0.125, 0, 0.75, 0, 0, 0, 0]


def test_one_hot_top1_votes_count_exactly():
    """N top-1 inputs (c, 1.0) into a Dirichlet layer: alpha_c = alpha0 + N, others alpha0."""
    m = O.OracleMap(O.Params(W=8, res=0.5, layers=[O.Layer(K, O.DIRICHLET, alpha0=1.0)]), round_store=False)
    T = np.eye(4)
    T[2, 3] = 1.0
    pts = np.array([[0.2, 0.2, -1.0]] * 5, np.float32)
    pairs = np.array([[3, 1.0]] * 5, np.float32)
    m.fuse_points(pts, T, [(O.TopK(pairs, K), [0])])
    assert list(m.layer_values(0)[36]) == [1, 1, 1, 6, 1, 1, 1]


def test_topk_pixels_equal_the_dense_image():
    """Image fusion with a top-k pixel source equals the dense image of the same values."""
    rng = np.random.default_rng(3)
    W, res = 16, 0.25
    T = np.eye(4)
    T[2, 3] = 0.6
    pts = np.column_stack([rng.uniform(-1.9, 1.9, size=(800, 2)), rng.uniform(-0.65, -0.55, 800)]).astype(np.float32)
    H, Wi = 24, 32
    probs = synth.dirichlet_probs(rng, H * Wi, K, 0.4)
    pairs = synth.topk_pairs(probs, 2)
    Kc = np.array([20.0, 20.0, 16.0, 12.0])
    Tc = np.eye(4)
    Tc[:3, :3] = [[0, 0, 1], [-1, 0, 0], [0, -1, 0]]   # optical z along world +x
    Tc[:3, :3] = Tc[:3, :3].T
    Tc[:3, 3] = [-2.0, 0.0, 1.0]
    out = []
    for src in (O.TopK(pairs, K), dense_of(pairs, K)):
        m = O.OracleMap(O.Params(W=W, res=res, layers=layers()))
        m.fuse_points(pts, T)
        r = m.fuse_image(H, Wi, [(src, [0, 1, 2, 3, 4])], Kc, Tc)
        out.append((m, r))
    assert out[0][1]["n_visible"] >= 5
    assert np.array_equal(out[0][1]["vis"], out[1][1]["vis"])
    states_equal(out[0][0], out[1][0])
