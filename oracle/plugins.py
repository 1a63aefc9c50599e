"""Float64 oracle of the PCA post-processing plugin (Sec. III-D and its figure: a plugin turns
feature layers into a PCA layer).

TEST INFRASTRUCTURE ONLY: used by the test suite to check the CUDA plugin; nothing in the
library imports it. Parity is pinned in tests/test_oracle_plugins.py (a known 3-D subspace,
unobserved cells, the sign convention, cell order).
"""
from __future__ import annotations

import numpy as np


def pca_of_features(feat: np.ndarray, observed: np.ndarray, n_comp: int = 3):
    """PCA post-processing layer of a d-dimensional feature layer (Sec. III-D and its figure: a
    plugin turns feature layers into a PCA layer; the reading is in the design notes). Over the
    observed cells, in float64: mean m, covariance S = (1/n) sum (f - m)(f - m)^T, its
    n_comp eigenvectors of largest eigenvalue (numpy's symmetric eigensolver), each signed so
    that its largest-magnitude component (the first such on a tie) is positive; every observed
    cell gets the projections (f - m) . v_k, other cells 0. Returns (proj [cells, n_comp],
    eigenvalues [n_comp], vectors [n_comp, d], mean [d])."""
    f = np.asarray(feat, np.float64)
    obs = np.asarray(observed, bool)
    X = f[obs]
    n, d = X.shape
    out = np.zeros((f.shape[0], n_comp))
    if n == 0:
        return out, np.zeros(n_comp), np.zeros((n_comp, d)), np.zeros(d)
    m = X.mean(axis=0)
    Xc = X - m
    S = Xc.T @ Xc / n
    w, V = np.linalg.eigh(S)
    order = np.argsort(-w, kind="stable")[:n_comp]
    w, V = w[order], V[:, order].T.copy()
    for k in range(n_comp):
        i = int(np.argmax(np.abs(V[k])))
        if V[k, i] < 0:
            V[k] = -V[k]
    out[obs] = Xc @ V.T
    return out, w, V, m


