"""FP64 oracle for the data pre-processing of §II-A: standardisation, PCA, min-max.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

* Standardisation: zero mean, unit variance per pixel over the training rows (population
  variance); a constant pixel keeps scale 1.
* PCA: the covariance C = Z^T Z / (m - 1) of the standardised training rows, its
  eigenvectors by numpy.linalg.eigh (a library routine), in order of decreasing eigenvalue;
  each component's sign is fixed so that its entry of largest magnitude is positive (the
  first such entry on ties). The leading n components are kept.
* Min-max: each projected feature mapped linearly so that the training rows span
  [0, range_max] (the paper's [0, 1]; [0, pi] for the feature map here), test rows clipped
  into that interval; a constant feature maps to 0.
"""
from __future__ import annotations

import numpy as np


def standardise_fit(x: np.ndarray):
    x = np.asarray(x, dtype=np.float64)
    mean = x.mean(axis=0)
    std = x.std(axis=0)
    scale = np.where(std > 0, std, 1.0)
    return mean, scale


def fix_signs(v: np.ndarray) -> np.ndarray:
    """Rows of v with the entry of largest magnitude (first on ties) made positive."""
    v = np.array(v, dtype=np.float64)
    idx = np.argmax(np.abs(v), axis=1)
    s = np.sign(v[np.arange(v.shape[0]), idx])
    s[s == 0] = 1.0
    return v * s[:, None]


def pca_fit(x: np.ndarray, k: int):
    """mean, scale, components (k x p, orthonormal rows) and eigenvalues (k, decreasing)."""
    x = np.asarray(x, dtype=np.float64)
    mean, scale = standardise_fit(x)
    z = (x - mean) / scale
    C = z.T @ z / (x.shape[0] - 1)
    w, V = np.linalg.eigh(C)
    order = _order(w)[:k]
    return mean, scale, fix_signs(V[:, order].T), w[order]


def _order(w):
    """Indices of the eigenvalues from largest to smallest (stable on ties)."""
    return np.argsort(-w, kind="stable")


def project(x, mean, scale, components):
    return ((np.asarray(x, dtype=np.float64) - mean) / scale) @ np.asarray(components).T


def minmax_fit(y: np.ndarray):
    return y.min(axis=0), y.max(axis=0)


def minmax_apply(y, lo, hi, range_max: float = np.pi):
    span = hi - lo
    out = np.where(span > 0, (y - lo) / np.where(span > 0, span, 1.0), 0.0) * range_max
    return np.clip(out, 0.0, range_max)
