"""Pins of the pre-processing oracle (oracle/preprocess.py), CPU.

* Closed form: points on a line y = 2x + 1 in two dimensions standardise to two identical
  columns, so C = m/(m-1) [[1, 1], [1, 1]]: eigenvalues 2m/(m-1) and 0, first component
  (1, 1)/sqrt(2).
* Invariants: orthonormal components, C v = lambda v, eigenvalues decreasing.
* Library routines: scikit-learn's StandardScaler and PCA give the same eigenvalues and
  components up to sign (skipped where sklearn is absent).
* Min-max: the training rows span exactly [0, range_max]; test rows are clipped; a constant
  feature maps to 0.
* Planted mistakes: an ascending eigenvalue order and a sample (ddof = 1) standard deviation
  each fail a pin above.
"""
import numpy as np
import pytest

from oracle import preprocess as pp


def _data(seed, m=300, p=12):
    rng = np.random.Generator(np.random.PCG64(seed))
    basis = np.linalg.qr(rng.normal(size=(p, p)))[0]
    spectrum = np.geomspace(4.0, 0.05, p)
    return rng.normal(size=(m, p)) * np.sqrt(spectrum) @ basis.T + rng.normal(size=p)


def test_line_closed_form():
    t = np.linspace(-1, 3, 50)
    x = np.stack([t, 2 * t + 1], axis=1)
    mean, scale, comps, w = pp.pca_fit(x, 2)
    m = 50
    np.testing.assert_allclose(w, [2 * m / (m - 1), 0.0], atol=1e-12)
    np.testing.assert_allclose(comps[0], [1 / np.sqrt(2), 1 / np.sqrt(2)], atol=1e-12)


def test_invariants():
    x = _data(1)
    mean, scale, comps, w = pp.pca_fit(x, 12)
    np.testing.assert_allclose(comps @ comps.T, np.eye(12), atol=1e-12)
    z = (x - mean) / scale
    C = z.T @ z / (x.shape[0] - 1)
    np.testing.assert_allclose(C @ comps.T, comps.T * w, atol=1e-10)
    assert np.all(np.diff(w) <= 0)
    assert np.all(np.abs(comps).argmax(axis=1) >= 0)
    big = comps[np.arange(12), np.abs(comps).argmax(axis=1)]
    assert np.all(big > 0)


def test_matches_sklearn():
    dec = pytest.importorskip("sklearn.decomposition")
    prep = pytest.importorskip("sklearn.preprocessing")
    x = _data(2)
    z = prep.StandardScaler().fit_transform(x)
    ref = dec.PCA(n_components=8, svd_solver="full").fit(z)
    _, _, comps, w = pp.pca_fit(x, 8)
    np.testing.assert_allclose(w, ref.explained_variance_, rtol=1e-10)
    np.testing.assert_allclose(comps, pp.fix_signs(ref.components_), atol=1e-10)


def test_minmax():
    x = _data(3)
    mean, scale, comps, _ = pp.pca_fit(x, 5)
    y = pp.project(x, mean, scale, comps)
    lo, hi = pp.minmax_fit(y)
    out = pp.minmax_apply(y, lo, hi)
    np.testing.assert_allclose(out.min(axis=0), 0.0, atol=1e-15)
    np.testing.assert_allclose(out.max(axis=0), np.pi, atol=1e-12)
    far = pp.minmax_apply(y * 3.0, lo, hi)
    assert far.min() >= 0.0 and far.max() <= np.pi
    const = pp.minmax_apply(np.ones((4, 1)), np.ones(1), np.ones(1))
    assert np.all(const == 0.0)


@pytest.mark.parametrize("mistake", ["ascending", "ddof1"])
def test_planted_mistakes_are_caught(monkeypatch, mistake):
    dec = pytest.importorskip("sklearn.decomposition")
    prep = pytest.importorskip("sklearn.preprocessing")
    x = _data(4)
    z = prep.StandardScaler().fit_transform(x)
    ref = dec.PCA(n_components=4, svd_solver="full").fit(z)
    if mistake == "ascending":
        monkeypatch.setattr(pp, "_order", lambda w: np.argsort(w, kind="stable"))
    else:
        good = pp.standardise_fit

        def ddof1(xx):
            mean, _ = good(xx)
            return mean, np.asarray(xx, dtype=np.float64).std(axis=0, ddof=1)
        monkeypatch.setattr(pp, "standardise_fit", ddof1)
    _, _, comps, w = pp.pca_fit(x, 4)
    assert not np.allclose(w, ref.explained_variance_, rtol=1e-10)
