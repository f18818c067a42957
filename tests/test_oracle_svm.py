"""Pins of the SVM oracle (oracle/svm.py) against things other than itself (CPU).

* Two samples of opposite labels: the dual has a closed form. With c = K11 + K22 - 2 K12 the
  unconstrained optimum is a1 = a2 = 2 / c with f(x1) = +1, f(x2) = -1, so
  b = 1 - a (K11 - K12); when 2 / c > C both sit at C and b is the midpoint -C (K11 - K22) / 2.
* Optimality: the returned multipliers satisfy the KKT conditions within the tolerance, are
  feasible, and no feasible perturbation lowers the dual objective.
* A library routine: scikit-learn's libsvm (SVC, precomputed kernel) gives the same
  one-against-one decision values and predictions (skipped where sklearn is absent).
* Planted mistakes: a bias with the wrong sign and a gradient update with a dropped term
  each fail one of the pins above.
"""
import numpy as np
import pytest

from oracle import svm


def _rbf(x, z, gamma):
    d2 = ((x[:, None, :] - z[None, :, :]) ** 2).sum(-1)
    return np.exp(-gamma * d2)


def _blobs(seed, m, n_class, dim=4, spread=0.9):
    rng = np.random.Generator(np.random.PCG64(seed))
    centres = rng.normal(0, 1.5, size=(n_class, dim))
    labels = np.arange(m) % n_class
    rng.shuffle(labels)
    x = centres[labels] + rng.normal(0, spread, size=(m, dim))
    return x, labels


@pytest.mark.parametrize("k11,k22,k12", [(1.0, 1.0, 0.3), (2.0, 1.5, -0.4), (1.0, 1.0, 0.9)])
def test_two_samples_closed_form(k11, k22, k12):
    K = np.array([[k11, k12], [k12, k22]])
    y = np.array([1.0, -1.0])
    c = k11 + k22 - 2 * k12
    a_free = 2.0 / c
    # unconstrained optimum inside the box
    a, b, _ = svm.smo(K, y, C=10 * a_free, tol=1e-12)
    np.testing.assert_allclose(a, [a_free, a_free], rtol=1e-10)
    assert b == pytest.approx(1.0 - a_free * (k11 - k12), abs=1e-10)
    # both multipliers at C
    C = 0.5 * a_free
    a, b, _ = svm.smo(K, y, C=C, tol=1e-12)
    np.testing.assert_allclose(a, [C, C], rtol=1e-12)
    assert b == pytest.approx(-C * (k11 - k22) / 2, abs=1e-10)


@pytest.mark.parametrize("C", [0.1, 1.0, 100.0])
def test_kkt_feasibility_and_local_optimality(C):
    x, labels = _blobs(3, 60, 2)
    K = _rbf(x, x, 0.3)
    y = np.where(labels == 0, 1.0, -1.0)
    a, b, it = svm.smo(K, y, C, tol=1e-9)
    assert it > 0
    assert np.all(a >= 0) and np.all(a <= C)
    assert abs(float(a @ y)) < 1e-9
    assert svm.kkt_violation(K, y, a, C) < 1e-8
    obj = svm.dual_objective(K, y, a)
    rng = np.random.Generator(np.random.PCG64(5))
    for _ in range(200):
        i, j = rng.choice(60, 2, replace=False)
        t = rng.normal(0, 0.05)
        a2 = a.copy()
        a2[i] += y[i] * t
        a2[j] -= y[j] * t
        if np.all(a2 >= 0) and np.all(a2 <= C):
            assert svm.dual_objective(K, y, a2) >= obj - 1e-12
    # the bias puts free support vectors on the margin: y f(x) = 1
    f = K @ (a * y) + b
    free = (a > 1e-9) & (a < C - 1e-9)
    if free.any():
        np.testing.assert_allclose(y[free] * f[free], 1.0, atol=1e-6)


def test_ovo_matches_libsvm():
    sk = pytest.importorskip("sklearn.svm")
    x, labels = _blobs(7, 150, 4)
    xt, lt = _blobs(8, 40, 4)
    K = _rbf(x, x, 0.25)
    Kt = _rbf(xt, x, 0.25)
    C = 2.0
    coef, bias = svm.ovo_train(K, labels, 4, C, tol=1e-10)
    dec = svm.ovo_decision(Kt, coef, bias)
    ref = sk.SVC(C=C, kernel="precomputed", tol=1e-10, decision_function_shape="ovo").fit(K, labels)
    np.testing.assert_allclose(dec, ref.decision_function(Kt), atol=1e-5)
    np.testing.assert_array_equal(svm.ovo_vote(dec, 4), ref.predict(Kt))


def test_vote_rule():
    # three classes, pairs (0,1), (0,2), (1,2); each row's votes by hand
    dec = np.array([[1.0, 1.0, 1.0],      # 0 beats 1, 0 beats 2, 1 beats 2 -> 0
                    [-1.0, -1.0, 1.0],    # 1, 2, 1 -> 1
                    [1.0, -1.0, 1.0],     # 0, 2, 1 -> one vote each -> smallest: 0
                    [-1.0, 1.0, -1.0]])   # 1, 0, 2 -> tie -> 0
    np.testing.assert_array_equal(svm.ovo_vote(dec, 3), [0, 1, 0, 0])


@pytest.mark.parametrize("mistake", ["bias_sign", "gradient_term"])
def test_planted_mistakes_are_caught(monkeypatch, mistake):
    x, labels = _blobs(11, 40, 2)
    K = _rbf(x, x, 0.3)
    y = np.where(labels == 0, 1.0, -1.0)
    if mistake == "bias_sign":
        good = svm._bias
        monkeypatch.setattr(svm, "_bias", lambda a, y_, g, C: -good(a, y_, g, C))
        a, b, _ = svm.smo(K, y, 1.0, tol=1e-9)
        f = K @ (a * y) + b
        free = (a > 1e-9) & (a < 1.0 - 1e-9)
        assert free.any()
        assert not np.allclose(y[free] * f[free], 1.0, atol=1e-6)   # the margin pin fails
    else:
        def without_j(g, y_, K_, i, j, da_i, da_j):
            g += y_ * (y_[i] * da_i * K_[:, i])
        monkeypatch.setattr(svm, "_grad_update", without_j)
        a, b, _ = svm.smo(K, y, 1.0, tol=1e-9, max_iter=5000)
        assert svm.kkt_violation(K, y, a, 1.0) > 1e-3                # the KKT pin fails
