"""Host logic of the SVM workflow (paper_2602_01330_gb300/svm.py), on the CPU: the stratified
fold split is seeded, covers every sample once, and deals each class evenly over the folds."""
import numpy as np

from paper_2602_01330_gb300.svm import stratified_folds


def test_stratified_folds():
    rng = np.random.Generator(np.random.PCG64(0))
    labels = rng.integers(0, 7, size=503)
    f1 = stratified_folds(labels, 5, seed=3)
    f2 = stratified_folds(labels, 5, seed=3)
    np.testing.assert_array_equal(f1, f2)
    assert not np.array_equal(f1, stratified_folds(labels, 5, seed=4))
    assert set(np.unique(f1)) == set(range(5))
    for c in range(7):
        counts = np.bincount(f1[labels == c], minlength=5)
        assert counts.max() - counts.min() <= 1
    sizes = np.bincount(f1, minlength=5)
    assert sizes.sum() == labels.size and sizes.max() - sizes.min() <= 7
