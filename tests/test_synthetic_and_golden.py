"""Input generator properties, and the oracle against its stored fixture (CPU)."""
import os

import numpy as np

import closed_forms as cf
from oracle import gram, mps
from paper_2602_01330_gb300 import synthetic

HERE = os.path.dirname(os.path.abspath(__file__))


def test_generator_is_seeded_and_in_range():
    a = synthetic.fmnist_like(50, 20, 64)
    b = synthetic.fmnist_like(50, 20, 64)
    assert np.array_equal(a["x_train"], b["x_train"]) and np.array_equal(a["x_test"], b["x_test"])
    for key in ("x_train", "x_test"):
        x = a[key]
        assert x.dtype == np.float32 and x.shape[1] == 64
        assert x.min() >= 0.0 and x.max() <= np.float32(np.pi)
    # train features span [0, pi] per feature (min-max fitted on train)
    assert np.allclose(a["x_train"].min(axis=0), 0.0) and np.allclose(a["x_train"].max(axis=0), np.pi, atol=1e-6)
    # labels balanced
    assert np.bincount(a["y_train"], minlength=10).tolist() == [5] * 10


def test_projection_is_orthonormal():
    q = synthetic.projection(32)
    assert np.allclose(q.T @ q, np.eye(32), atol=1e-12)


def test_raw_pixels_at_784():
    d = synthetic.fmnist_like(12, 0, 784)["x_train"]
    assert d.shape == (12, 784)


def test_golden_tiny_case_reproduced_by_oracle():
    # The stored fixture came from the statevector oracle; the MPS + transfer oracle and
    # the one-repetition Ising closed form must reproduce it.
    stored = np.loadtxt(os.path.join(HERE, "golden", "cfg1_kq16.txt"))
    x = synthetic.uniform_angles(64, 8, seed=0)[:16]
    sites, _ = mps.build_mps(x, 1)
    kq, _ = gram.gram_from_mps(sites, sites)
    assert np.max(np.abs(kq - stored)) < 1e-12
    for i in range(0, 16, 5):
        for j in range(0, 16, 3):
            assert abs(np.exp(cf.ising_log_kernel(x[i], x[j])) - stored[i, j]) < 1e-12
