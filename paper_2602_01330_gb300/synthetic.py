"""Seeded synthetic inputs shaped like the paper's data (§II-A, §III).

The paper trains on Fashion-MNIST: 28x28 grey images, 10 classes, flattened to 784
features, reduced to the leading n components and min-max scaled (§II-A). That data
set is not available here, so this module draws images from a seeded class-template
model of the same shape and applies the same kind of pre-processing:

* 10 class templates; each is a sum of 6 Gaussian blobs (centre ~ U[4,24]^2 pixels,
  width ~ U[1.5,4] pixels, amplitude ~ U[0.5,1]), drawn from one seed;
* a sample is its class template plus N(0, 0.1^2) pixel noise, clipped to [0,1];
  labels are balanced (i mod 10) and then shuffled;
* d < 784 features come from projecting the 784 pixels onto a seeded orthonormal
  basis (a stand-in for the paper's PCA, which needs the real data); d = 784 keeps
  the raw pixels;
* features are min-max scaled per feature to [0, pi] with limits fitted on the
  training set, applied to the test set and clipped; constant features map to 0.

Nothing here computes any part of the kernel: both the CUDA path and the oracle
take the arrays produced here as their inputs.
"""
from __future__ import annotations

import numpy as np

N_CLASSES = 10
IMG_SIDE = 28
N_PIXELS = IMG_SIDE * IMG_SIDE
BLOBS_PER_CLASS = 6
PIXEL_NOISE = 0.1

SEED_TEMPLATES = 0
SEED_TRAIN = 1
SEED_TEST = 2
SEED_PROJECTION = 3


def class_templates(seed: int = SEED_TEMPLATES) -> np.ndarray:
    """(10, 784) float64 templates in [0, 1] (each a clipped sum of Gaussian blobs)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    yy, xx = np.meshgrid(np.arange(IMG_SIDE), np.arange(IMG_SIDE), indexing="ij")
    out = np.zeros((N_CLASSES, IMG_SIDE, IMG_SIDE))
    for c in range(N_CLASSES):
        for _ in range(BLOBS_PER_CLASS):
            cy, cx = rng.uniform(4.0, 24.0, size=2)
            sigma = rng.uniform(1.5, 4.0)
            amp = rng.uniform(0.5, 1.0)
            out[c] += amp * np.exp(-((yy - cy) ** 2 + (xx - cx) ** 2) / (2.0 * sigma * sigma))
    return np.clip(out, 0.0, 1.0).reshape(N_CLASSES, N_PIXELS)


def images(n_samples: int, seed: int, template_seed: int = SEED_TEMPLATES):
    """Draw n_samples flattened images in [0, 1] and their balanced, shuffled labels."""
    templates = class_templates(template_seed)
    rng = np.random.Generator(np.random.PCG64(seed))
    labels = np.arange(n_samples) % N_CLASSES
    rng.shuffle(labels)
    noise = rng.normal(0.0, PIXEL_NOISE, size=(n_samples, N_PIXELS))
    x = np.clip(templates[labels] + noise, 0.0, 1.0)
    return x, labels


def projection(d: int, seed: int = SEED_PROJECTION) -> np.ndarray:
    """(784, d) matrix with orthonormal columns (the Q factor of a seeded Gaussian matrix)."""
    if not 1 <= d <= N_PIXELS:
        raise ValueError(f"d must lie in [1, {N_PIXELS}], got {d}")
    rng = np.random.Generator(np.random.PCG64(seed))
    q, _ = np.linalg.qr(rng.normal(size=(N_PIXELS, d)))
    return q


def minmax_fit(x: np.ndarray):
    return x.min(axis=0), x.max(axis=0)


def minmax_apply(x: np.ndarray, lo: np.ndarray, hi: np.ndarray, top: float = np.pi) -> np.ndarray:
    span = hi - lo
    safe = np.where(span > 0, span, 1.0)
    y = (x - lo) / safe * top
    y = np.where(span > 0, y, 0.0)
    return np.clip(y, 0.0, top)


def fmnist_like(n_train: int, n_test: int, d: int,
                seed_train: int = SEED_TRAIN, seed_test: int = SEED_TEST,
                seed_templates: int = SEED_TEMPLATES, seed_projection: int = SEED_PROJECTION):
    """Train/test features in [0, pi] (float32) with d columns, plus labels.

    d = 784 keeps raw pixels; smaller d projects onto a seeded orthonormal basis.
    """
    xtr, ytr = images(n_train, seed_train, seed_templates)
    xte, yte = images(n_test, seed_test, seed_templates) if n_test > 0 else (np.zeros((0, N_PIXELS)), np.zeros(0, int))
    if d < N_PIXELS:
        q = projection(d, seed_projection)
        xtr = xtr @ q
        xte = xte @ q
    lo, hi = minmax_fit(xtr)
    ftr = minmax_apply(xtr, lo, hi).astype(np.float32)
    fte = minmax_apply(xte, lo, hi).astype(np.float32)
    return {"x_train": ftr, "y_train": ytr, "x_test": fte, "y_test": yte}


def uniform_angles(m: int, n: int, seed: int = 0, dtype=np.float64) -> np.ndarray:
    """m x n features drawn uniformly from [0, pi] (the tiny n=8 check case uses seed 0)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.uniform(0.0, np.pi, size=(m, n)).astype(dtype)


def near_copies(x: np.ndarray, sigma_lo: float, sigma_hi: float, seed: int) -> np.ndarray:
    """Perturbed copies of the rows of x: row i plus N(0, sigma_i^2) noise on every feature,
    clipped to [0, pi], with sigma_i log-uniform in [sigma_lo, sigma_hi] (seeded). Pairs of
    a row and its copy have quantum kernel values spread from near 0 to near 1 even at
    hundreds of qubits, where independent samples give values far below 1e-100. Returns
    the dtype of x."""
    rng = np.random.Generator(np.random.PCG64(seed))
    m = x.shape[0]
    sigma = np.exp(rng.uniform(np.log(sigma_lo), np.log(sigma_hi), size=m))
    y = x.astype(np.float64) + rng.normal(0.0, 1.0, size=x.shape) * sigma[:, None]
    return np.clip(y, 0.0, np.pi).astype(x.dtype)
