"""The data pre-processing of §II-A on the GPU: standardise the raw pixels, project onto the
leading n principal components of the training rows, and min-max scale every feature to
[0, range_max] (the paper's [0, 1]; [0, pi] here, the range of the feature map's angles).

``PCAPreprocessor`` fits once on the training rows (``dk_pca_fit``, all components up to
``k_max``) and then gives features for any n <= k_max (``dk_pca_transform`` with the leading
n components): the feature-dimension sweep needs one fit, not one per n. All arithmetic runs
in libdualk's kernels; this module only keeps the fitted tensors.
"""
from __future__ import annotations

import math

import torch

from . import dualk


class PCAPreprocessor:
    def __init__(self, ctx: dualk.Context, k_max: int | None = None, sweeps: int = 10, range_max: float = math.pi):
        self.ctx, self.k_max, self.sweeps, self.range_max = ctx, k_max, sweeps, range_max
        self.model = None

    def fit(self, x_train: torch.Tensor):
        """Standardisation and PCA on the raw training rows (m x p float32, CUDA)."""
        k = self.k_max or x_train.shape[1]
        self.model = dualk.pca_fit(self.ctx, x_train.contiguous(), k, self.sweeps)
        return self

    def features(self, x_train: torch.Tensor, x_test: torch.Tensor, n: int):
        """(train, test) features on the leading n components, scaled by the training range."""
        sub = {"mean": self.model["mean"], "scale": self.model["scale"],
               "components": self.model["components"][:n].contiguous()}
        ftr = dualk.pca_transform(self.ctx, x_train.contiguous(), sub, fit_range=True, range_max=self.range_max)
        fte = dualk.pca_transform(self.ctx, x_test.contiguous(), sub, fit_range=False, range_max=self.range_max)
        return ftr, fte
