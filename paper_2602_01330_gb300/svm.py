"""Dual-kernel SVM on the GPU: the consumer of the Gram matrices (§II-B, Eqs. 1-5; §II-D).

The paper trains a one-against-one SVM on the mixed kernel K = w K_q + (1 - w) K_c, picking
C and w by 5-fold cross-validation, then classifies the test samples from their kernel rows
K(x_i, x). Here every step runs in libdualk's kernels:

* ``cross_validate``: stratified folds (seeded), and the whole grid folds x C x w as ONE
  ``dk_svm_ovo_train`` launch (one job per fold and grid point, each job a list of sample
  indices into the training Gram) plus ONE ``dk_svm_ovo_predict`` launch over the held-out
  samples; the accuracies per grid point come back as a small host array.
* ``fit``: the final model on all training samples at the chosen (C, w).
* ``predict``: votes for the test samples from the rows of ``dual_kernel_rows``.
* ``run_pipeline``: synthetic data -> MPS -> Gram and rows -> CV -> fit -> test accuracy,
  timed per phase.

This module only builds index lists and reads back a few numbers.
"""
from __future__ import annotations

import json
import time
from dataclasses import dataclass

import numpy as np
import torch

from . import dualk


def stratified_folds(labels: np.ndarray, n_folds: int = 5, seed: int = 0) -> np.ndarray:
    """Fold number of every sample: each class shuffled (PCG64 seed) and dealt round-robin."""
    rng = np.random.Generator(np.random.PCG64(seed))
    fold = np.empty(labels.size, dtype=np.int64)
    for c in np.unique(labels):
        sel = np.flatnonzero(labels == c)
        sel = sel[rng.permutation(sel.size)]
        fold[sel] = np.arange(sel.size) % n_folds
    return fold


@dataclass
class CVResult:
    grid: list            # [(C, w)]
    accuracy: np.ndarray  # mean held-out accuracy per grid point
    per_fold: np.ndarray  # (grid, folds)
    best: tuple           # (C, w) with the highest mean accuracy (first on ties)
    train_ms: float
    predict_ms: float
    jobs: int
    binary_problems: int
    job_list: list        # [(fold, C, w)] in launch order
    pred: np.ndarray      # (jobs, r_max) predicted classes of each job's held-out samples
    folds: np.ndarray     # fold number of every training sample


class DualKernelSVM:
    """One-against-one SVM on w K_q + (1 - w) K_c with C and w chosen by cross-validation."""

    def __init__(self, ctx: dualk.Context, n_class: int, Cs=(0.1, 1.0, 10.0, 100.0),
                 ws=(0.0, 0.25, 0.5, 0.75, 1.0), n_folds: int = 5, seed: int = 0, tol: float = 1e-3):
        self.ctx, self.n_class = ctx, n_class
        self.Cs, self.ws = tuple(Cs), tuple(ws)
        self.n_folds, self.seed, self.tol = n_folds, seed, tol
        self.model = None

    def _dev(self, a, dt):
        return torch.from_numpy(np.ascontiguousarray(a, dtype=dt)).to(self.device)

    def cross_validate(self, kq: torch.Tensor, kc: torch.Tensor, labels: np.ndarray) -> CVResult:
        self.device = kq.device
        m = labels.size
        fold = stratified_folds(labels, self.n_folds, self.seed)
        grid = [(C, w) for C in self.Cs for w in self.ws]
        jobs = [(f, C, w) for (C, w) in grid for f in range(self.n_folds)]
        tr = [np.flatnonzero(fold != f) for f in range(self.n_folds)]
        va = [np.flatnonzero(fold == f) for f in range(self.n_folds)]
        m_max, r_max = max(t.size for t in tr), max(v.size for v in va)
        idx = np.zeros((len(jobs), m_max), np.int32)
        cnt = np.zeros(len(jobs), np.int32)
        rows = np.zeros((len(jobs), r_max), np.int32)
        rcnt = np.zeros(len(jobs), np.int32)
        for j, (f, C, w) in enumerate(jobs):
            idx[j, :tr[f].size], cnt[j] = tr[f], tr[f].size
            rows[j, :va[f].size], rcnt[j] = va[f], va[f].size
        di, dn, dr, drc = (self._dev(idx, np.int32), self._dev(cnt, np.int32), self._dev(rows, np.int32),
                           self._dev(rcnt, np.int32))
        wt = self._dev([w for _, _, w in jobs], np.float32)
        Ct = self._dev([C for _, C, _ in jobs], np.float32)
        lab = self._dev(labels, np.int32)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        ev[0].record()
        model = dualk.svm_ovo_train(self.ctx, kq, kc, wt, Ct, di, dn, lab, self.n_class, tol=self.tol)
        ev[1].record()
        out = dualk.svm_ovo_predict(self.ctx, kq, kc, wt, model, self.n_class, rows=dr, row_count=drc, idx=di,
                                    count=dn, want_decision=False)
        ev[2].record()
        pred = out["pred"].cpu().numpy()
        self.ctx.sync_status()
        per = np.zeros((len(grid), self.n_folds))
        for j, (f, C, w) in enumerate(jobs):
            g = grid.index((C, w))
            per[g, f] = np.mean(pred[j, :va[f].size] == labels[va[f]])
        acc = per.mean(axis=1)
        best = grid[int(np.argmax(acc))]
        return CVResult(grid, acc, per, best, ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2]), len(jobs),
                        len(jobs) * self.n_class * (self.n_class - 1) // 2, jobs, pred, fold)

    def fit(self, kq: torch.Tensor, kc: torch.Tensor, labels: np.ndarray, C: float, w: float):
        """Final model on all training samples (one job)."""
        self.device = kq.device
        m = labels.size
        self.w = self._dev([w], np.float32)
        self.idx = self._dev(np.arange(m)[None, :], np.int32)
        self.cnt = self._dev([m], np.int32)
        self.model = dualk.svm_ovo_train(self.ctx, kq, kc, self.w, self._dev([C], np.float32), self.idx, self.cnt,
                                         self._dev(labels, np.int32), self.n_class, tol=self.tol)
        return self.model

    def predict(self, kq_rows: torch.Tensor, kc_rows: torch.Tensor, want_decision: bool = False):
        """Classes of the samples whose kernel rows (against the training samples) are given."""
        return dualk.svm_ovo_predict(self.ctx, kq_rows, kc_rows, self.w, self.model, self.n_class,
                                     want_decision=want_decision)


def run_pipeline(ctx: dualk.Context, n_train: int = 2000, n_test: int = 500, d: int = 784, reps: int = 2,
                 Cs=(0.1, 1.0, 10.0, 100.0), ws=(0.0, 0.25, 0.5, 0.75, 1.0), seed: int = 0,
                 gram=None, features: str = "projection", block: int = 0, entangler: str = "chain") -> dict:
    """The §II-D workflow on synthetic Fashion-MNIST-shaped data: Gram + rows (or the given
    `gram` = (kq, kc, kq_rows, kc_rows) tensors), 5-fold CV over C x w, final fit, test
    accuracy. features = "projection": the generator's seeded projection and scaling;
    "pca": the raw images through the GPU pre-processing of §II-A (standardise, PCA to d,
    min-max to [0, pi]). block = b >= 1: the block-structured map (entanglers only inside
    blocks of b qubits, `entangler` "chain" or "full"), its Gram and rows computed exactly by
    per-block statevector overlaps (dk_block_states, dk_gram_blocks). Accuracies on synthetic
    data are a consistency check, not the paper's results."""
    from . import synthetic
    pre_ms = None
    if features == "pca":
        from .preprocess import PCAPreprocessor
        xr, ytr = synthetic.images(n_train, synthetic.SEED_TRAIN)
        xs, yte = synthetic.images(n_test, synthetic.SEED_TEST)
        xr = torch.from_numpy(xr.astype(np.float32)).cuda()
        xs = torch.from_numpy(xs.astype(np.float32)).cuda()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev[0].record()
        pre = PCAPreprocessor(ctx, k_max=d).fit(xr)
        ftr, fte = pre.features(xr, xs, d)
        ev[1].record()
        torch.cuda.synchronize()
        pre_ms = ev[0].elapsed_time(ev[1])
        data = {"x_train": ftr, "x_test": fte}
    else:
        data = synthetic.fmnist_like(n_train, n_test, d)
        ytr, yte = data["y_train"], data["y_test"]
        data = {"x_train": torch.from_numpy(data["x_train"]).cuda(), "x_test": torch.from_numpy(data["x_test"]).cuda()}
    ytr, yte = np.asarray(ytr), np.asarray(yte)
    n_class = int(max(ytr.max(), yte.max())) + 1
    t0 = time.perf_counter()
    if gram is None and block > 0:
        ent = dualk.DK_ENT_FULL if entangler == "full" else dualk.DK_ENT_CHAIN
        fb = dualk.FeatureMap(reps=reps, block=block)
        str_ = dualk.block_states(ctx, data["x_train"], fb, ent)
        ste = dualk.block_states(ctx, data["x_test"], fb, ent)
        g = dualk.gram_blocks(ctx, str_, w=1.0, want=("kq", "kc"))
        r = dualk.gram_blocks(ctx, ste, str_, w=1.0, want=("kq", "kc"))
        kq, kc, kqr, kcr = g["kq"], g["kc"], r["kq"], r["kc"]
    elif gram is None:
        fm = dualk.FeatureMap(reps=reps, chi_max=4)
        mtr = dualk.mps_build(ctx, data["x_train"], fm)
        mte = dualk.mps_build(ctx, data["x_test"], fm)
        g = dualk.gram(ctx, mtr, w=1.0, want=("kq", "kc"))
        r = dualk.dual_kernel_rows(ctx, mte, mtr, w=1.0, want=("kq", "kc"))
        kq, kc, kqr, kcr = g["kq"], g["kc"], r["kq"], r["kc"]
    else:
        kq, kc, kqr, kcr = gram
    torch.cuda.synchronize()
    t_gram = time.perf_counter() - t0
    clf = DualKernelSVM(ctx, n_class, Cs, ws, seed=seed)
    cv = clf.cross_validate(kq, kc, ytr)
    C, w = cv.best
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    ev[0].record()
    clf.fit(kq, kc, ytr, C, w)
    ev[1].record()
    pred = clf.predict(kqr, kcr)["pred"][0]
    ev[2].record()
    pred = pred.cpu().numpy()
    ctx.sync_status()
    return {
        "workload": f"fmnist-shaped d={d} train={n_train} test={n_test} classes={n_class}, features={features}, "
                    + (f"blocks of {block} ({entangler} ZZ), " if block > 0 else "")
                    + f"{len(cv.grid)} (C, w) points x 5 folds",
        "preprocess_ms": pre_ms,
        "gram_and_rows_s": t_gram,
        "cv_jobs": cv.jobs, "cv_binary_problems": cv.binary_problems,
        "cv_train_ms": cv.train_ms, "cv_predict_ms": cv.predict_ms,
        "cv_best": {"C": C, "w": w, "accuracy": float(cv.accuracy.max())},
        "cv_accuracy_by_w": {str(wv): float(max(cv.accuracy[i] for i, (Cv, wx) in enumerate(cv.grid) if wx == wv))
                             for wv in ws},
        "fit_ms": ev[0].elapsed_time(ev[1]), "predict_ms": ev[1].elapsed_time(ev[2]),
        "test_accuracy": float(np.mean(pred == yte)),
    }


def main():
    """Dual-kernel SVM pipeline on the bench-sized synthetic workload."""
    import argparse

    ap = argparse.ArgumentParser(description=main.__doc__)
    ap.add_argument("--n-train", type=int, default=2000)
    ap.add_argument("--n-test", type=int, default=500)
    ap.add_argument("--d", type=int, default=784)
    ap.add_argument("--features", choices=("projection", "pca"), default="projection")
    ap.add_argument("--block", type=int, default=0, help="block-structured map with blocks of this many qubits")
    ap.add_argument("--entangler", choices=("chain", "full"), default="chain")
    args = ap.parse_args()
    ctx = dualk.Context(0)
    print(json.dumps(run_pipeline(ctx, args.n_train, args.n_test, args.d, features=args.features, block=args.block,
                                  entangler=args.entangler)))
    ctx.close()


if __name__ == "__main__":
    main()
