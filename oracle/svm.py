"""FP64 oracle for the SVM that consumes the kernel matrices (§II-B, Eqs. 1-2, 4-5; §II-D).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Binary problem (§II-B, Eqs. 1-2): with labels y_i in {-1, +1} and a precomputed kernel K,

    minimise  1/2 sum_ij a_i a_j y_i y_j K_ij - sum_i a_i
    subject to sum_i a_i y_i = 0,  0 <= a_i <= C.

The minimiser is found by sequential minimal optimisation with the second-order
working-set rule of Fan, Chen and Lin (JMLR 6, 2005), written here in plain NumPy float64
from the published method: each step picks the most violating index i of the upper set,
then the j of the lower set with the largest guaranteed decrease of the objective, solves
the two-variable problem exactly, clips it to the box and updates the gradient. It stops
when the largest KKT violation m(a) - M(a) falls below `tol`.

Bias (Eq. 5, f(x) = sum_i a_i y_i K(x_i, x) + b): minus the mean of y_t grad_t over the free
multipliers (0 < a_t < C); with none free, minus the midpoint of the feasible interval.

Multiclass (§II-B, one-against-one): one binary problem per class pair (c1, c2), c1 < c2,
on the samples of those two classes with y = +1 for c1; each classifier votes c1 if
f > 0, else c2; the prediction is the class with most votes, the smallest index on ties.
"""
from __future__ import annotations

import numpy as np


def smo(K: np.ndarray, y: np.ndarray, C: float, tol: float = 1e-6, max_iter: int = 1_000_000,
        tau: float = 1e-12):
    """Dual SVM (Eqs. 1-2) on kernel K (m x m) and labels y in {-1, +1}.

    Returns (alpha, b, iterations)."""
    K = np.asarray(K, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    m = y.size
    a = np.zeros(m)
    g = -np.ones(m)                      # gradient of the objective, Q a - e
    kd = np.diag(K).copy()
    it = 0
    while it < max_iter:
        v = -y * g                        # -y_t grad_t
        up = ((y > 0) & (a < C)) | ((y < 0) & (a > 0))
        low = ((y > 0) & (a > 0)) | ((y < 0) & (a < C))
        if not up.any() or not low.any():
            break
        i = int(np.flatnonzero(up)[np.argmax(v[up])])
        vmax = v[i]
        vmin = v[low].min()
        if vmax - vmin < tol:
            break
        # second-order choice of j among the lower set with -y_t grad_t < vmax
        cand = low & (v < vmax)
        bgap = vmax - v[cand]
        curv = kd[i] + kd[cand] - 2.0 * K[i, cand]
        curv = np.where(curv > 0, curv, tau)
        j = int(np.flatnonzero(cand)[np.argmin(-(bgap * bgap) / curv)])
        # exact two-variable step along y_i a_i + y_j a_j = const, clipped to [0, C]^2
        ai, aj = a[i], a[j]
        eta = kd[i] + kd[j] - 2.0 * K[i, j]
        eta = eta if eta > 0 else tau
        # moving a_i by +y_i t and a_j by -y_j t changes the objective at rate -(vmax - v_j)
        t = (vmax - v[j]) / eta
        # bounds on t from 0 <= a_i + y_i t <= C and 0 <= a_j - y_j t <= C
        lo, hi = -np.inf, np.inf
        for aa, s in ((ai, y[i]), (aj, -y[j])):
            if s > 0:
                lo, hi = max(lo, -aa), min(hi, C - aa)
            else:
                lo, hi = max(lo, aa - C), min(hi, aa)
        t = min(max(t, lo), hi)
        da_i, da_j = y[i] * t, -y[j] * t
        a[i] = ai + da_i
        a[j] = aj + da_j
        _grad_update(g, y, K, i, j, da_i, da_j)
        it += 1
    return a, _bias(a, y, g, C), it


def _grad_update(g, y, K, i, j, da_i, da_j):
    """grad_k += y_k y_i K_ki da_i + y_k y_j K_kj da_j (in place)."""
    g += y * (y[i] * da_i * K[:, i] + y[j] * da_j * K[:, j])


def _bias(a, y, g, C) -> float:
    """b of Eq. 5 from the final gradient: minus the mean of y_t grad_t over the free
    multipliers, or minus the midpoint of the feasible interval when none is free."""
    yg = y * g
    free = (a > 0) & (a < C)
    if free.any():
        r = yg[free].mean()
    else:
        at_c = a >= C
        at_0 = a <= 0
        ub_set = (at_c & (y < 0)) | (at_0 & (y > 0))
        lb_set = (at_c & (y > 0)) | (at_0 & (y < 0))
        ub = yg[ub_set].min() if ub_set.any() else np.inf
        lb = yg[lb_set].max() if lb_set.any() else -np.inf
        r = 0.5 * (ub + lb) if np.isfinite(ub) and np.isfinite(lb) else (ub if np.isfinite(ub) else lb)
    return -float(r)


def dual_objective(K: np.ndarray, y: np.ndarray, a: np.ndarray) -> float:
    """The dual objective of Eq. 1 at a."""
    ay = a * y
    return 0.5 * float(ay @ K @ ay) - float(a.sum())


def kkt_violation(K: np.ndarray, y: np.ndarray, a: np.ndarray, C: float) -> float:
    """max over the upper set minus min over the lower set of -y_t grad_t (0 at the optimum)."""
    g = (y * (K @ (a * y))) - 1.0
    v = -y * g
    up = ((y > 0) & (a < C)) | ((y < 0) & (a > 0))
    low = ((y > 0) & (a > 0)) | ((y < 0) & (a < C))
    if not up.any() or not low.any():
        return 0.0
    return max(0.0, float(v[up].max() - v[low].min()))


def class_pairs(n_class: int):
    return [(c1, c2) for c1 in range(n_class) for c2 in range(c1 + 1, n_class)]


def ovo_train(K: np.ndarray, labels: np.ndarray, n_class: int, C: float, tol: float = 1e-6):
    """One binary SVM per class pair on the full kernel K of the training samples.

    Returns coef (P x m, a_i y_i in the pair's problem, 0 elsewhere) and bias (P)."""
    labels = np.asarray(labels)
    m = labels.size
    pairs = class_pairs(n_class)
    coef = np.zeros((len(pairs), m))
    bias = np.zeros(len(pairs))
    for p, (c1, c2) in enumerate(pairs):
        sel = np.flatnonzero((labels == c1) | (labels == c2))
        if sel.size == 0 or np.all(labels[sel] == labels[sel[0]]):
            continue
        y = np.where(labels[sel] == c1, 1.0, -1.0)
        a, b, _ = smo(K[np.ix_(sel, sel)], y, C, tol)
        coef[p, sel] = a * y
        bias[p] = b
    return coef, bias


def ovo_decision(K_rows: np.ndarray, coef: np.ndarray, bias: np.ndarray) -> np.ndarray:
    """Decision values f_p(x) = sum_i coef_pi K(x_i, x) + b_p (Eq. 5) for the rows of
    K_rows (r x m kernel values against the training samples): r x P."""
    return np.asarray(K_rows, dtype=np.float64) @ coef.T + bias[None, :]


def ovo_vote(decision: np.ndarray, n_class: int) -> np.ndarray:
    """One-against-one voting: class pair (c1, c2) votes c1 if f > 0 else c2; most votes
    wins, the smallest class index on ties."""
    pairs = class_pairs(n_class)
    votes = np.zeros((decision.shape[0], n_class), dtype=np.int64)
    for p, (c1, c2) in enumerate(pairs):
        win1 = decision[:, p] > 0
        votes[win1, c1] += 1
        votes[~win1, c2] += 1
    return np.argmax(votes, axis=1)
