"""Quantum kernel by transfer contraction, RBF kernel and dual-kernel mix.

Test infrastructure only (see the package header).

* Quantum kernel, §II-C, Eqs. 7-10: for a pair (x_i, x_j) the amplitude
  a = <psi(x_i)|psi(x_j)> (Eq. 9 gives its complex conjugate, which has the same
  modulus) is contracted site by site from the left,

      E_0 = [1],   E_k = sum_{s in {0,1}} A_s^(k)(x_i)^dagger  E_{k-1}  A_s^(k)(x_j),

  and a = E_n (a 1 x 1 matrix). After each site E is multiplied by an exact power of
  two, 2^-e with e the binary exponent of max |E|, and e is added to an integer
  counter, so that a = mantissa * 2^counter never underflows. K_q = |a|^2 (Eq. 10),
  log K_q = 2 (ln|mantissa| + counter ln 2).
* RBF kernel, §II-B, Eq. 3: K_c = exp(-gamma ||x_i - x_j||^2).
* Dual kernel, §II-D, Eq. 11: K = w K_q + (1 - w) K_c (the paper's alpha is w here).
"""
from __future__ import annotations

import numpy as np

from .mps import build_mps

LN2 = float(np.log(2.0))


def transfer_overlaps(rows, cols, i_idx, j_idx):
    """Amplitudes <psi(x_i)|psi(x_j)> for the listed pairs, as (mantissa, exponent2).

    rows / cols are MPS site lists (see ``oracle.mps.build_mps``); i_idx / j_idx index
    their samples. Returns complex mantissas and int64 binary exponents.
    """
    i_idx = np.asarray(i_idx, dtype=np.int64)
    j_idx = np.asarray(j_idx, dtype=np.int64)
    p = i_idx.shape[0]
    e = np.ones((p, 1, 1), dtype=np.complex128)
    exp2 = np.zeros(p, dtype=np.int64)
    for a_all, b_all in zip(rows, cols):
        a = a_all[i_idx]          # (p, Dl, 2, Dr)  -- conjugated side
        b = b_all[j_idx]
        t = np.einsum("pab,pbsd->pasd", e, b)
        e = np.einsum("pasc,pasd->pcd", np.conj(a), t)
        mx = np.max(np.abs(e), axis=(1, 2))
        _, ex = np.frexp(mx)
        ex = np.where(mx > 0, ex, 0).astype(np.int64)
        e = np.ldexp(e.real, -ex[:, None, None]) + 1j * np.ldexp(e.imag, -ex[:, None, None])
        exp2 += ex
    return e[:, 0, 0], exp2


def kq_from_overlap(mantissa, exp2):
    """(K_q, log K_q) from a = mantissa * 2^exp2 (Eq. 10). log K_q = -inf for a = 0."""
    mod = np.abs(mantissa)
    with np.errstate(divide="ignore"):
        log_kq = 2.0 * (np.log(mod) + exp2 * LN2)
    return np.exp(log_kq), log_kq


def pair_values(rows, cols, i_idx, j_idx, chunk: int = 8192):
    """K_q and log K_q for the listed pairs, in chunks of pairs."""
    i_idx = np.asarray(i_idx)
    j_idx = np.asarray(j_idx)
    kq = np.empty(i_idx.shape[0])
    lkq = np.empty(i_idx.shape[0])
    for s in range(0, i_idx.shape[0], chunk):
        mant, e2 = transfer_overlaps(rows, cols, i_idx[s:s + chunk], j_idx[s:s + chunk])
        kq[s:s + chunk], lkq[s:s + chunk] = kq_from_overlap(mant, e2)
    return kq, lkq


def gram_from_mps(rows, cols, chunk: int = 8192):
    """Full K_q and log K_q matrices (rows x cols) from two MPS batches."""
    mr = rows[0].shape[0]
    mc = cols[0].shape[0]
    ii, jj = np.meshgrid(np.arange(mr), np.arange(mc), indexing="ij")
    kq, lkq = pair_values(rows, cols, ii.ravel(), jj.ravel(), chunk)
    return kq.reshape(mr, mc), lkq.reshape(mr, mc)


def quantum_gram(x_rows, x_cols=None, reps: int = 2, angle_scale: float = 2.0,
                 entangle: bool = True, chi_cap=None, cutoff: float = 1e-14, block: int = 0):
    """K_q and log K_q for all pairs of rows of x_rows and x_cols (x_cols defaults to x_rows).
    block: 0 for the open ZZ chain, b >= 1 for blocks of b qubits (``circuit.entangled_bonds``)."""
    rows, _ = build_mps(x_rows, reps, angle_scale, entangle, chi_cap, cutoff, block)
    cols = rows if x_cols is None else build_mps(x_cols, reps, angle_scale, entangle, chi_cap, cutoff, block)[0]
    return gram_from_mps(rows, cols)


def rbf(x_rows, x_cols, gamma: float):
    """K_c[i, j] = exp(-gamma * sum_f (x_rows[i, f] - x_cols[j, f])^2) (Eq. 3), row by row."""
    a = np.asarray(x_rows, dtype=np.float64)
    b = np.asarray(x_cols, dtype=np.float64)
    out = np.empty((a.shape[0], b.shape[0]))
    for i in range(a.shape[0]):
        diff = b - a[i][None, :]
        out[i] = np.exp(-gamma * np.sum(diff * diff, axis=1))
    return out


def rbf_pairs(x_rows, x_cols, i_idx, j_idx, gamma: float):
    """K_c for the listed pairs only: exp(-gamma ||x_rows[i] - x_cols[j]||^2) (Eq. 3)."""
    a = np.asarray(x_rows, dtype=np.float64)[np.asarray(i_idx)]
    b = np.asarray(x_cols, dtype=np.float64)[np.asarray(j_idx)]
    diff = a - b
    return np.exp(-gamma * np.sum(diff * diff, axis=1))


def dual_kernel(kq, kc, w: float):
    """K = w K_q + (1 - w) K_c (Eq. 11)."""
    return w * np.asarray(kq) + (1.0 - w) * np.asarray(kc)
