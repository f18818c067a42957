"""MPS of a block-structured feature map from its block statevectors, with SVD truncation.

Test infrastructure only (see the package header).

For a block product structure (§II-C: entanglers only inside blocks of b consecutive
qubits) the state is the Kronecker product of the blocks' states, so the MPS splits at the
block boundaries (bond 1 there) and each block's piece follows from that block's dense
statevector (b <= 12) by a left-to-right sweep of singular value decompositions:

1. psi_B of every sample, by ``circuit.statevector`` on the block's features (any
   entangler inside the block, including all-to-all ZZ, whose bonds exceed 2^reps);
2. for the cut after each qubit q of the block: reshape the remainder to
   (D_left * 2) x 2^(b - q - 1), take its SVD (numpy.linalg.svd, a library routine), keep
   the singular values s > cutoff * s_0 and at most chi_cap of them, record the discarded
   squared weight relative to the whole spectrum, rescale the kept values to the norm of
   the whole spectrum, store U as the site tensor and carry diag(s) V^H to the next qubit;
3. the last qubit's site tensor is the remaining (D_left * 2) vector.

This is the truncation reading for the paper's SVD cutoff: drop s_k < cutoff * s_0, cap
at chi, renormalise to unit norm, report the discarded weight. As in ``mps.build_mps``, all
samples share bond dimensions (the largest kept rank of the batch); a sample's own dropped
singular values are set to zero.
"""
from __future__ import annotations

import numpy as np

from .circuit import statevector


def block_ranges(n: int, block: int):
    """[(start, stop)] of the blocks of b consecutive qubits (the last may be shorter)."""
    b = n if block <= 0 else block
    return [(s, min(s + b, n)) for s in range(0, n, b)]


def _truncate(s, chi_cap, cutoff):
    """Kept mask of the singular values s (m x r, descending) and the batch rank."""
    s0 = s[:, :1]
    keep = s > cutoff * np.where(s0 > 0, s0, 1.0)
    if chi_cap is not None:
        keep[:, chi_cap:] = False
    return keep, max(1, int(keep.sum(axis=1).max()))


def block_mps(psi: np.ndarray, chi_cap=None, cutoff: float = 1e-10):
    """Sites (m, D_l, 2, D_r) of the block states psi (m x 2^b) and the discarded weight."""
    psi = np.asarray(psi, dtype=np.complex128)
    m, dim = psi.shape
    b = int(round(np.log2(dim)))
    sites = []
    discarded = np.zeros(m)
    rest = psi.reshape(m, 1, dim)  # (m, D_left, 2^(qubits left))
    for q in range(b - 1):
        dl = rest.shape[1]
        mat = rest.reshape(m, dl * 2, -1)
        u, s, vh = np.linalg.svd(mat, full_matrices=False)
        keep, rank = _truncate(s, chi_cap, cutoff)
        total = np.sum(s * s, axis=1)
        s_kept = np.where(keep, s, 0.0)[:, :rank]
        kept = np.sum(s_kept * s_kept, axis=1)
        discarded += np.where(total > 0, (total - kept) / np.where(total > 0, total, 1.0), 0.0)
        s_kept = s_kept * np.sqrt(np.where(kept > 0, total / np.where(kept > 0, kept, 1.0), 1.0))[:, None]
        sites.append(u[:, :, :rank].reshape(m, dl, 2, rank))
        rest = s_kept[:, :, None] * vh[:, :rank, :]
    sites.append(rest.reshape(m, rest.shape[1], 2, 1))
    return sites, discarded


def mps_from_block_states(x, reps: int, block: int, entangler: str = "full", angle_scale: float = 2.0,
                          chi_cap=None, cutoff: float = 1e-10):
    """(sites, discarded) of the block-structured map for the samples in x (m x n)."""
    x = np.atleast_2d(np.asarray(x, dtype=np.float64))
    m, n = x.shape
    sites = []
    discarded = np.zeros(m)
    for s, e in block_ranges(n, block):
        if e - s > 12:
            raise ValueError("block statevectors are limited to 12 qubits")
        psi = np.stack([statevector(row[s:e], reps, angle_scale, True, 0, entangler) for row in x])
        part, disc = block_mps(psi, chi_cap, cutoff)
        sites.extend(part)
        discarded += disc
    return sites, discarded
