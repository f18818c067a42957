"""Matrix product state of the feature-map state (§II-C, Eq. 6), built gate by gate.

Test infrastructure only (see the package header).

The state |psi(x)> = U(x)|0>^n is held as n site tensors A[k] of shape
(m, D_left, 2, D_right) -- one MPS per sample, m samples side by side -- and the
circuit is applied in order (time-evolving block decimation):

1. start from the product state |0...0> (all bonds 1);
2. per repetition: H, then RZ(angle_scale * x_k), on every site (single-site
   contraction on the physical leg);
3. per repetition, if entanglers are on: bring the MPS to right-canonical form
   (orthogonality centre on site 0), then for k = 0 .. n-2 in order apply
   RZZ(2 (pi - x_k)(pi - x_{k+1})) where the pair (k, k+1) is entangled (every pair of
   the chain, or only pairs inside a block for the block product structure, see
   ``circuit.entangled_bonds``), and split the two-site block by SVD, keeping the
   singular values s > cutoff * s_0 (at most chi_cap of them), rescaling the kept ones
   to the norm of the full spectrum, and moving the centre one site right. Across a
   block boundary no gate acts and the split only moves the centre (the bond there
   falls to 1).

With the default cutoff (1e-14) nothing but numerically zero singular values is
dropped, so the MPS equals the statevector to rounding. All samples of one call share
bond dimensions: the kept rank is the largest over the batch, and a sample's own
dropped singular values are set to zero instead.
"""
from __future__ import annotations

import numpy as np

from .circuit import entangled_bonds, entangler_angles, hadamard, rz, rzz_phases, single_qubit_angles


def _product_zero(m: int, n: int):
    sites = []
    for _ in range(n):
        a = np.zeros((m, 1, 2, 1), dtype=np.complex128)
        a[:, 0, 0, 0] = 1.0
        sites.append(a)
    return sites


def _apply_single_site(a: np.ndarray, gates: np.ndarray) -> np.ndarray:
    """a'[m, l, s, r] = sum_t gates[m, s, t] a[m, l, t, r]."""
    return np.einsum("mst,mltr->mlsr", gates, a)


def _right_canonicalize(sites) -> None:
    """Sweep right to left with LQ factorisations; afterwards sites 1..n-1 are right-orthonormal."""
    n = len(sites)
    for k in range(n - 1, 0, -1):
        a = sites[k]
        m, dl, _, dr = a.shape
        mat = a.reshape(m, dl, 2 * dr)
        # LQ of mat from the QR of its conjugate transpose: mat^H = q r  =>  mat = r^H q^H.
        q, r = np.linalg.qr(np.conj(np.swapaxes(mat, 1, 2)))
        rank = q.shape[2]
        sites[k] = np.conj(np.swapaxes(q, 1, 2)).reshape(m, rank, 2, dr)
        left = np.conj(np.swapaxes(r, 1, 2))  # (m, dl, rank)
        sites[k - 1] = np.einsum("mlsa,mar->mlsr", sites[k - 1], left)


def build_mps(x, reps: int, angle_scale: float = 2.0, entangle: bool = True,
              chi_cap: int | None = None, cutoff: float = 1e-14, block: int = 0):
    """Return (sites, discarded) for the samples in x (shape m x n).

    sites[k] has shape (m, D_{k}, 2, D_{k+1}); discarded[m] is the squared weight of the
    singular values dropped over the whole build (relative to a unit-norm state).
    """
    x = np.atleast_2d(np.asarray(x, dtype=np.float64))
    m, n = x.shape
    sites = _product_zero(m, n)
    discarded = np.zeros(m)
    h = hadamard()
    phis = single_qubit_angles(x, angle_scale)          # (m, n)
    thetas = np.stack([entangler_angles(row) for row in x]) if n > 1 else np.zeros((m, 0))
    bonds = entangled_bonds(n, block)
    for _ in range(reps):
        for k in range(n):
            gates = np.stack([rz(phis[i, k]) @ h for i in range(m)])
            sites[k] = _apply_single_site(sites[k], gates)
        if not entangle or n == 1:
            continue
        _right_canonicalize(sites)
        for k in range(n - 1):
            a, b = sites[k], sites[k + 1]
            dl, dr = a.shape[1], b.shape[3]
            pair = np.einsum("mlsa,matr->mlstr", a, b)
            if bonds[k]:
                phase = np.stack([rzz_phases(thetas[i, k]) for i in range(m)])  # (m, 2, 2)
                pair = pair * phase[:, None, :, :, None]
            mat = pair.reshape(m, dl * 2, 2 * dr)
            u, s, vh = np.linalg.svd(mat, full_matrices=False)
            s0 = s[:, :1]
            keep = s > cutoff * np.where(s0 > 0, s0, 1.0)
            if chi_cap is not None:
                keep[:, chi_cap:] = False
            rank = max(1, int(keep.sum(axis=1).max()))
            total = np.sum(s * s, axis=1)
            s_kept = np.where(keep, s, 0.0)[:, :rank]
            kept = np.sum(s_kept * s_kept, axis=1)
            discarded += np.where(total > 0, (total - kept) / np.where(total > 0, total, 1.0), 0.0)
            rescale = np.sqrt(np.where(kept > 0, total / np.where(kept > 0, kept, 1.0), 1.0))
            s_kept = s_kept * rescale[:, None]
            sites[k] = u[:, :, :rank].reshape(m, dl, 2, rank)
            sites[k + 1] = (s_kept[:, :, None] * vh[:, :rank, :]).reshape(m, rank, 2, dr)
    return sites, discarded


def bond_dims(sites):
    """[D_0, D_1, ..., D_n]: the bond dimension left of each site, and 1 at the right end."""
    return [sites[0].shape[1]] + [a.shape[3] for a in sites]


def to_statevector(sites, sample: int = 0) -> np.ndarray:
    """Contract one sample's MPS into a dense vector (qubit 0 most significant). Small n only."""
    v = sites[0][sample]  # (1, 2, D)
    v = v.reshape(2, -1)
    for a in sites[1:]:
        t = a[sample]  # (D, 2, D')
        v = np.einsum("pa,asr->psr", v, t).reshape(-1, t.shape[2])
    return v.reshape(-1)

