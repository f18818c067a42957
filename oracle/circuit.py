"""Dense statevector simulation of the feature-map circuit (§II-C, Eq. 6).

Test infrastructure only (see the package header). Plain and slow: the state is a
complex128 array of shape (2,)*n, axis q is qubit q, and gates are applied one at a
time in circuit order. Use for n <= 14.
"""
from __future__ import annotations

import numpy as np


def hadamard() -> np.ndarray:
    return np.array([[1.0, 1.0], [1.0, -1.0]], dtype=np.complex128) / np.sqrt(2.0)


def rz(phi: float) -> np.ndarray:
    """RZ(phi) = diag(exp(-i phi/2), exp(+i phi/2))."""
    return np.diag([np.exp(-0.5j * phi), np.exp(0.5j * phi)]).astype(np.complex128)


def rzz_phases(theta: float) -> np.ndarray:
    """Diagonal of RZZ(theta) = exp(-i theta/2 Z(x)Z) as a 2x2 array indexed [z_a, z_b]."""
    same = np.exp(-0.5j * theta)
    diff = np.exp(0.5j * theta)
    return np.array([[same, diff], [diff, same]], dtype=np.complex128)


def single_qubit_angles(x: np.ndarray, angle_scale: float = 2.0) -> np.ndarray:
    """Rotation angle of RZ on each qubit: angle_scale * x_i."""
    return angle_scale * np.asarray(x, dtype=np.float64)


def entangler_angles(x: np.ndarray) -> np.ndarray:
    """RZZ angle on the pair (i, i+1) of the open chain: 2 (pi - x_i)(pi - x_{i+1})."""
    x = np.asarray(x, dtype=np.float64)
    return 2.0 * (np.pi - x[:-1]) * (np.pi - x[1:])


def entangled_bonds(n: int, block: int = 0) -> np.ndarray:
    """Which neighbouring pairs (i, i+1), i = 0 .. n-2, carry an RZZ.

    block = 0 (or >= n): every pair, the open chain. block = b >= 1: the block product
    (BPS) structure of §II-C, qubits grouped into blocks of b consecutive qubits with
    entanglers only inside a block, so pair (i, i+1) is entangled when i and i+1 fall in
    the same block (the last block may be shorter).
    """
    i = np.arange(max(n - 1, 0))
    if block <= 0:
        return np.ones(i.shape, dtype=bool)
    return (i // block) == ((i + 1) // block)


def entangled_pairs(n: int, block: int = 0, entangler: str = "chain"):
    """The qubit pairs (i, j), i < j, that carry an RZZ(2 (pi - x_i)(pi - x_j)).

    entangler = "chain": neighbouring pairs (i, i+1) inside a block (``entangled_bonds``).
    entangler = "full": every pair inside a block (all-to-all two-local ZZ within each block;
    block = 0 makes the whole register one block).
    """
    if entangler == "chain":
        return [(i, i + 1) for i in np.flatnonzero(entangled_bonds(n, block))]
    if entangler != "full":
        raise ValueError(f"unknown entangler {entangler!r}")
    b = n if block <= 0 else block
    return [(i, j) for i in range(n) for j in range(i + 1, n) if i // b == j // b]


def _apply_1q(psi: np.ndarray, gate: np.ndarray, q: int) -> np.ndarray:
    out = np.tensordot(gate, psi, axes=([1], [q]))
    return np.moveaxis(out, 0, q)


def _apply_zz(psi: np.ndarray, theta: float, q: int, r: int | None = None) -> np.ndarray:
    """RZZ(theta) on qubits q and r (default q + 1)."""
    r = q + 1 if r is None else r
    n = psi.ndim
    shape = [1] * n
    shape[q] = 2
    shape[r] = 2
    return psi * rzz_phases(theta).reshape(shape)


def statevector(x, reps: int, angle_scale: float = 2.0, entangle: bool = True, block: int = 0,
                entangler: str = "chain") -> np.ndarray:
    """|psi(x)> = [U_ZZ(x) . (x)_i RZ(angle_scale x_i) . H^(x)n]^reps |0...0>, flattened.

    U_ZZ holds the RZZ of every pair that ``entangled_pairs(n, block, entangler)`` lists
    (the gates are diagonal and commute). Qubit 0 is the most significant bit of the
    flattened index.
    """
    x = np.asarray(x, dtype=np.float64)
    n = x.shape[0]
    if n > 14:
        raise ValueError("statevector oracle is limited to n <= 14")
    psi = np.zeros((2,) * n, dtype=np.complex128)
    psi[(0,) * n] = 1.0
    h = hadamard()
    phis = single_qubit_angles(x, angle_scale)
    pairs = entangled_pairs(n, block, entangler)
    for _ in range(reps):
        for q in range(n):
            psi = _apply_1q(psi, h, q)
        for q in range(n):
            psi = _apply_1q(psi, rz(phis[q]), q)
        if entangle:
            for q, r in pairs:
                psi = _apply_zz(psi, 2.0 * (np.pi - x[q]) * (np.pi - x[r]), q, r)
    return psi.reshape(-1)


def kernel_matrix(x_rows, x_cols, reps: int, angle_scale: float = 2.0, entangle: bool = True,
                  block: int = 0, entangler: str = "chain") -> np.ndarray:
    """K_q[i, j] = |<psi(x_i)|psi(x_j)>|^2 (Eq. 7) by brute-force statevectors."""
    a = np.stack([statevector(x, reps, angle_scale, entangle, block, entangler) for x in np.asarray(x_rows)])
    b = np.stack([statevector(x, reps, angle_scale, entangle, block, entangler) for x in np.asarray(x_cols)])
    amp = a.conj() @ b.T
    return np.abs(amp) ** 2
