"""Work accounting for the transfer-chain Gram (units, algorithmic flops and bytes).

Unit of work: one entry x qubit = one (row, column) pair advanced through one site of
the transfer chain. For a pair the exact bond dimensions of the ZZ-chain MPS are
D_k = min(2^k, 2^(n-k), 2^reps) (D_0 = D_n = 1).

Dense count: site k costs 4 D_{k-1} D_k (D_{k-1} + D_k) complex multiply-adds =
16 (D_{k-1}^2 D_k + D_{k-1} D_k^2) real flops (2048 at D = 4).

Block count (what the kernels execute): every bond splits into two blocks by the copied
computational bit of the qubit on its left (sizes d = D/2, or (1, 0) for the trivial
left bond of site 1 and (1, 1) for the summed right bond of site n), the transfer
matrix is block diagonal, and site k costs
sum_{s,t} (d_{k-1,t}^2 d_{k,s} + d_{k-1,t} d_{k,s}^2) complex multiply-adds, 8 flops each
(512 at D = 4). The roofline uses the block count.
"""
from __future__ import annotations

from functools import lru_cache

FP32_LANES_PER_SM = 128  # FP32 FMA lanes per Blackwell SM


def exact_bonds(n: int, reps: int):
    return [min(2 ** k, 2 ** (n - k), 2 ** reps) for k in range(n + 1)]


@lru_cache(maxsize=None)
def dense_flops_per_pair(n: int, reps: int) -> int:
    d = exact_bonds(n, reps)
    return sum(16 * (d[k - 1] ** 2 * d[k] + d[k - 1] * d[k] ** 2) for k in range(1, n + 1))


def _blocks(n: int, reps: int, k: int):
    """Block sizes (block 0, block 1) of the bond left of site k (k = 0..n)."""
    d = exact_bonds(n, reps)[k]
    if k == 0:
        return (1, 0)
    if k == n:
        return (1, 1)
    return (d // 2, d // 2)


@lru_cache(maxsize=None)
def flops_per_pair(n: int, reps: int) -> int:
    total = 0
    for k in range(1, n + 1):
        left = _blocks(n, reps, k - 1)
        right = _blocks(n, reps, k)
        for dt in left:
            for ds in right:
                total += 8 * (dt * dt * ds + dt * ds * ds)
    return total


def gram_entries(m: int, symmetric: bool = True, b: int | None = None) -> int:
    """Unique entries: m(m+1)/2 for a symmetric Gram, b*m for a row block."""
    if symmetric:
        return m * (m + 1) // 2
    return int(b) * m


def fp32_peak_tflops(sm_count: int, sm_mhz: float) -> float:
    """FP32 FMA peak: SMs x 128 lanes x 2 flops x clock."""
    return sm_count * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12


def mps_site_bytes(chi_max: int, complex_bytes: int = 8) -> int:
    return 2 * chi_max * chi_max * complex_bytes
