"""Pin checks of the oracle: each returns the largest deviation from something the
paper or the mathematics fixes (brute force, closed forms, invariants, library
routines). ``test_oracle_pins`` asserts they are small; ``test_oracle_mutations``
plants mistakes in the oracle and asserts that some pin then fails.
"""
from __future__ import annotations

import numpy as np
from scipy.spatial.distance import cdist

import closed_forms as cf
from oracle import circuit, gram, mps
from paper_2602_01330_gb300 import synthetic


def statevector_vs_product(reps: int, c: float = 2.0, n: int = 6, seed: int = 11) -> float:
    """Statevector kernel with entanglers off vs the product closed forms (forms 1, 2)."""
    x = synthetic.uniform_angles(5, n, seed)
    k = circuit.kernel_matrix(x, x, reps, angle_scale=c, entangle=False)
    err = 0.0
    for i in range(5):
        for j in range(5):
            if reps == 1:
                ref = cf.product_kernel_r1(x[i], x[j], c)
            else:
                ref = float(np.prod(np.abs(cf.product_amplitudes_r2(x[i], x[j], c)) ** 2))
            err = max(err, abs(k[i, j] - ref))
    return err


def statevector_vs_ising(n: int = 7, c: float = 2.0, seed: int = 12) -> float:
    """Statevector kernel with entanglers, one repetition, vs the Ising form (form 3)."""
    x = synthetic.uniform_angles(5, n, seed)
    k = circuit.kernel_matrix(x, x, 1, angle_scale=c, entangle=True)
    err = 0.0
    for i in range(5):
        for j in range(5):
            err = max(err, abs(k[i, j] - np.exp(cf.ising_log_kernel(x[i], x[j], c))))
    return err


def statevector_vs_dense(n: int = 4, reps: int = 2, c: float = 2.0, seed: int = 18) -> float:
    """Oracle statevector kernel vs dense expm/Kronecker unitaries (form 5), any reps."""
    x = synthetic.uniform_angles(4, n, seed)
    k = circuit.kernel_matrix(x, x, reps, angle_scale=c, entangle=True)
    states = [cf.dense_state(row, reps, c) for row in x]
    err = 0.0
    for i in range(4):
        for j in range(4):
            err = max(err, abs(k[i, j] - abs(np.vdot(states[i], states[j])) ** 2))
    return err


def mps_vs_statevector(n: int, reps: int, entangle: bool = True, c: float = 2.0, seed: int = 13) -> float:
    """Oracle MPS + transfer Gram vs brute-force statevector overlaps (n <= 12)."""
    x = synthetic.uniform_angles(6, n, seed)
    ref = circuit.kernel_matrix(x, x, reps, angle_scale=c, entangle=entangle)
    sites, _ = mps.build_mps(x, reps, angle_scale=c, entangle=entangle)
    kq, _ = gram.gram_from_mps(sites, sites)
    return float(np.max(np.abs(kq - ref)))


def mps_statevector_amplitudes(n: int, reps: int, seed: int = 14) -> float:
    """Each sample's contracted MPS equals its statevector up to a global phase."""
    x = synthetic.uniform_angles(3, n, seed)
    sites, _ = mps.build_mps(x, reps)
    err = 0.0
    for i in range(3):
        v = mps.to_statevector(sites, i)
        s = circuit.statevector(x[i], reps)
        ph = np.vdot(v, s)
        ph = ph / abs(ph) if abs(ph) > 0 else 1.0
        err = max(err, float(np.max(np.abs(v * ph - s))))
    return err


def large_n_ising(n: int = 784, seed: int = 21) -> float:
    """Oracle log K_q at large n, one repetition, vs the Ising recursion; relative in log."""
    d = synthetic.fmnist_like(6, 0, n)["x_train"].astype(np.float64)
    rng = np.random.Generator(np.random.PCG64(seed))
    near = np.clip(d[:2] + rng.normal(0, 1e-3, size=d[:2].shape), 0, np.pi)
    x = np.concatenate([d, near])
    sites, _ = mps.build_mps(x, 1)
    pairs = [(0, 1), (0, 2), (3, 5), (0, 6), (1, 7), (4, 4)]
    i_idx = [p[0] for p in pairs]
    j_idx = [p[1] for p in pairs]
    _, lkq = gram.pair_values(sites, sites, i_idx, j_idx)
    err = 0.0
    for (i, j), got in zip(pairs, lkq):
        ref = cf.ising_log_kernel(x[i], x[j])
        err = max(err, abs(got - ref) / max(1.0, abs(ref)))
    return err


def large_n_product(n: int = 784, reps: int = 2, seed: int = 22) -> float:
    """Entanglers off at large n vs the product closed forms, relative in log."""
    x = synthetic.uniform_angles(4, n, seed)
    x[3] = np.clip(x[0] + 1e-3, 0, np.pi)
    sites, _ = mps.build_mps(x, reps, entangle=False)
    pairs = [(0, 1), (1, 2), (0, 3), (2, 2)]
    _, lkq = gram.pair_values(sites, sites, [p[0] for p in pairs], [p[1] for p in pairs])
    err = 0.0
    for (i, j), got in zip(pairs, lkq):
        ref = cf.product_log_kernel_r1(x[i], x[j]) if reps == 1 else cf.product_log_kernel_r2(x[i], x[j])
        err = max(err, abs(got - ref) / max(1.0, abs(ref)))
    return err


def near_duplicate_abs(n: int = 784, seed: int = 23) -> float:
    """|K_q - closed form| for a near-duplicate pair at large n (K_q close to 1)."""
    x = synthetic.uniform_angles(1, n, seed)
    rng = np.random.Generator(np.random.PCG64(seed + 1))
    y = np.clip(x + rng.normal(0, 2e-3, size=x.shape), 0, np.pi)
    both = np.concatenate([x, y])
    sites, _ = mps.build_mps(both, 1)
    kq, _ = gram.pair_values(sites, sites, [0], [1])
    return float(abs(kq[0] - np.exp(cf.ising_log_kernel(x[0], y[0]))))


def bond_ranks(n: int = 9, reps: int = 2, seed: int = 15) -> int:
    """Number of bonds whose oracle-MPS dimension or statevector Schmidt rank differs from
    min(2^k, 2^(n-k), 2^reps)."""
    x = synthetic.uniform_angles(2, n, seed)
    sites, _ = mps.build_mps(x, reps)
    dims = mps.bond_dims(sites)
    bad = 0
    for k in range(1, n):
        want = cf.exact_bond_rank(n, reps, k)
        psi = circuit.statevector(x[0], reps)
        sv = np.linalg.svd(psi.reshape(2 ** k, 2 ** (n - k)), compute_uv=False)
        rank = int(np.sum(sv > 1e-12 * sv[0]))
        bad += int(dims[k] != want) + int(rank != want)
    return bad


def invariants(n: int = 64, m: int = 40, reps: int = 2) -> float:
    """Diagonal = 1, symmetry, 0 <= K <= 1, PSD, chain reversal, on Fashion-MNIST-shaped data."""
    x = synthetic.fmnist_like(m, 0, n)["x_train"].astype(np.float64)
    sites, _ = mps.build_mps(x, reps)
    kq, _ = gram.gram_from_mps(sites, sites)
    err = float(np.max(np.abs(np.diag(kq) - 1.0)))
    err = max(err, float(np.max(np.abs(kq - kq.T))))
    err = max(err, float(max(0.0, -kq.min())), float(max(0.0, kq.max() - 1.0 - 1e-12)))
    lam = np.linalg.eigvalsh(0.5 * (kq + kq.T))
    err = max(err, float(max(0.0, -lam.min())))
    rev, _ = mps.build_mps(x[:, ::-1].copy(), reps)
    kr, _ = gram.gram_from_mps(rev, rev)
    err = max(err, float(np.max(np.abs(kr - kq))))
    return err


def rbf_vs_library(seed: int = 16) -> float:
    x = synthetic.fmnist_like(30, 10, 64)
    a, b = x["x_train"].astype(np.float64), x["x_test"].astype(np.float64)
    gamma = 1.0 / 64
    ref = np.exp(-gamma * cdist(a, b, "sqeuclidean"))
    return float(np.max(np.abs(gram.rbf(a, b, gamma) - ref)))


def rbf_pairs_vs_library(seed: int = 19) -> float:
    """The oracle's pair-list RBF (used by the CPU baseline) against scipy's squared
    Euclidean cdist on the same pairs: random (i, j) of a rectangular set, i = j, and pairs
    listed out of order and repeated."""
    x = synthetic.fmnist_like(30, 12, 64)
    a, b = x["x_train"].astype(np.float64), x["x_test"].astype(np.float64)
    gamma = 1.0 / 64
    rng = np.random.Generator(np.random.PCG64(seed))
    ii = np.concatenate([rng.integers(0, 30, 50), np.arange(12), [29, 0, 29]])
    jj = np.concatenate([rng.integers(0, 12, 50), np.arange(12), [11, 0, 11]])
    ref = np.exp(-gamma * cdist(a, b, "sqeuclidean"))[ii, jj]
    err = float(np.max(np.abs(gram.rbf_pairs(a, b, ii, jj, gamma) - ref)))
    same = np.exp(-gamma * cdist(a, a, "sqeuclidean"))[ii, ii[::-1]]
    return max(err, float(np.max(np.abs(gram.rbf_pairs(a, a, ii, ii[::-1], gamma) - same))))


def mix_limits() -> float:
    x = synthetic.uniform_angles(8, 5, 17)
    kq, _ = gram.quantum_gram(x, reps=2)
    kc = gram.rbf(x, x, 0.2)
    e = float(np.max(np.abs(gram.dual_kernel(kq, kc, 1.0) - kq)))
    e = max(e, float(np.max(np.abs(gram.dual_kernel(kq, kc, 0.0) - kc))))
    return e


def _blocks(n: int, b: int):
    return [(s, min(s + b, n)) for s in range(0, n, b)]


def bps_statevector_vs_kron(n: int = 11, reps: int = 2, b: int = 4, seed: int = 21) -> float:
    """Block product structure (§II-C): the oracle statevector with blocks of b qubits vs
    the Kronecker product of the blocks' own chain states from dense unitaries (form 5)."""
    from functools import reduce
    x = synthetic.uniform_angles(3, n, seed)
    err = 0.0
    for row in x:
        got = circuit.statevector(row, reps, block=b)
        ref = reduce(np.kron, [cf.dense_state(row[s:e], reps) for s, e in _blocks(n, b)])
        err = max(err, float(np.max(np.abs(got - ref))))
    return err


def bps_log_kernel_vs_block_products(n: int = 40, reps: int = 2, b: int = 6, seed: int = 22) -> float:
    """Oracle MPS + transfer log K_q with blocks of b qubits vs the sum over blocks of
    log |<psi_B(x)|psi_B(y)>|^2, each block state from dense unitaries (form 5). Exact at
    any n, so it pins the oracle's long-chain path at reps >= 2 (largest relative error)."""
    x = synthetic.uniform_angles(4, n, seed)
    sites, _ = mps.build_mps(x, reps, block=b)
    ii, jj = np.triu_indices(4, 1)
    _, lkq = gram.pair_values(sites, sites, ii, jj)
    err = 0.0
    for p, (i, j) in enumerate(zip(ii, jj)):
        ref = 0.0
        for s, e in _blocks(n, b):
            a = np.vdot(cf.dense_state(x[i, s:e], reps), cf.dense_state(x[j, s:e], reps))
            ref += np.log(abs(a) ** 2)
        err = max(err, abs(lkq[p] - ref) / max(1.0, abs(ref)))
    return err


def bps_bond_ranks(n: int = 17, reps: int = 2, b: int = 5) -> int:
    """Bond dimensions of the oracle MPS with blocks of b qubits vs the exact Schmidt ranks:
    1 at a block boundary, min(2^(k - start), 2^(end - k), 2^reps) inside a block. Returns
    the number of mismatching bonds."""
    x = synthetic.uniform_angles(3, n, 23)
    sites, _ = mps.build_mps(x, reps, block=b)
    dims = mps.bond_dims(sites)
    bad = 0
    for k in range(1, n):
        s = (k // b) * b
        e = min(s + b, n)
        ref = 1 if k == s else min(2 ** (k - s), 2 ** (e - k), 2 ** reps)
        bad += int(dims[k] != ref)
    return bad


def full_statevector_vs_dense(n: int = 6, reps: int = 2, b: int = 4, seed: int = 25) -> float:
    """All-to-all ZZ inside blocks: the oracle statevector vs the Kronecker product of dense
    expm unitaries with the ZZ generator on every pair of each block (form 5)."""
    from functools import reduce
    x = synthetic.uniform_angles(3, n, seed)
    err = 0.0
    for row in x:
        got = circuit.statevector(row, reps, block=b, entangler="full")
        ref = reduce(np.kron, [cf.dense_state(row[s:e], reps, all_pairs=True) for s, e in _blocks(n, b)])
        err = max(err, float(np.max(np.abs(got - ref))))
    return err


def block_mps_vs_products(n: int = 30, reps: int = 2, b: int = 6, entangler: str = "full", seed: int = 26) -> float:
    """Untruncated MPS from block states + the transfer Gram vs the sum over blocks of log
    overlaps of dense block states (form 5), largest relative error of log K_q."""
    from oracle import blocks
    x = synthetic.uniform_angles(4, n, seed)
    sites, disc = blocks.mps_from_block_states(x, reps, b, entangler, cutoff=1e-14)
    ii, jj = np.triu_indices(4, 1)
    _, lkq = gram.pair_values(sites, sites, ii, jj)
    err = float(np.max(disc))
    for p, (i, j) in enumerate(zip(ii, jj)):
        ref = 0.0
        for s, e in _blocks(n, b):
            a = np.vdot(cf.dense_state(x[i, s:e], reps, all_pairs=entangler == "full"),
                        cf.dense_state(x[j, s:e], reps, all_pairs=entangler == "full"))
            ref += np.log(abs(a) ** 2)
        err = max(err, abs(lkq[p] - ref) / max(1.0, abs(ref)))
    return err


def block_mps_ranks(b: int = 7, reps: int = 2, seed: int = 27) -> int:
    """Bond dimensions of the untruncated block MPS vs the numerical Schmidt ranks of the
    dense block state (form 5) at every cut; number of mismatches."""
    from oracle import blocks, mps as omps
    x = synthetic.uniform_angles(1, b, seed)
    sites, _ = blocks.mps_from_block_states(x, reps, b, "full", cutoff=1e-10)
    dims = omps.bond_dims(sites)
    psi = cf.dense_state(x[0], reps, all_pairs=True)
    bad = 0
    for k in range(1, b):
        s = np.linalg.svd(psi.reshape(2 ** k, -1), compute_uv=False)
        bad += int(dims[k] != int(np.sum(s > 1e-10 * s[0])))
    return bad


def single_cut_truncation(reps: int = 2, seed: int = 28) -> float:
    """A 6-qubit all-to-all block capped at bond 4: only the middle cut (rank 8) truncates.
    Eckart-Young: the discarded weight is the squared tail of that cut's singular values of
    the dense state, and the renormalised result has |<psi_t|psi>|^2 = 1 - discarded.
    Returns the larger deviation of the two."""
    from oracle import blocks, mps as omps
    x = synthetic.uniform_angles(2, 6, seed)
    sites, disc = blocks.mps_from_block_states(x, reps, 6, "full", chi_cap=4)
    err = 0.0
    for i in range(2):
        psi = cf.dense_state(x[i], reps, all_pairs=True)
        s = np.linalg.svd(psi.reshape(8, 8), compute_uv=False)
        tail = float(np.sum(s[4:] ** 2) / np.sum(s ** 2))
        fid = abs(np.vdot(omps.to_statevector(sites, i), psi)) ** 2
        err = max(err, abs(disc[i] - tail), abs(fid - (1.0 - tail)))
        if tail < 1e-6:  # the pin needs a truncation that bites
            return 1.0
    return err


def chain_closed_form_vs_statevector(n: int = 6, reps: int = 2, seed: int = 51) -> float:
    """Form 6 (the chain MPS written from the gate algebra) against the oracle's brute-force
    statevector overlaps: largest |ln|a| difference|."""
    x = synthetic.uniform_angles(3, n, seed)
    err = 0.0
    for i in range(2):
        a = np.vdot(circuit.statevector(x[i], reps), circuit.statevector(x[i + 1], reps))
        err = max(err, abs(np.log(abs(a)) - cf.chain_log_overlap(x[i], x[i + 1], reps)))
    return err


def chain_large_n_vs_closed_form(n: int = 784, reps: int = 2, pairs: int = 3) -> float:
    """The oracle's TEBD MPS + transfer log K_q of the chain at large n against form 6 (an
    independent algorithm: closed-form tensors, no SVD), largest relative error."""
    x = synthetic.fmnist_like(pairs + 1, 0, n)["x_train"].astype(np.float64)
    sites, _ = mps.build_mps(x, reps)
    _, lkq = gram.pair_values(sites, sites, list(range(pairs)), list(range(1, pairs + 1)))
    ref = np.array([2.0 * cf.chain_log_overlap(x[i], x[i + 1], reps) for i in range(pairs)])
    return float(np.max(np.abs(np.asarray(lkq) - ref) / np.maximum(1.0, np.abs(ref))))
