"""The FP64 oracle against brute force, closed forms, invariants and library routines.

CPU only. Citations: feature state §II-C Eq. 6, quantum kernel Eqs. 7-10, RBF §II-B
Eq. 3, dual kernel §II-D Eq. 11.
"""
import numpy as np
import pytest

import closed_forms as cf
import pins
from oracle import circuit, gram, mps
from paper_2602_01330_gb300 import synthetic


@pytest.mark.parametrize("reps", [1, 2])
@pytest.mark.parametrize("c", [2.0, 1.0])
def test_statevector_product_closed_form(reps, c):
    # c = 1 gives prod cos^2((x - y)/2), c = 2 gives prod cos^2(x - y).
    assert pins.statevector_vs_product(reps, c) < 1e-13


@pytest.mark.parametrize("n", [2, 5, 8])
def test_statevector_ising_closed_form(n):
    assert pins.statevector_vs_ising(n) < 1e-13


@pytest.mark.parametrize("n,reps", [(3, 2), (4, 2), (4, 3), (5, 2)])
def test_statevector_matches_dense_unitaries(n, reps):
    assert pins.statevector_vs_dense(n, reps) < 1e-12


def test_ising_two_qubits_by_hand():
    x = synthetic.uniform_angles(6, 2, 31)
    for i in range(3):
        a = cf.two_qubit_amplitude(x[i], x[i + 3])
        la, ph = cf.ising_log_amplitude(x[i], x[i + 3])
        assert abs(np.exp(la) * ph - a) < 1e-14
        sv = circuit.statevector(x[i], 1)
        sw = circuit.statevector(x[i + 3], 1)
        assert abs(abs(np.vdot(sv, sw)) - abs(a)) < 1e-14


def test_statevector_is_normalised():
    x = synthetic.uniform_angles(3, 9, 32)
    for row in x:
        assert abs(np.linalg.norm(circuit.statevector(row, 3)) - 1.0) < 1e-13


@pytest.mark.parametrize("n,reps", [(2, 1), (3, 2), (8, 1), (8, 2), (9, 3), (10, 2), (12, 2)])
def test_mps_matches_statevector(n, reps):
    assert pins.mps_vs_statevector(n, reps) < 1e-12


def test_mps_matches_statevector_entanglers_off():
    assert pins.mps_vs_statevector(8, 2, entangle=False) < 1e-12


@pytest.mark.parametrize("n,reps", [(6, 1), (7, 2), (9, 3)])
def test_mps_amplitudes_match_statevector(n, reps):
    assert pins.mps_statevector_amplitudes(n, reps) < 1e-12


@pytest.mark.parametrize("reps", [1, 2, 3])
def test_bond_dimensions_are_exact_ranks(reps):
    assert pins.bond_ranks(9, reps) == 0


@pytest.mark.parametrize("n,reps,b", [(11, 2, 4), (12, 3, 6), (9, 2, 3), (7, 2, 7), (6, 2, 1)])
def test_bps_statevector_is_kron_of_blocks(n, reps, b):
    # b = n is the plain chain and b = 1 has no entanglers (cross-checks both ends)
    assert pins.bps_statevector_vs_kron(n, reps, b) < 1e-12


@pytest.mark.parametrize("n,reps,b", [(40, 2, 6), (784, 2, 6), (100, 3, 5)])
def test_bps_log_kernel_is_sum_over_blocks(n, reps, b):
    # n = 784 at two repetitions: the long-chain path (rescaling, log domain) exactly pinned
    assert pins.bps_log_kernel_vs_block_products(n, reps, b) < 1e-10


@pytest.mark.parametrize("reps", [1, 2, 3])
def test_bps_bond_dimensions(reps):
    assert pins.bps_bond_ranks(17, reps, 5) == 0


def test_block_limits():
    x = synthetic.uniform_angles(2, 9, 24)
    for row in x:
        np.testing.assert_allclose(circuit.statevector(row, 2, block=9), circuit.statevector(row, 2), atol=1e-15)
        np.testing.assert_allclose(circuit.statevector(row, 2, block=1),
                                   circuit.statevector(row, 2, entangle=False), atol=1e-15)
    assert circuit.entangled_bonds(7, 3).tolist() == [True, True, False, True, True, False]
    assert circuit.entangled_bonds(4, 0).tolist() == [True, True, True]


@pytest.mark.parametrize("n,reps,b", [(6, 2, 4), (8, 2, 8), (7, 3, 3)])
def test_full_entangler_statevector_vs_dense(n, reps, b):
    assert pins.full_statevector_vs_dense(n, reps, b) < 1e-12


@pytest.mark.parametrize("n,reps,b,ent", [(30, 2, 6, "full"), (23, 3, 5, "full"), (20, 2, 5, "chain"),
                                          (96, 2, 8, "full")])
def test_block_mps_untruncated_vs_block_products(n, reps, b, ent):
    assert pins.block_mps_vs_products(n, reps, b, ent) < 1e-10


@pytest.mark.parametrize("b,reps", [(7, 2), (8, 3), (6, 1)])
def test_block_mps_ranks_are_schmidt_ranks(b, reps):
    assert pins.block_mps_ranks(b, reps) == 0


@pytest.mark.parametrize("reps", [2, 3])
def test_single_cut_truncation_eckart_young(reps):
    assert pins.single_cut_truncation(reps) < 1e-12


def test_block_mps_chain_matches_tebd():
    """The chain entangler through block states + SVD equals the gate-by-gate TEBD MPS with
    the same blocks: same log K_q and the same bond dimensions (cutoff removes the exact zeros)."""
    from oracle import blocks
    x = synthetic.uniform_angles(4, 26, 29)
    a, _ = blocks.mps_from_block_states(x, 2, 7, "chain")
    t, _ = mps.build_mps(x, 2, block=7)
    ii, jj = np.triu_indices(4, 1)
    la = gram.pair_values(a, a, ii, jj)[1]
    lt = gram.pair_values(t, t, ii, jj)[1]
    np.testing.assert_allclose(la, lt, rtol=1e-11)
    assert mps.bond_dims(a) == mps.bond_dims(t)


@pytest.mark.parametrize("n,reps", [(5, 1), (6, 2), (7, 3), (4, 4), (3, 5)])
def test_chain_closed_form_matches_statevector(n, reps):
    assert pins.chain_closed_form_vs_statevector(n, reps) < 1e-12


@pytest.mark.parametrize("n,reps", [(784, 2), (784, 3), (256, 5)])
def test_oracle_chain_at_large_n_matches_closed_form(n, reps):
    # the plain chain at two or more repetitions, where no product or Ising form exists:
    # the oracle's gate-by-gate TEBD against the closed-form tensors, exact to rounding
    assert pins.chain_large_n_vs_closed_form(n, reps) < 1e-10


def test_large_n_ising_log_domain():
    # n = 784, one repetition with entanglers: off-diagonal K_q far below 1e-300.
    assert pins.large_n_ising(784) < 1e-10


@pytest.mark.parametrize("reps", [1, 2])
def test_large_n_product_log_domain(reps):
    assert pins.large_n_product(784, reps) < 1e-10


def test_near_duplicate_large_n_absolute():
    assert pins.near_duplicate_abs(784) < 1e-12


def test_invariants_fmnist_shape():
    assert pins.invariants(64, 40, 2) < 1e-12


def test_rbf_matches_scipy():
    assert pins.rbf_vs_library() < 1e-14


def test_rbf_pairs_matches_scipy():
    assert pins.rbf_pairs_vs_library() < 1e-14


def test_rbf_matches_sklearn():
    skl = pytest.importorskip("sklearn.metrics.pairwise")
    x = synthetic.fmnist_like(20, 0, 16)["x_train"].astype(np.float64)
    assert np.max(np.abs(gram.rbf(x, x, 1 / 16) - skl.rbf_kernel(x, x, gamma=1 / 16))) < 1e-14


def test_mix_limits():
    assert pins.mix_limits() < 1e-15


def test_underflowing_pair_keeps_log():
    # A pair whose K_q is below the float64 range still has a finite log K_q.
    x = synthetic.uniform_angles(2, 2000, 41)
    sites, _ = mps.build_mps(x, 1)
    kq, lkq = gram.pair_values(sites, sites, [0], [1])
    assert np.isfinite(lkq[0]) and lkq[0] < -745 and kq[0] == 0.0
    ref = cf.ising_log_kernel(x[0], x[1])
    assert abs(lkq[0] - ref) < 1e-10 * abs(ref)


def test_truncation_cap_reports_discarded_weight():
    x = synthetic.uniform_angles(3, 10, 42)
    _, disc_exact = mps.build_mps(x, 3)
    sites, disc = mps.build_mps(x, 3, chi_cap=4)
    assert np.all(disc_exact < 1e-20)
    assert np.all(disc > 1e-6)
    assert max(mps.bond_dims(sites)) <= 4
    # a truncated state stays normalised
    kq, _ = gram.gram_from_mps(sites, sites)
    assert np.max(np.abs(np.diag(kq) - 1.0)) < 1e-12
