"""Plant plausible mistakes in the oracle (on the CPU) and check that a pin catches each.

This is what makes the pins worth trusting: a dropped term, a wrong sign or index, a
transposed operand, a missing conjugate or a missing rescale in the oracle must each
move at least one pin past its tolerance.
"""
import numpy as real_np
import pytest

import closed_forms as cf
import pins
from oracle import blocks, circuit, gram, mps
from paper_2602_01330_gb300 import synthetic


class _Proxy:
    """Stands in for a module, overriding some attributes."""

    def __init__(self, base, **over):
        self._base = base
        self._over = over

    def __getattr__(self, name):
        if name in self._over:
            return self._over[name]
        return getattr(self._base, name)


def deep_underflow(n=2000):
    x = synthetic.uniform_angles(2, n, 41)
    sites, _ = mps.build_mps(x, 1)
    _, lkq = gram.pair_values(sites, sites, [0], [1])
    ref = cf.ising_log_kernel(x[0], x[1])
    got = lkq[0]
    return abs(got - ref) / abs(ref) if real_np.isfinite(got) else real_np.inf


PIN_SUITE = [
    ("product r1", lambda: pins.statevector_vs_product(1), 1e-12),
    ("product r2", lambda: pins.statevector_vs_product(2), 1e-12),
    ("ising", lambda: pins.statevector_vs_ising(6), 1e-12),
    ("dense r2", lambda: pins.statevector_vs_dense(4, 2), 1e-12),
    ("mps vs sv", lambda: pins.mps_vs_statevector(6, 2), 1e-11),
    ("mps vs sv r3", lambda: pins.mps_vs_statevector(7, 3), 1e-11),
    ("ranks", lambda: float(pins.bond_ranks(7, 2)), 0.5),
    ("deep underflow", deep_underflow, 1e-9),
    ("chain form 6 large n", lambda: pins.chain_large_n_vs_closed_form(60, 2, 2), 1e-10),
    ("bps kron", lambda: pins.bps_statevector_vs_kron(9, 2, 4), 1e-12),
    ("bps blocks", lambda: pins.bps_log_kernel_vs_block_products(20, 2, 6), 1e-10),
    ("full sv", lambda: pins.full_statevector_vs_dense(5, 2, 4), 1e-12),
    ("block mps", lambda: pins.block_mps_vs_products(12, 2, 6), 1e-10),
    ("single cut", pins.single_cut_truncation, 1e-12),
    ("rbf", pins.rbf_vs_library, 1e-12),
    ("rbf pairs", pins.rbf_pairs_vs_library, 1e-12),
    ("mix", pins.mix_limits, 1e-12),
]


def _failing_pins():
    failed = []
    for name, fn, tol in PIN_SUITE:
        try:
            val = fn()
        except Exception:  # a crash also counts as caught
            failed.append(name)
            continue
        if not (val <= tol):
            failed.append(name)
    return failed


def test_unmutated_oracle_passes_all_pins():
    assert _failing_pins() == []


_orig_rz = circuit.rz
_orig_rzz = circuit.rzz_phases


def _mut_rz_half(mp):
    f = lambda phi: _orig_rz(phi / 2)
    mp.setattr(circuit, "rz", f)
    mp.setattr(mps, "rz", f)


def _mut_rzz_sign(mp):
    f = lambda th: _orig_rzz(-th)
    mp.setattr(circuit, "rzz_phases", f)
    mp.setattr(mps, "rzz_phases", f)


def _mut_entangler_index(mp):
    def f(x):
        x = real_np.asarray(x, dtype=real_np.float64)
        return 2.0 * (real_np.pi - x[:-1]) ** 2
    mp.setattr(circuit, "entangler_angles", f)
    mp.setattr(mps, "entangler_angles", f)


def _mut_transposed_gate(mp):
    mp.setattr(mps, "_apply_single_site", lambda a, g: real_np.einsum("mts,mltr->mlsr", g, a))


def _mut_no_conj(mp):
    mp.setattr(gram, "np", _Proxy(real_np, conj=lambda a: a))


def _mut_svd_drops_s(mp):
    def svd(a, full_matrices=True):
        u, s, vh = real_np.linalg.svd(a, full_matrices=full_matrices)
        return u, real_np.ones_like(s), vh
    mp.setattr(mps, "np", _Proxy(real_np, linalg=_Proxy(real_np.linalg, svd=svd)))


def _mut_no_rescale(mp):
    mp.setattr(gram, "np", _Proxy(real_np, frexp=lambda a: (a, real_np.zeros(real_np.shape(a), dtype=int))))


def _mut_rbf_no_square(mp):
    mp.setattr(gram, "np", _Proxy(real_np, sum=lambda a, axis=None: real_np.sum(real_np.sqrt(real_np.abs(a)), axis=axis)))


_orig_rbf_pairs = gram.rbf_pairs


def _mut_rbf_pairs_one_side(mp):
    # both samples of a pair taken from the row set
    mp.setattr(gram, "rbf_pairs", lambda xr, xc, i, j, g: _orig_rbf_pairs(xr, xr, i, j, g))


def _mut_rbf_pairs_indices_swapped(mp):
    mp.setattr(gram, "rbf_pairs", lambda xr, xc, i, j, g: _orig_rbf_pairs(xr, xc, j, i, g))


def _mut_mix_swapped(mp):
    mp.setattr(gram, "dual_kernel", lambda kq, kc, w: (1 - w) * real_np.asarray(kq) + w * real_np.asarray(kc))


def _mut_hadamard_sign(mp):
    h = real_np.array([[1.0, 1.0], [-1.0, 1.0]], dtype=real_np.complex128) / real_np.sqrt(2.0)
    mp.setattr(circuit, "hadamard", lambda: h)
    mp.setattr(mps, "hadamard", lambda: h)


def _mut_block_boundary_shifted(mp):
    def bonds(n, block=0):
        i = real_np.arange(max(n - 1, 0))
        if block <= 0:
            return real_np.ones(i.shape, dtype=bool)
        return ((i + 1) // block) == ((i + 2) // block)
    mp.setattr(circuit, "entangled_bonds", bonds)
    mp.setattr(mps, "entangled_bonds", bonds)


def _mut_full_pairs_short_range(mp):
    good = circuit.entangled_pairs

    def pairs(n, block=0, entangler="chain"):
        return [(i, j) for i, j in good(n, block, entangler) if j - i <= 2]
    mp.setattr(circuit, "entangled_pairs", pairs)


def _mut_keeps_smallest(mp):
    def svd(a, full_matrices=True):
        u, s, vh = real_np.linalg.svd(a, full_matrices=full_matrices)
        return u[..., ::-1], s[..., ::-1], vh[..., ::-1, :]
    mp.setattr(blocks, "np", _Proxy(real_np, linalg=_Proxy(real_np.linalg, svd=svd)))


def _mut_no_renormalisation(mp):
    mp.setattr(blocks, "np", _Proxy(real_np, sqrt=lambda a: real_np.ones_like(a)))


MUTATIONS = {
    "full entangler skips long-range pairs": _mut_full_pairs_short_range,
    "truncation keeps the smallest singular values": _mut_keeps_smallest,
    "truncation not renormalised": _mut_no_renormalisation,
    "block boundary shifted by one": _mut_block_boundary_shifted,
    "rz angle halved": _mut_rz_half,
    "rzz sign flipped": _mut_rzz_sign,
    "entangler uses wrong neighbour": _mut_entangler_index,
    "single-site gate transposed": _mut_transposed_gate,
    "transfer without conjugate": _mut_no_conj,
    "svd split drops singular values": _mut_svd_drops_s,
    "no per-site rescale": _mut_no_rescale,
    "rbf distance not squared": _mut_rbf_no_square,
    "rbf pairs read both samples from the rows": _mut_rbf_pairs_one_side,
    "rbf pairs swap the pair indices": _mut_rbf_pairs_indices_swapped,
    "mix weights swapped": _mut_mix_swapped,
    "hadamard transposed": _mut_hadamard_sign,
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_mutation_is_caught(name, monkeypatch):
    MUTATIONS[name](monkeypatch)
    failed = _failing_pins()
    assert failed, f"planted mistake '{name}' passed every pin"
