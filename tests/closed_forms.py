"""Closed forms that pin the oracle, derived by hand and independent of oracle/.

ZZ-chain feature map, qubit i carries x_i:
  per repetition H on every qubit, RZ(c x_i) with RZ(p) = diag(e^{-ip/2}, e^{ip/2}),
  then RZZ(2 (pi - x_i)(pi - x_{i+1})) = exp(-i (pi-x_i)(pi-x_{i+1}) Z_i Z_{i+1}).

1. Entanglers off, one repetition. Each qubit is RZ(c x)H|0> =
   (e^{-icx/2}|0> + e^{icx/2}|1>)/sqrt2, so <psi(x)|psi(y)> = prod_i cos(c (x_i - y_i)/2)
   and K_q = prod_i cos^2(c (x_i - y_i)/2); for c = 2 this is prod cos^2(x_i - y_i).
2. Entanglers off, two repetitions. Per qubit, with p = c x and q = c y,
   (RZ H)^2 |0> = (e^{-ip/2} cos(p/2), -i e^{ip/2} sin(p/2)), hence
   <.|.> = e^{i(p-q)/2} cos(p/2)cos(q/2) + e^{-i(p-q)/2} sin(p/2)sin(q/2).
3. Entanglers on, one repetition (Ising form). With sigma_i = (-1)^{z_i},
   psi_x(sigma) = 2^{-n/2} exp(-i sum c x_i sigma_i/2 - i sum (pi-x_i)(pi-x_{i+1}) sigma_i sigma_{i+1}),
   so <psi(x)|psi(y)> = 2^{-n} sum_sigma exp(i sum h_i sigma_i + i sum J_i sigma_i sigma_{i+1})
   with h_i = c (x_i - y_i)/2 and J_i = (pi-x_i)(pi-x_{i+1}) - (pi-y_i)(pi-y_{i+1}).
   The sum over sigma is a 2-state transfer recursion along the chain, kept in log scale.
4. n = 2 of form 3 by hand: sum over sigma_2 first gives
   a = (e^{i h_1} cos(h_2 + J_1) + e^{-i h_1} cos(h_2 - J_1)) / 2.
5. Any number of repetitions, small n: the circuit as a product of dense 2^n x 2^n
   unitaries, each the matrix exponential of its Pauli generator (RZ(p) = exp(-i p Z/2),
   RZZ(t) = exp(-i t Z(x)Z/2), H = (X + Z)/sqrt2) placed by Kronecker products. This
   shares nothing with the oracle's gate-by-gate tensor contractions.
"""
from __future__ import annotations

import numpy as np


def product_kernel_r1(x, y, c=2.0):
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    return float(np.prod(np.cos(c * (x - y) / 2.0) ** 2))


def product_log_kernel_r1(x, y, c=2.0):
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    return float(np.sum(2.0 * np.log(np.abs(np.cos(c * (x - y) / 2.0)))))


def product_amplitudes_r2(x, y, c=2.0):
    p = c * np.asarray(x, dtype=np.float64)
    q = c * np.asarray(y, dtype=np.float64)
    d = (p - q) / 2.0
    return np.exp(1j * d) * np.cos(p / 2) * np.cos(q / 2) + np.exp(-1j * d) * np.sin(p / 2) * np.sin(q / 2)


def product_log_kernel_r2(x, y, c=2.0):
    return float(np.sum(2.0 * np.log(np.abs(product_amplitudes_r2(x, y, c)))))


def ising_log_amplitude(x, y, c=2.0):
    """(log|a|, a / |a|) of a = <psi(x)|psi(y)> for one repetition with entanglers."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    n = x.shape[0]
    h = c * (x - y) / 2.0
    jj = (np.pi - x[:-1]) * (np.pi - x[1:]) - (np.pi - y[:-1]) * (np.pi - y[1:])
    sig = np.array([1.0, -1.0])
    v = np.exp(1j * h[0] * sig) / 2.0
    log_scale = 0.0
    for k in range(1, n):
        coupling = np.exp(1j * jj[k - 1] * np.outer(sig, sig))  # [sigma, sigma']
        v = (v @ coupling) * np.exp(1j * h[k] * sig) / 2.0
        s = np.max(np.abs(v))
        if s > 0:
            v = v / s
            log_scale += np.log(s)
    a = np.sum(v)
    if a == 0:
        return -np.inf, 0.0
    return float(np.log(np.abs(a)) + log_scale), a / np.abs(a)


def ising_log_kernel(x, y, c=2.0):
    la, _ = ising_log_amplitude(x, y, c)
    return 2.0 * la


def two_qubit_amplitude(x, y, c=2.0):
    h1 = c * (x[0] - y[0]) / 2.0
    h2 = c * (x[1] - y[1]) / 2.0
    j1 = (np.pi - x[0]) * (np.pi - x[1]) - (np.pi - y[0]) * (np.pi - y[1])
    return 0.5 * (np.exp(1j * h1) * np.cos(h2 + j1) + np.exp(-1j * h1) * np.cos(h2 - j1))


def dense_state(x, reps, c=2.0, entangle=True, all_pairs=False):
    """Form 5: U(x)|0...0> from Kronecker products of expm'd Pauli generators (n <= 8);
    all_pairs puts the ZZ generator on every pair (q, r), q < r, not just neighbours."""
    from functools import reduce
    from scipy.linalg import expm

    x = np.asarray(x, dtype=np.float64)
    n = x.shape[0]
    pauli_x = np.array([[0, 1], [1, 0]], dtype=np.complex128)
    pauli_z = np.array([[1, 0], [0, -1]], dtype=np.complex128)
    eye = np.eye(2, dtype=np.complex128)
    had = (pauli_x + pauli_z) / np.sqrt(2.0)

    def place(ops):
        return reduce(np.kron, [ops.get(q, eye) for q in range(n)])

    u = np.eye(2 ** n, dtype=np.complex128)
    for _ in range(reps):
        for q in range(n):
            u = place({q: had}) @ u
        for q in range(n):
            u = expm(-0.5j * c * x[q] * place({q: pauli_z})) @ u
        if entangle:
            pairs = [(q, r) for q in range(n) for r in range(q + 1, n)] if all_pairs else \
                [(q, q + 1) for q in range(n - 1)]
            for q, r in pairs:
                t = 2.0 * (np.pi - x[q]) * (np.pi - x[r])
                u = expm(-0.5j * t * place({q: pauli_z, r: pauli_z})) @ u
    return u[:, 0]


def exact_bond_rank(n: int, reps: int, bond: int) -> int:
    """Schmidt rank bound across the cut left of site `bond` (1..n-1) for the ZZ chain."""
    return min(2 ** bond, 2 ** (n - bond), 2 ** reps)


def chain_site_tensors(x, reps, c=2.0):
    """Form 6: the ZZ-chain state as an MPS written down from the gate algebra, for any reps.

    Expanding every H^(x)n layer over computational-basis states, the amplitude of the final
    basis state is a sum over the intermediate bit strings b^(1..reps-1) (b^(0) = 0...0). Per
    qubit q collect its bits across repetitions into c_q (bit rho-1 = b^(rho)_q, so the top bit
    is the output bit). Each H contributes 2^(-1/2) (-1)^(b^(rho)_q b^(rho-1)_q), each RZ layer
    exp(-i c x_q z/2) and each RZZ layer exp(-i (pi - x_q)(pi - x_{q+1}) z_q z_{q+1}), z = 1 - 2b.
    Summed over rho these depend on c_q alone (site factor) and on (c_q, c_{q+1}) (bond
    factor), so A^(q)_s[c_{q-1}][c_q] = [top bit of c_q = s] F_q(c_q) W_{q-1}(c_{q-1}, c_q).
    Returns a list of arrays (2, D_left, D_right) with D = 2^reps (1 at the left end)."""
    x = np.asarray(x, dtype=np.float64)
    n = x.shape[0]
    dim = 2 ** reps
    cs = np.arange(dim)
    bits = (cs[:, None] >> np.arange(reps)[None, :]) & 1          # [c, rho-1] = b^(rho)
    z = 1 - 2 * bits
    had = np.array([(-1.0) ** sum(bits[cc, r] * bits[cc, r - 1] for r in range(1, reps)) for cc in cs])
    top = bits[:, reps - 1]
    sites = []
    for q in range(n):
        f = 2.0 ** (-reps / 2) * had * np.exp(-0.5j * c * x[q] * z.sum(axis=1))
        if q == 0:
            w = np.ones((1, dim))
        else:
            j = (np.pi - x[q - 1]) * (np.pi - x[q])
            w = np.exp(-1j * j * (z[:, None, :] * z[None, :, :]).sum(axis=2))   # [c_{q-1}, c_q]
        a = np.zeros((2, w.shape[0], dim), dtype=np.complex128)
        for s in (0, 1):
            a[s] = w * (f * (top == s))[None, :]
        sites.append(a)
    return sites


def chain_log_overlap(x, y, reps, c=2.0):
    """ln|<psi(x)|psi(y)>| from the form-6 tensors by a left-to-right transfer contraction
    with an exact power-of-two rescale after every site (the right end sums the bond)."""
    ax, ay = chain_site_tensors(x, reps, c), chain_site_tensors(y, reps, c)
    e = np.ones((1, 1), dtype=np.complex128)
    exp2 = 0
    for a, b in zip(ax, ay):
        e = a[0].conj().T @ e @ b[0] + a[1].conj().T @ e @ b[1]
        _, ex = np.frexp(np.max(np.abs(e)))
        e = e * np.ldexp(1.0, -int(ex))  # an exact power of two
        exp2 += int(ex)
    amp = e.sum()
    return float(np.log(abs(amp)) + exp2 * np.log(2.0))
