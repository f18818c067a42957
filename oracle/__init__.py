"""FP64 CPU oracle for the quantum-classical dual kernel.

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline / reference leg of ``bench.py`` may import this package. The library in
``paper_2602_01330_gb300`` never imports it, and this package imports nothing from
the library: the two share no code. Both take their inputs from
``paper_2602_01330_gb300.synthetic``, which holds input generation only.

What it computes, in plain NumPy float64 / complex128 and in the paper's order:

* ``circuit``  -- the feature-map state |psi(x)> = U(x)|0>^n (§II-C, Eq. 6) by dense
  statevector simulation, for n <= 14;
* ``mps``      -- the same state as a matrix product state, built gate by gate with
  two-site SVD splits (time-evolving block decimation), for any n;
* ``blocks``   -- the MPS of a block-structured map (entanglers only inside blocks of b
  qubits, chain or all-to-all inside) from its dense block states by SVD sweeps with the
  cutoff / cap truncation and the discarded weight;
* ``gram``     -- the quantum kernel K_q = |<psi(x_i)|psi(x_j)>|^2 (§II-C, Eqs. 7-10)
  from the MPS by a left-to-right transfer contraction with power-of-two rescaling,
  the RBF kernel (§II-B, Eq. 3) and the linear mix (§II-D, Eq. 11);
* ``preprocess`` -- the data pre-processing of §II-A: standardisation, PCA (eigh of the
  covariance), min-max scaling;
* ``svm``      -- the SVM that consumes the kernel matrices: the dual problem of §II-B
  (Eqs. 1-2) by sequential minimal optimisation, the decision function (Eq. 5) and
  one-against-one voting.

Feature map. The paper's circuit figure (Fig. 1(B)) is not part of its text; §II-C
only says that Hadamards and data-dependent rotations alternate with local
entanglers. The reading taken is the ZZ chain: per repetition, H on every qubit,
RZ(angle_scale * x_i) on qubit i, then RZZ(2 (pi - x_i)(pi - x_{i+1})) on each
neighbouring pair of an open chain; the repetitions re-upload the same x.

Parity pins: every function here is checked in ``tests/test_oracle_pins.py`` against
brute force, closed forms and invariants that do not use this package's code.
"""
