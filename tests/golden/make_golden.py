"""Write the stored expected values under tests/golden/ (calls only oracle/ and the input generator).

cfg1_kq16.txt: K_q (§II-C, Eq. 7) for the first 16 of the 64 tiny-case samples
(n = 8 qubits, features uniform in [0, pi] from PCG64 seed 0, ZZ-chain map, one
repetition), by brute-force statevector overlaps. Re-run this script only when the
oracle's arithmetic changes for a reason that the commit message cites.
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import circuit  # noqa: E402
from paper_2602_01330_gb300 import synthetic  # noqa: E402


def main():
    x = synthetic.uniform_angles(64, 8, seed=0)
    k = circuit.kernel_matrix(x[:16], x[:16], reps=1)
    header = ("K_q = |<psi(x_i)|psi(x_j)>|^2, paper §II-C Eq. 7; tiny case: n=8, 64 samples "
              "uniform in [0,pi] (PCG64 seed 0), ZZ-chain map, reps=1; rows/cols = samples 0..15; "
              "written by tests/golden/make_golden.py from the statevector oracle")
    np.savetxt(os.path.join(HERE, "cfg1_kq16.txt"), k, fmt="%.17e", header=header)


if __name__ == "__main__":
    main()
