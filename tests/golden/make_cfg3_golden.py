"""Write tests/golden/cfg3_sampled_pairs.txt: FP64 oracle values of the precision-form
workload on its sampled pairs (calls only oracle/, through tests/oracle_pool.py, and the
input generator).

Workload (precision form): d = 256 Fashion-MNIST-shaped features, 4000 samples
(synthetic.fmnist_like(4000, 0, 256), training seed), ZZ-chain map at reps = 3 (exact
bond 8) and reps = 5 (bond 32, the tensor-core case). Pairs, drawn with PCG64 seed 0:

* 1000 uniform pairs i < j;
* 500 nearest-neighbour pairs (sample i and its nearest other sample by Euclidean
  distance of the features, i drawn without replacement);
* 500 diagonal pairs (i, i);
* 200 near-duplicate pairs: sample b_k (drawn without replacement) against its perturbed
  copy synthetic.near_copies(x[b], 1e-4, 2.5e-2, seed=65)[k]. At 256 qubits even nearest
  neighbours have K_q far below 1e-3; these pairs spread K_q over about 1e-3 .. 1.

Per pair the file stores K_q and log K_q (§II-C Eqs. 7-10) at both repetition counts, in
FP64 from the oracle's TEBD MPS and transfer contraction (no truncation: the cutoff 1e-14
drops nothing but numerical zeros, and the exact bond never exceeds 32 here). The header
holds the SHA-256 of the float32 input bytes so that a run on another machine can tell
whether its generated inputs are the same. Re-run only when the oracle's arithmetic changes
for a reason that the commit message cites. Takes a few minutes on 8 cores.
"""
import hashlib
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.dirname(HERE))

from paper_2602_01330_gb300 import synthetic  # noqa: E402

M, D = 4000, 256
N_UNIFORM, N_NEAREST, N_DIAG, N_NEAR = 1000, 500, 500, 200
NEAR_SIGMA = (1e-4, 2.5e-2)
NEAR_SEED = 65
OUT = os.path.join(HERE, "cfg3_sampled_pairs.txt")


def inputs():
    x = synthetic.fmnist_like(M, 0, D)["x_train"]
    return x


def input_sha256(x, xn):
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(x, dtype=np.float32).tobytes())
    h.update(np.ascontiguousarray(xn, dtype=np.float32).tobytes())
    return h.hexdigest()


def sample_pairs(x):
    rng = np.random.Generator(np.random.PCG64(0))
    groups = []
    while len(groups) < N_UNIFORM:
        i, j = sorted(int(v) for v in rng.integers(0, M, size=2))
        if i < j:
            groups.append(("uniform", i, j))
    xd = x.astype(np.float64)
    sq = (xd * xd).sum(1)
    for i in rng.choice(M, size=N_NEAREST, replace=False):
        d2 = sq + sq[i] - 2.0 * (xd @ xd[i])
        d2[i] = np.inf
        j = int(np.argmin(d2))
        groups.append(("nearest", min(int(i), j), max(int(i), j)))
    for i in rng.choice(M, size=N_DIAG, replace=False):
        groups.append(("diagonal", int(i), int(i)))
    base = rng.choice(M, size=N_NEAR, replace=False)
    for k, b in enumerate(base):
        groups.append(("near_copy", int(b), k))  # column k indexes the perturbed copies
    return groups, base


def main():
    import oracle_pool
    x = inputs()
    groups, base = sample_pairs(x)
    xn = synthetic.near_copies(x[base], NEAR_SIGMA[0], NEAR_SIGMA[1], seed=NEAR_SEED)
    xa = np.stack([x[i] for _, i, _ in groups])
    xb = np.stack([xn[j] if g == "near_copy" else x[j] for g, _, j in groups])
    cols = {}
    for reps in (3, 5):
        kq, lkq = oracle_pool.aligned_pairs(xa, xb, reps)
        cols[reps] = (kq, lkq)
        print(f"reps {reps}: done", flush=True)
    header = "\n".join([
        "FP64 oracle K_q and log K_q (paper §II-C Eqs. 7-10) of the precision-form sampled pairs;",
        f"inputs: synthetic.fmnist_like({M}, 0, {D})['x_train'] (float32), near copies: "
        f"synthetic.near_copies(x[base], {NEAR_SIGMA[0]}, {NEAR_SIGMA[1]}, seed={NEAR_SEED});",
        f"input_sha256 {input_sha256(x, xn)}",
        "ZZ-chain map, reps 3 (bond 8) and reps 5 (bond 32), oracle TEBD MPS + transfer contraction;",
        "written by tests/golden/make_cfg3_golden.py; near_copy rows: column j indexes the copies.",
        "group i j kq_r3 logkq_r3 kq_r5 logkq_r5",
    ])
    with open(OUT, "w") as f:
        for line in header.split("\n"):
            f.write("# " + line + "\n")
        for p, (g, i, j) in enumerate(groups):
            f.write(f"{g} {i} {j} {cols[3][0][p]:.17e} {cols[3][1][p]:.17e} "
                    f"{cols[5][0][p]:.17e} {cols[5][1][p]:.17e}\n")


def load(path: str = OUT):
    """(rows as dicts, input sha256) from the stored file."""
    rows, sha = [], None
    with open(path) as f:
        for line in f:
            if line.startswith("# input_sha256"):
                sha = line.split()[2]
            if line.startswith("#"):
                continue
            g, i, j, a, b, c, d = line.split()
            rows.append({"group": g, "i": int(i), "j": int(j), "kq_r3": float(a), "logkq_r3": float(b),
                         "kq_r5": float(c), "logkq_r5": float(d)})
    return rows, sha


if __name__ == "__main__":
    main()
