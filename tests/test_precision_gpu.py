"""Precision form on the GPU: FP32 (bond 8 and 32) and split-BF16 tensor cores (bond 32)
against the FP64 oracle on sampled pairs of the d = 256 Fashion-MNIST-shaped data.

Tolerances: 1e-6 for the FP32 paths, 1e-4 for bf16x3 (the stated mixed-precision bound).
The measured numbers are printed as one JSON line (run pytest with -s to see it)."""
import json

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_precision_paths_vs_oracle_on_sampled_pairs():
    from oracle import gram, mps
    from paper_2602_01330_gb300 import build, precision
    build.build()
    res, pairs, blocks, x = precision.compare(m=256, pool=96, n_uniform=24, n_near=16, n_diag=6, return_blocks=True)
    idx = sorted({i for p in pairs for i in p})
    pos = {v: k for k, v in enumerate(idx)}
    report = {}
    for reps, chi, names in ((3, 8, ("fp32",)), (5, 32, ("fp32", "bf16x3"))):
        sites, _ = mps.build_mps(x[idx].astype(np.float64), reps)
        ref, _ = gram.pair_values(sites, sites, [pos[i] for i, _ in pairs], [pos[j] for _, j in pairs])
        for name in names:
            got = np.array([blocks[(chi, name)][i, j] for i, j in pairs])
            err = float(np.max(np.abs(got - ref)))
            report[f"chi{chi}_{name}"] = {"max_abs_dK": err, "gram_entry_qubits_per_s":
                                          res[f"chi{chi}_{name}"]["entry_qubits_per_s"]}
            assert err <= (1e-4 if name == "bf16x3" else 1e-6), (chi, name, err)
        report[f"chi{chi}_largest_offdiag_K"] = float(ref[:-6].max())
    report["bf16x3_vs_fp32_block"] = res["chi32_max_abs_dK_bf16x3_vs_fp32_block"]
    print(json.dumps(report))
