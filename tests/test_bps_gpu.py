"""GPU parity of the block-structured (block product state) feature map, §II-C: entanglers
only inside blocks of b consecutive qubits, so the state is a product of the blocks' own
chain states and log K_q a sum of per-block terms.

The reference is the oracle's statevector of each block (at most 12 qubits), which makes
this parity exact at any n, including n = 784 at two repetitions, where the plain chain
has no closed form. Tolerances as for the chain: |dK| <= 1e-6 on K_q for the FP32 and
complex128 paths, 1e-4 for bf16x3; log K_q within 1e-3 * max(1, |log K_q|) wherever the
reference log K_q > -700, and within 1e-4 relative at n = 784 where every value is far below
that (the FP32 chain's rounding grows about linearly with n, not with |log K_q|)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dk():
    import torch
    from paper_2602_01330_gb300 import build, dualk
    build.build()
    ctx = dualk.Context(0)
    yield dualk, ctx, torch
    ctx.close()


def _dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _block_reference(x_rows, x_cols, reps, b):
    """log K_q[i, j] = sum over blocks of log |<psi_B(x_i)|psi_B(x_j)>|^2, block states by
    the oracle's dense statevector of the block's chain."""
    from oracle import circuit
    n = x_rows.shape[1]
    out = np.zeros((x_rows.shape[0], x_cols.shape[0]))
    for s in range(0, n, b):
        e = min(s + b, n)
        a = np.stack([circuit.statevector(r[s:e].astype(np.float64), reps) for r in x_rows])
        c = np.stack([circuit.statevector(r[s:e].astype(np.float64), reps) for r in x_cols])
        with np.errstate(divide="ignore"):
            out += np.log(np.abs(a.conj() @ c.T) ** 2)
    return out


@pytest.mark.parametrize("n,b,dtype", [(64, 8, "c64"), (64, 8, "c128"), (61, 7, "c64")])
def test_bps_chi4_vs_block_statevectors(dk, n, b, dtype):
    """Bond 4 (reps = 2): a symmetric Gram of 70 samples (ragged tiles) and 20 x 70 rows,
    element by element; n = 61 with b = 7 leaves a short last block."""
    dualk, ctx, torch = dk
    from paper_2602_01330_gb300 import synthetic
    d = synthetic.fmnist_like(70, 20, n) if n == 64 else {"x_train": synthetic.uniform_angles(70, n, 7),
                                                          "x_test": synthetic.uniform_angles(20, n, 8)}
    xtr, xte = d["x_train"], d["x_test"]
    fm = dualk.FeatureMap(reps=2, chi_max=4, block=b)
    dt = dualk.DK_C128 if dtype == "c128" else dualk.DK_C64
    mtr = dualk.mps_build(ctx, _dev(torch, xtr), fm, dtype=dt)
    mte = dualk.mps_build(ctx, _dev(torch, xte), fm, dtype=dt)
    g = dualk.gram(ctx, mtr, w=1.0, want=("kq", "logkq"))
    r = dualk.dual_kernel_rows(ctx, mte, mtr, w=1.0, want=("kq", "logkq"))
    torch.cuda.synchronize()
    for out, xa in ((g, xtr), (r, xte)):
        ref = _block_reference(xa, xtr, 2, b)
        kq = out["kq"].cpu().numpy().astype(np.float64)
        lkq = out["logkq"].cpu().numpy().astype(np.float64)
        assert np.max(np.abs(kq - np.exp(ref))) <= 1e-6
        sel = ref > -700
        assert np.all(np.abs(lkq[sel] - ref[sel]) <= 1e-3 * np.maximum(1.0, np.abs(ref[sel])))
    assert np.all(np.diag(g["kq"].cpu().numpy()) == 1.0)
    ctx.sync_status()


def test_bps_chi4_n784_log_kernel(dk):
    """n = 784 (all pixels), reps = 2, blocks of 8: 48 synthetic images, every pair's log K_q
    against the sum of 98 block terms."""
    dualk, ctx, torch = dk
    from paper_2602_01330_gb300 import synthetic
    x = synthetic.fmnist_like(48, 0, 784)["x_train"]
    fm = dualk.FeatureMap(reps=2, chi_max=4, block=8)
    m = dualk.mps_build(ctx, _dev(torch, x), fm)
    g = dualk.gram(ctx, m, w=1.0, want=("kq", "logkq"))
    torch.cuda.synchronize()
    ref = _block_reference(x, x, 2, 8)
    lkq = g["logkq"].cpu().numpy().astype(np.float64)
    off = ~np.eye(48, dtype=bool)
    assert np.all(ref[off] < -100)  # the concentrated regime: only the log is informative
    assert np.max(np.abs(lkq[off] - ref[off]) / np.abs(ref[off])) <= 1e-4
    assert np.all(np.diag(g["kq"].cpu().numpy()) == 1.0)
    ctx.sync_status()


@pytest.mark.parametrize("reps,chi,b,n", [(3, 8, 6, 40), (5, 32, 12, 36)])
def test_bps_wide_bonds_vs_block_statevectors(dk, reps, chi, b, n):
    """Bond 8 (reps = 3, blocks of 6: inside a block the rank reaches 8) and bond 32
    (reps = 5, blocks of 12: rank 32 at the block centre), FP32; bond 32 also bf16x3."""
    dualk, ctx, torch = dk
    from paper_2602_01330_gb300 import synthetic
    x = synthetic.fmnist_like(40, 0, n)["x_train"]
    m = dualk.mps_build(ctx, _dev(torch, x), dualk.FeatureMap(reps=reps, chi_max=chi, block=b))
    ref = np.exp(_block_reference(x, x, reps, b))
    precs = [(dualk.DK_PREC_F32, 1e-6)] + ([(dualk.DK_PREC_BF16X3, 1e-4)] if chi == 32 else [])
    for prec, tol in precs:
        g = dualk.gram(ctx, m, w=1.0, want=("kq",), prec=prec)
        torch.cuda.synchronize()
        kq = g["kq"].cpu().numpy().astype(np.float64)
        assert np.max(np.abs(kq - ref)) <= tol, (prec, np.max(np.abs(kq - ref)))
    ctx.sync_status()


def test_block_limits_bit_identical(dk):
    """block >= n is the chain and block = 1 has no entanglers: the same closed form with the
    same phases, so the results are bit-identical to those maps."""
    dualk, ctx, torch = dk
    from paper_2602_01330_gb300 import synthetic
    x = _dev(torch, synthetic.fmnist_like(33, 0, 20)["x_train"])
    pairs = (
        (dualk.FeatureMap(reps=2, chi_max=4, block=20), dualk.FeatureMap(reps=2, chi_max=4)),
        (dualk.FeatureMap(reps=2, chi_max=4, block=1), dualk.FeatureMap(reps=2, chi_max=4, entangle=False)),
        (dualk.FeatureMap(reps=3, chi_max=8, block=50), dualk.FeatureMap(reps=3, chi_max=8)),
    )
    for a, b in pairs:
        ga = dualk.gram(ctx, dualk.mps_build(ctx, x, a), w=0.5)
        gb = dualk.gram(ctx, dualk.mps_build(ctx, x, b), w=0.5)
        torch.cuda.synchronize()
        for key in ("k", "kq", "kc", "logkq"):
            assert torch.equal(ga[key], gb[key]), key
    with pytest.raises(dualk.DualKError):
        dualk.mps_build(ctx, x, dualk.FeatureMap(reps=2, chi_max=4, block=-1))
    ctx.sync_status()
