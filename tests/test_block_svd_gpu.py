"""GPU parity of dk_mps_build_blocks: block-structured maps built from block statevectors by
truncating SVD sweeps (§II-C; the SVD cutoff reading: drop s < cutoff s_0, cap the bond,
renormalise, report the discarded weight), then contracted by the existing Gram kernels.

References, all from ``oracle/``: the per-block statevector overlaps (exact, any n) for
untruncated builds, and ``oracle.blocks.mps_from_block_states`` (numpy SVD, same cutoff and
cap) for truncated ones. Tolerances: |dK| <= 1e-6 on K_q for the FP32 Gram, 1e-4 for
bf16x3; discarded weights within 1e-6 relative (FP64 sweeps, float32 output); bond
dimensions exact."""
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


def _block_log_overlaps(x, reps, b, entangler):
    from oracle import blocks, circuit
    out = np.zeros((x.shape[0], x.shape[0]))
    for s, e in blocks.block_ranges(x.shape[1], b):
        st = np.stack([circuit.statevector(r[s:e].astype(np.float64), reps, entangler=entangler,
                                           block=0) for r in x])
        with np.errstate(divide="ignore"):
            out += np.log(np.abs(st.conj() @ st.T) ** 2)
    return out


@pytest.mark.parametrize("n,b,reps,chi", [(40, 8, 2, 32), (25, 9, 2, 32), (25, 8, 1, 32), (30, 4, 3, 8)])
def test_full_entangler_untruncated_vs_block_statevectors(dk, n, b, reps, chi):
    """All-to-all ZZ inside blocks with a cap at the exact bond (16 at the centre of a block
    of 8 or 9, 4 for a block of 4): nothing is truncated, and the bonds are beyond the
    2^reps of the chain; n = 25 leaves a short last block."""
    dualk, ctx, torch = dk
    from oracle import blocks, mps as omps
    from paper_2602_01330_gb300 import synthetic
    x = synthetic.fmnist_like(30, 0, n)["x_train"]
    ref_sites, disc_ref = blocks.mps_from_block_states(x.astype(np.float64), reps, b, "full", chi_cap=chi // 2)
    assert disc_ref.max() <= 1e-20
    m, disc = dualk.mps_build_blocks(ctx, _dev(torch, x), dualk.FeatureMap(reps=reps, chi_max=chi, block=b),
                                     dualk.DK_ENT_FULL)
    ref = np.exp(_block_log_overlaps(x, reps, b, "full"))
    precs = [(dualk.DK_PREC_F32, 1e-6)] + ([(dualk.DK_PREC_BF16X3, 1e-4)] if chi == 32 else [])
    for prec, tol in precs:
        g = dualk.gram(ctx, m, w=1.0, want=("kq",), prec=prec)
        torch.cuda.synchronize()
        kq = g["kq"].cpu().numpy().astype(np.float64)
        assert np.max(np.abs(kq - ref)) <= tol, (prec, float(np.max(np.abs(kq - ref))))
        assert np.all(np.diag(kq) == 1.0)
    assert np.all(disc.cpu().numpy() <= 1e-12)
    assert m.bond_dims.cpu().tolist() == omps.bond_dims(ref_sites)
    ctx.sync_status()


@pytest.mark.parametrize("b,reps", [(10, 2), (12, 2)])
def test_full_entangler_truncated_vs_oracle(dk, b, reps):
    """Blocks of 10 and 12 with all-to-all ZZ: exact bonds 32 and 64 at the block centre, cap
    16 (chi_max 32). The discarded weight, the kept bond dimensions and K_q (FP32 Gram) match
    the oracle's truncated MPS; K_q(x, x) stays exactly 1."""
    dualk, ctx, torch = dk
    from oracle import blocks, gram as og, mps as omps
    from paper_2602_01330_gb300 import synthetic
    n = 3 * b
    x = synthetic.uniform_angles(24, n, b).astype(np.float32).astype(np.float64)  # the GPU's inputs
    sites, disc_ref = blocks.mps_from_block_states(x, reps, b, "full", chi_cap=16)
    assert disc_ref.min() > 1e-3  # the cap really truncates every sample
    kq_ref, _ = og.gram_from_mps(sites, sites)
    m, disc = dualk.mps_build_blocks(ctx, _dev(torch, x), dualk.FeatureMap(reps=reps, chi_max=32, block=b),
                                     dualk.DK_ENT_FULL)
    g = dualk.gram(ctx, m, w=1.0, want=("kq",))
    torch.cuda.synchronize()
    d = disc.cpu().numpy().astype(np.float64)
    np.testing.assert_allclose(d, disc_ref, rtol=1e-6, atol=1e-12)
    assert m.bond_dims.cpu().tolist() == omps.bond_dims(sites)
    kq = g["kq"].cpu().numpy().astype(np.float64)
    assert np.max(np.abs(kq - kq_ref)) <= 1e-6
    assert np.all(np.diag(kq) == 1.0)
    ctx.sync_status()


def test_chain_blocks_agree_with_closed_form_build(dk):
    """The chain entangler through block statevectors + SVD (bond cap 4 at chi_max 8) and the
    closed-form build with the same blocks (dk_mps_build, chi_max 4) are two independent GPU
    constructions of one state: K_q agrees to 1e-6, and the kept bonds are the exact ranks
    min(2^k, 2^(b-k), 2^reps) inside each block."""
    dualk, ctx, torch = dk
    from paper_2602_01330_gb300 import synthetic
    n, b = 50, 7
    x = _dev(torch, synthetic.fmnist_like(40, 0, n)["x_train"])
    a, disc = dualk.mps_build_blocks(ctx, x, dualk.FeatureMap(reps=2, chi_max=8, block=b), dualk.DK_ENT_CHAIN)
    c = dualk.mps_build(ctx, x, dualk.FeatureMap(reps=2, chi_max=4, block=b))
    ka = dualk.gram(ctx, a, w=0.5)
    kc = dualk.gram(ctx, c, w=0.5)
    torch.cuda.synchronize()
    assert torch.max(torch.abs(ka["kq"] - kc["kq"])).item() <= 1e-6
    assert torch.max(torch.abs(ka["k"] - kc["k"])).item() <= 1e-6
    assert torch.equal(ka["kc"], kc["kc"])
    dims = a.bond_dims.cpu().tolist()
    for k in range(n + 1):
        s = (k // b) * b
        e = min(s + b, n)
        ref = 1 if k == s or k == n else min(2 ** (k - s), 2 ** (e - k), 4)
        assert dims[k] == ref, (k, dims[k], ref)
    assert np.all(disc.cpu().numpy() <= 1e-12)
    ctx.sync_status()


def test_complex128_product_and_errors(dk):
    """complex128 output at chi_max 4 (one repetition, chain: exact bond 2) against the
    per-block reference; entanglers off gives the product kernel; bad arguments are refused."""
    dualk, ctx, torch = dk
    from paper_2602_01330_gb300 import synthetic
    x = synthetic.uniform_angles(20, 23, 9).astype(np.float32).astype(np.float64)
    m, _ = dualk.mps_build_blocks(ctx, _dev(torch, x), dualk.FeatureMap(reps=1, chi_max=4, block=5),
                                  dualk.DK_ENT_CHAIN, dtype=dualk.DK_C128)
    g = dualk.gram(ctx, m, w=1.0, want=("kq",))
    p, _ = dualk.mps_build_blocks(ctx, _dev(torch, x), dualk.FeatureMap(reps=1, chi_max=4, block=5, entangle=False),
                                  dualk.DK_ENT_FULL)
    gp = dualk.gram(ctx, p, w=1.0, want=("kq",))
    torch.cuda.synchronize()
    ref = np.exp(_block_log_overlaps(x, 1, 5, "chain"))
    assert np.max(np.abs(g["kq"].cpu().numpy() - ref)) <= 1e-6
    prod = np.prod(np.cos(x[:, None, :] - x[None, :, :]) ** 2, axis=2)  # one repetition, no entanglers
    assert np.max(np.abs(gp["kq"].cpu().numpy() - prod)) <= 1e-6
    xt = _dev(torch, x)
    for fm, ent, cut in ((dualk.FeatureMap(reps=1, chi_max=4, block=13), dualk.DK_ENT_FULL, 1e-10),
                         (dualk.FeatureMap(reps=1, chi_max=4, block=5), 2, 1e-10),
                         (dualk.FeatureMap(reps=1, chi_max=4, block=5), dualk.DK_ENT_FULL, 1.5),
                         (dualk.FeatureMap(reps=1, chi_max=6, block=5), dualk.DK_ENT_FULL, 1e-10)):
        with pytest.raises(dualk.DualKError):
            dualk.mps_build_blocks(ctx, xt, fm, ent, cut)
    ctx.sync_status()
