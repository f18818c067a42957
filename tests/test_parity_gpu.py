"""GPU parity: every C-ABI entry point against the FP64 oracle on the same seeded inputs.

Tolerance (written here, used below): |dK| <= 1e-6 for K, K_q and K_c on the FP32
path (complex64 MPS, FP32 transfer arithmetic, float32 outputs); log K_q within
1e-3 * max(1, |log K_q|) wherever the oracle's log K_q > -700. The complex128 path
also writes float32 outputs, so it is held to the same 1e-6.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL_K = 1e-6


def _tol_log(ref):
    return 1e-3 * np.maximum(1.0, np.abs(ref))


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


def _oracle_block(x_rows, x_cols, reps, entangle=True, angle_scale=2.0):
    from oracle import gram, mps
    r, _ = mps.build_mps(x_rows.astype(np.float64), reps, angle_scale, entangle)
    c, _ = mps.build_mps(x_cols.astype(np.float64), reps, angle_scale, entangle)
    return gram.gram_from_mps(r, c)


def _check_block(out, kq_ref, lkq_ref, kc_ref, w):
    kq = out["kq"].cpu().numpy().astype(np.float64)
    kc = out["kc"].cpu().numpy().astype(np.float64)
    k = out["k"].cpu().numpy().astype(np.float64)
    lkq = out["logkq"].cpu().numpy().astype(np.float64)
    assert np.max(np.abs(kq - kq_ref)) <= TOL_K
    assert np.max(np.abs(kc - kc_ref)) <= TOL_K
    assert np.max(np.abs(k - (w * kq_ref + (1 - w) * kc_ref))) <= TOL_K
    sel = lkq_ref > -700
    assert np.all(np.abs(lkq[sel] - lkq_ref[sel]) <= _tol_log(lkq_ref[sel]))


def test_tiny_case_complex128_vs_statevector(dk):
    """n = 8, 64 samples uniform in [0, pi] (seed 0), reps = 1, complex128, exact bond 2:
    the full 64 x 64 K_q against brute-force 256-amplitude statevectors."""
    dualk, ctx, torch = dk
    from oracle import circuit
    from paper_2602_01330_gb300 import synthetic
    x = synthetic.uniform_angles(64, 8, seed=0)
    ref = circuit.kernel_matrix(x, x, 1)
    m = dualk.mps_build(ctx, _dev(torch, x), dualk.FeatureMap(reps=1, chi_max=4), dtype=dualk.DK_C128)
    out = dualk.gram(ctx, m, w=1.0)
    torch.cuda.synchronize()
    kq = out["kq"].cpu().numpy()
    assert np.max(np.abs(kq - ref)) <= TOL_K
    assert np.array_equal(kq, kq.T)
    assert np.all(np.diag(kq) == 1.0)
    stored = np.loadtxt(__import__("os").path.join(__import__("os").path.dirname(__file__), "golden", "cfg1_kq16.txt"))
    assert np.max(np.abs(kq[:16, :16] - stored)) <= TOL_K
    assert m.bond_dims.cpu().tolist() == [1, 2, 2, 2, 2, 2, 2, 2, 1]
    ctx.sync_status()


@pytest.mark.parametrize("reps,chi,dtype", [(1, 4, "c64"), (2, 4, "c64"), (1, 4, "c128"), (2, 4, "c128")])
def test_small_n_vs_statevector(dk, reps, chi, dtype):
    dualk, ctx, torch = dk
    from oracle import circuit
    from paper_2602_01330_gb300 import synthetic
    x = synthetic.uniform_angles(37, 10, seed=5)
    ref = circuit.kernel_matrix(x, x, reps)
    dt = dualk.DK_C64 if dtype == "c64" else dualk.DK_C128
    m = dualk.mps_build(ctx, _dev(torch, x), dualk.FeatureMap(reps=reps, chi_max=chi), dtype=dt)
    out = dualk.gram(ctx, m, w=1.0)
    torch.cuda.synchronize()
    assert np.max(np.abs(out["kq"].cpu().numpy() - ref)) <= TOL_K


def test_fmnist_d64_reps2_all_mixes(dk):
    """d = 64 Fashion-MNIST-shaped features, reps = 2 (chi = 4), complex64: Gram of 200
    train samples (12 full 16-tiles + a ragged one) and 50 x 200 dual-kernel rows, at
    w in {0, 0.25, 0.5, 0.75, 1}, element by element against the oracle."""
    dualk, ctx, torch = dk
    from oracle import gram as og
    from paper_2602_01330_gb300 import synthetic
    d = synthetic.fmnist_like(200, 50, 64)
    xtr, xte = d["x_train"], d["x_test"]
    kq_tr, lkq_tr = _oracle_block(xtr, xtr, 2)
    kq_te, lkq_te = _oracle_block(xte, xtr, 2)
    kc_tr = og.rbf(xtr, xtr, 1 / 64)
    kc_te = og.rbf(xte, xtr, 1 / 64)
    fm = dualk.FeatureMap(reps=2, chi_max=4)
    mtr = dualk.mps_build(ctx, _dev(torch, xtr), fm)
    mte = dualk.mps_build(ctx, _dev(torch, xte), fm)
    for w in (0.0, 0.25, 0.5, 0.75, 1.0):
        out = dualk.gram(ctx, mtr, w=w)
        rows = dualk.dual_kernel_rows(ctx, mte, mtr, w=w)
        torch.cuda.synchronize()
        _check_block(out, kq_tr, lkq_tr, kc_tr, w)
        _check_block(rows, kq_te, lkq_te, kc_te, w)
    ctx.sync_status()


def test_gram_invariants_and_determinism(dk):
    dualk, ctx, torch = dk
    from paper_2602_01330_gb300 import synthetic
    x = synthetic.fmnist_like(150, 0, 64)["x_train"]
    m = dualk.mps_build(ctx, _dev(torch, x), dualk.FeatureMap(reps=2, chi_max=4))
    out = dualk.gram(ctx, m, w=1.0)
    rows = dualk.dual_kernel_rows(ctx, m, m, w=1.0)
    blk = dualk.gram_tile(ctx, m, m, row0=17, nrows=60, col0=40, ncols=77, w=1.0)
    torch.cuda.synchronize()
    kq = out["kq"].cpu().numpy()
    assert np.array_equal(kq, kq.T)
    assert np.all(np.diag(kq) == 1.0)
    assert kq.min() >= 0.0 and kq.max() <= 1.0 + 1e-6
    lam = np.linalg.eigvalsh(kq.astype(np.float64))
    assert lam.min() >= -150 * 1e-6
    # the same pair gives the same bits whatever tile or call computes it
    r = rows["kq"].cpu().numpy()
    iu = np.triu_indices(150)
    assert np.array_equal(r[iu], kq[iu])
    b = blk["kq"].cpu().numpy()
    sub = kq[17:77, 40:117]
    ii, jj = np.meshgrid(np.arange(17, 77), np.arange(40, 117), indexing="ij")
    upper = ii <= jj
    assert np.array_equal(b[upper], sub[upper])


def test_edge_cases(dk):
    dualk, ctx, torch = dk
    from oracle import circuit, gram as og
    from paper_2602_01330_gb300 import synthetic
    fm = dualk.FeatureMap(reps=2, chi_max=4)
    # n = 1 and n = 2 qubits, m = 1 sample, odd sizes
    for n, msz in ((1, 5), (2, 3), (3, 1), (5, 19)):
        x = synthetic.uniform_angles(msz, n, seed=n)
        ref = circuit.kernel_matrix(x, x, 2)
        m = dualk.mps_build(ctx, _dev(torch, x), fm)
        out = dualk.gram(ctx, m, w=0.5)
        torch.cuda.synchronize()
        assert np.max(np.abs(out["kq"].cpu().numpy() - ref)) <= TOL_K
        kc = og.rbf(x, x, 1.0 / n)
        assert np.max(np.abs(out["kc"].cpu().numpy() - kc)) <= TOL_K
    # entanglers off: product closed form
    x = synthetic.uniform_angles(20, 30, seed=9)
    m = dualk.mps_build(ctx, _dev(torch, x), dualk.FeatureMap(reps=1, entangle=False, chi_max=4))
    out = dualk.gram(ctx, m, w=1.0, want=("kq",))
    torch.cuda.synchronize()
    xx = x.astype(np.float32).astype(np.float64)
    ref = np.prod(np.cos(xx[:, None, :] - xx[None, :, :]) ** 2, axis=2)
    assert np.max(np.abs(out["kq"].cpu().numpy() - ref)) <= TOL_K
    # only one output requested, ld larger than the block, into a bigger buffer
    x = synthetic.uniform_angles(40, 12, seed=10)
    m = dualk.mps_build(ctx, _dev(torch, x), fm)
    big = torch.full((50, 64), -7.0, device="cuda")
    dualk.gram_tile(ctx, m, m, row0=3, nrows=20, col0=5, ncols=30, w=1.0, out={"kq": big}, ld=64)
    full = dualk.gram(ctx, m, w=1.0, want=("kq",))
    torch.cuda.synchronize()
    bb = big.cpu().numpy()
    assert np.all(bb[20:, :] == -7.0) and np.all(bb[:, 30:] == -7.0)
    ref = full["kq"].cpu().numpy()[3:23, 5:35]
    gi, gj = np.meshgrid(np.arange(3, 23), np.arange(5, 35), indexing="ij")
    # pairs with i <= j are contracted with the same operand roles as in the symmetric
    # call, so they agree bit for bit; the others agree to rounding
    np.testing.assert_array_equal(bb[:20, :30][gi <= gj], ref[gi <= gj])
    assert np.max(np.abs(bb[:20, :30] - ref)) <= TOL_K


def test_host_errors(dk):
    dualk, ctx, torch = dk
    x = torch.rand(4, 6, device="cuda") * 3
    with pytest.raises(dualk.DualKError) as e:
        dualk.mps_build(ctx, x, dualk.FeatureMap(reps=3, chi_max=4))  # needs chi >= 8
    assert e.value.status == 2
    with pytest.raises(dualk.DualKError) as e:
        dualk.mps_build(ctx, x, dualk.FeatureMap(reps=0, chi_max=4))
    assert e.value.status == 1
    with pytest.raises(dualk.DualKError) as e:
        dualk.mps_build(ctx, x, dualk.FeatureMap(reps=2, chi_max=4, qr_prec=2))  # neither F32 nor F64
    assert e.value.status == 1
    m = dualk.mps_build(ctx, x, dualk.FeatureMap(reps=2, chi_max=4))
    with pytest.raises(dualk.DualKError) as e:
        dualk.gram_tile(ctx, m, m, row0=2, nrows=3)  # runs past the 4 samples
    assert e.value.status == 1
    ctx.sync_status()


def test_n784_bench_shape_sampled(dk):
    """The benchmarked workload: d = 784 raw pixels, 2000 train + 500 test, reps = 2,
    chi = 4, in the bench launch configuration; 64 train samples (Gram block) and 16
    test samples (rows) are checked element by element against the oracle."""
    dualk, ctx, torch = dk
    from oracle import gram as og
    from paper_2602_01330_gb300 import synthetic
    d = synthetic.fmnist_like(2000, 500, 784)
    xtr, xte = d["x_train"], d["x_test"]
    fm = dualk.FeatureMap(reps=2, chi_max=4)
    mtr = dualk.mps_build(ctx, _dev(torch, xtr), fm)
    mte = dualk.mps_build(ctx, _dev(torch, xte), fm)
    out = dualk.gram(ctx, mtr, w=0.5)
    rows = dualk.dual_kernel_rows(ctx, mte, mtr, w=0.5)
    torch.cuda.synchronize()
    rng = np.random.Generator(np.random.PCG64(7))
    si = np.sort(rng.choice(2000, 64, replace=False))
    ti = np.sort(rng.choice(500, 16, replace=False))
    kq_ref, lkq_ref = _oracle_block(xtr[si], xtr[si], 2)
    kc_ref = og.rbf(xtr[si], xtr[si], 1 / 784)
    sub = {k: v[si][:, si] for k, v in out.items()}
    _check_block(sub, kq_ref, lkq_ref, kc_ref, 0.5)
    kq_ref, lkq_ref = _oracle_block(xte[ti], xtr[si], 2)
    kc_ref = og.rbf(xte[ti], xtr[si], 1 / 784)
    sub = {k: v[ti][:, si] for k, v in rows.items()}
    _check_block(sub, kq_ref, lkq_ref, kc_ref, 0.5)
    kq = out["kq"]
    assert bool(torch.all(torch.diagonal(kq) == 1.0))
    assert bool(torch.equal(kq, kq.T))
    ctx.sync_status()


@pytest.mark.parametrize("dtype,qr", [("c64", "f32"), ("c64", "f64"), ("c128", "f64")])
def test_bond4_build_kernels_agree_small_and_large_sets(dk, dtype, qr):
    """The bond-4 MPS build runs its QR in FP32 (complex64, the default) or FP64 (complex64
    on request, complex128 always). The FP64 form has two launches chosen by the sample
    count: 8 threads per sample up to 40 samples per SM, 2 threads per sample above; the
    FP32 form uses 8 threads at every size. 6400 samples, d = 40, reps = 2: the Gram block
    between the first 48 and the last 48 samples against the oracle, the same 96 samples
    built as a small set giving the same block, and for both sets the fused ln-norms close
    to the self-overlap entry point's and a unit Gram diagonal (exact in FP32)."""
    dualk, ctx, torch = dk
    from oracle import gram as og
    from paper_2602_01330_gb300 import synthetic
    dt = dualk.DK_C64 if dtype == "c64" else dualk.DK_C128
    m, n = 6400, 40
    x = synthetic.fmnist_like(m, 0, n)["x_train"]
    fm = dualk.FeatureMap(reps=2, chi_max=4, qr_prec=dualk.DK_PREC_F32 if qr == "f32" else dualk.DK_PREC_F64)
    big = dualk.mps_build(ctx, _dev(torch, x), fm, dtype=dt)
    out = dualk.gram_tile(ctx, big, big, 0, 48, m - 48, 48, w=0.5)
    sel = np.r_[0:48, m - 48:m]
    small = dualk.mps_build(ctx, _dev(torch, x[sel]), fm, dtype=dt)
    out_s = dualk.gram_tile(ctx, small, small, 0, 48, 48, 48, w=0.5)
    torch.cuda.synchronize()
    kq_ref, lkq_ref = _oracle_block(x[:48], x[m - 48:], 2)
    kc_ref = og.rbf(x[:48], x[m - 48:], 1 / n)
    _check_block(out, kq_ref, lkq_ref, kc_ref, 0.5)
    _check_block(out_s, kq_ref, lkq_ref, kc_ref, 0.5)
    prec = dualk.DK_PREC_F32 if dtype == "c64" else dualk.DK_PREC_F64
    for mp in (big, small):
        fused = mp.log_norm.clone()
        sep = dualk.self_overlap(ctx, mp, prec)
        diag = dualk.gram_tile(ctx, mp, mp, 0, 48, 0, 48, w=1.0, want=("kq",))["kq"]
        torch.cuda.synchronize()
        assert torch.max(torch.abs(fused - sep)).item() <= 1e-5
        if dtype == "c64":
            assert bool(torch.all(torch.diagonal(diag) == 1.0))
        else:
            assert torch.max(torch.abs(torch.diagonal(diag) - 1.0)).item() <= TOL_K
    ctx.sync_status()


@pytest.mark.parametrize("d", [8, 16])
def test_bond4_fp32_build_relative_accuracy(dk, d):
    """The complex64 build factorises in FP32. On 96 uniform-angle samples (seed 5),
    reps = 2, where many K_q are O(1): |dK| <= 1e-6 everywhere and the relative error of
    every K_q > 1e-3 within 2e-5 of the oracle (an FP64 factorisation rounded to complex64
    storage reaches about 2e-6 here; the FP32 one about 4e-6)."""
    dualk, ctx, torch = dk
    from paper_2602_01330_gb300 import synthetic
    x = synthetic.uniform_angles(96, d, seed=5).astype(np.float32)
    m = dualk.mps_build(ctx, _dev(torch, x), dualk.FeatureMap(reps=2, chi_max=4))
    kq = dualk.gram(ctx, m, w=1.0, want=("kq",))["kq"].cpu().numpy().astype(np.float64)
    kq_ref, _ = _oracle_block(x, x, 2)
    assert np.max(np.abs(kq - kq_ref)) <= TOL_K
    big = kq_ref > 1e-3
    assert big.sum() > 96
    assert np.max(np.abs(kq - kq_ref)[big] / kq_ref[big]) <= 2e-5
    ctx.sync_status()


@pytest.mark.parametrize("n,reps", [(8, 3), (11, 3)])
def test_chi8_fp32_vs_statevector(dk, n, reps):
    """reps = 3 keeps the exact bond 8: the chi = 8 FP32 kernels against brute force."""
    dualk, ctx, torch = dk
    from oracle import circuit
    from paper_2602_01330_gb300 import synthetic
    x = synthetic.uniform_angles(21, n, seed=n)
    ref = circuit.kernel_matrix(x, x, reps)
    m = dualk.mps_build(ctx, _dev(torch, x), dualk.FeatureMap(reps=reps, chi_max=8))
    out = dualk.gram(ctx, m, w=1.0)
    torch.cuda.synchronize()
    kq = out["kq"].cpu().numpy()
    assert np.max(np.abs(kq - ref)) <= TOL_K
    assert np.all(np.diag(kq) == 1.0)
    assert m.bond_dims.cpu().tolist()[:5] == [1, 2, 4, 8, 8][:5]


def test_chi8_fmnist_d256_sampled(dk):
    """reps = 3 at d = 256 (the precision-form data, exact bond 8): 40 train x 40 train and
    10 test rows against the oracle, element by element."""
    dualk, ctx, torch = dk
    from oracle import gram as og
    from paper_2602_01330_gb300 import synthetic
    d = synthetic.fmnist_like(40, 10, 256)
    xtr, xte = d["x_train"], d["x_test"]
    fm = dualk.FeatureMap(reps=3, chi_max=8)
    mtr = dualk.mps_build(ctx, _dev(torch, xtr), fm)
    mte = dualk.mps_build(ctx, _dev(torch, xte), fm)
    out = dualk.gram(ctx, mtr, w=0.5)
    rows = dualk.dual_kernel_rows(ctx, mte, mtr, w=0.5)
    torch.cuda.synchronize()
    kq, lkq = _oracle_block(xtr, xtr, 3)
    _check_block(out, kq, lkq, og.rbf(xtr, xtr, 1 / 256), 0.5)
    kq, lkq = _oracle_block(xte, xtr, 3)
    _check_block(rows, kq, lkq, og.rbf(xte, xtr, 1 / 256), 0.5)


def test_chi8_every_tile_shape_bit_identical(dk):
    """Every bond-8 tile shape (reps = 3, d = 40) gives bit-identical K_q, log K_q and K_c for
    a symmetric Gram with ragged tiles (150 samples) and a rectangular block: each pair is
    contracted by the same arithmetic whatever tile, stage depth or CTA count it lands in."""
    dualk, ctx, torch = dk
    from paper_2602_01330_gb300 import synthetic
    d = synthetic.fmnist_like(150, 37, 40)
    fm = dualk.FeatureMap(reps=3, chi_max=8)
    mtr = dualk.mps_build(ctx, _dev(torch, d["x_train"]), fm)
    mte = dualk.mps_build(ctx, _dev(torch, d["x_test"]), fm)
    ref = None
    try:
        for cid in range(1, dualk.gram_config_count(dualk.DK_C64, 8) + 1):
            ctx.set_gram_config(cid)
            g = dualk.gram(ctx, mtr, w=0.5)
            r = dualk.dual_kernel_rows(ctx, mte, mtr, w=0.5)
            got = [t.cpu() for t in (g["kq"], g["logkq"], g["kc"], r["kq"], r["logkq"])]
            if ref is None:
                ref = got
            else:
                for a, b in zip(ref, got):
                    assert torch.equal(a, b)
    finally:
        ctx.set_gram_config(0)
    assert dualk.gram_config_count(dualk.DK_C64, 8) >= 5
    ctx.sync_status()


def test_bounded_wait_reports_timeout_and_context_survives(dk):
    """A device wait that nothing satisfies gives up after its bound, the status word says
    DK_ERR_TIMEOUT, and the same context then runs a Gram normally."""
    dualk, ctx, torch = dk
    ctx.sync_status()
    ctx.selftest_wait_timeout(50_000_000)
    with pytest.raises(dualk.DualKError) as e:
        ctx.sync_status()
    assert e.value.status == 4
    ctx.sync_status()  # cleared
    x = torch.rand(9, 6, device="cuda") * 3
    m = dualk.mps_build(ctx, x, dualk.FeatureMap(reps=2, chi_max=4))
    out = dualk.gram(ctx, m, w=1.0, want=("kq",))
    torch.cuda.synchronize()
    assert bool(torch.all(torch.diagonal(out["kq"]) == 1.0))
    ctx.sync_status()


def test_chi32_fp32_vs_statevector(dk):
    """reps = 5 reaches bond 32 at n = 12: the bond-32 FP32 kernels against brute force."""
    dualk, ctx, torch = dk
    from oracle import circuit
    from paper_2602_01330_gb300 import synthetic
    x = synthetic.uniform_angles(11, 12, seed=12)
    ref = circuit.kernel_matrix(x, x, 5)
    m = dualk.mps_build(ctx, _dev(torch, x), dualk.FeatureMap(reps=5, chi_max=32))
    out = dualk.gram(ctx, m, w=1.0)
    torch.cuda.synchronize()
    kq = out["kq"].cpu().numpy()
    assert np.max(np.abs(kq - ref)) <= TOL_K
    assert np.all(np.diag(kq) == 1.0)
    assert np.array_equal(kq, kq.T)
    assert m.bond_dims.cpu().tolist() == [1, 2, 4, 8, 16, 32, 32, 32, 32, 32, 32, 32, 1]
    ctx.sync_status()


def test_chi32_fmnist_d256_sampled(dk):
    """The precision-form data (d = 256) at reps = 5 (bond 32): 8 train x 8 train and
    4 test rows against the oracle (TEBD, untruncated), element by element."""
    dualk, ctx, torch = dk
    from oracle import gram as og
    from paper_2602_01330_gb300 import synthetic
    d = synthetic.fmnist_like(8, 4, 256)
    xtr, xte = d["x_train"], d["x_test"]
    fm = dualk.FeatureMap(reps=5, chi_max=32)
    mtr = dualk.mps_build(ctx, _dev(torch, xtr), fm)
    mte = dualk.mps_build(ctx, _dev(torch, xte), fm)
    out = dualk.gram(ctx, mtr, w=0.5)
    rows = dualk.dual_kernel_rows(ctx, mte, mtr, w=0.5)
    torch.cuda.synchronize()
    kq, lkq = _oracle_block(xtr, xtr, 5)
    _check_block(out, kq, lkq, og.rbf(xtr, xtr, 1 / 256), 0.5)
    kq, lkq = _oracle_block(xte, xtr, 5)
    _check_block(rows, kq, lkq, og.rbf(xte, xtr, 1 / 256), 0.5)
    ctx.sync_status()


TOL_MIXED = 1e-4  # split-BF16 (bf16x3) tensor-core path


def test_chi32_bf16x3_vs_statevector_and_fp32(dk):
    """Tensor-core bond-32 path: within 1e-4 of brute force at n = 12, exact diagonal, and
    within 1e-4 of the FP32 bond-32 path on the same tensors."""
    dualk, ctx, torch = dk
    from oracle import circuit
    from paper_2602_01330_gb300 import synthetic
    x = synthetic.uniform_angles(11, 12, seed=12)
    ref = circuit.kernel_matrix(x, x, 5)
    m = dualk.mps_build(ctx, _dev(torch, x), dualk.FeatureMap(reps=5, chi_max=32))
    mixed = dualk.gram(ctx, m, w=1.0, prec=dualk.DK_PREC_BF16X3)
    fp32 = dualk.gram(ctx, m, w=1.0)
    torch.cuda.synchronize()
    kq = mixed["kq"].cpu().numpy()
    assert np.max(np.abs(kq - ref)) <= TOL_MIXED
    assert np.all(np.diag(kq) == 1.0)
    assert np.max(np.abs(kq - fp32["kq"].cpu().numpy())) <= TOL_MIXED
    ctx.sync_status()


def test_chi32_bf16x3_fmnist_d256(dk):
    dualk, ctx, torch = dk
    from oracle import gram as og
    from paper_2602_01330_gb300 import synthetic
    d = synthetic.fmnist_like(8, 4, 256)
    xtr, xte = d["x_train"], d["x_test"]
    fm = dualk.FeatureMap(reps=5, chi_max=32)
    mtr = dualk.mps_build(ctx, _dev(torch, xtr), fm)
    mte = dualk.mps_build(ctx, _dev(torch, xte), fm)
    out = dualk.gram(ctx, mtr, w=0.5, prec=dualk.DK_PREC_BF16X3)
    rows = dualk.dual_kernel_rows(ctx, mte, mtr, w=0.5, prec=dualk.DK_PREC_BF16X3)
    torch.cuda.synchronize()
    for got, xa, xb in ((out, xtr, xtr), (rows, xte, xtr)):
        kq, lkq = _oracle_block(xa, xb, 5)
        assert np.max(np.abs(got["kq"].cpu().numpy() - kq)) <= TOL_MIXED
        k_ref = og.dual_kernel(kq, og.rbf(xa, xb, 1 / 256), 0.5)
        assert np.max(np.abs(got["k"].cpu().numpy() - k_ref)) <= TOL_MIXED
    ctx.sync_status()
