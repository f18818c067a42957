"""GPU parity of the block-statevector Gram (dk_block_states + dk_gram_blocks) for
block-structured feature maps (§II-C): K_q = prod_B |<psi_B(x_i)|psi_B(x_j)>|^2, exact at any
n, with the RBF kernel and the mix fused as in every Gram call.

Reference: the oracle's dense statevector of every block (``oracle.circuit.statevector``),
summed in log domain. Tolerances as for the MPS Gram: |dK| <= 1e-6 on K, K_q and K_c (FP32
dot products, float32 outputs); log K_q within 1e-3 * max(1, |log K_q|) where the reference
is above -700, and 1e-4 relative at n = 784. The MPS paths for the same maps (closed-form
chain build with blocks, and the SVD build of all-to-all blocks) must agree to 1e-6."""
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


FORMS = ("tcgen05", "mma_sync")


class _form:
    """Selects the split-BF16 block kernels of the context for a with-block."""

    def __init__(self, dualk, ctx, name):
        self.dualk, self.ctx = dualk, ctx
        self.form = dualk.DK_BLOCK_TCGEN05 if name == "tcgen05" else dualk.DK_BLOCK_MMA_SYNC

    def __enter__(self):
        self.ctx.set_block_gram_form(self.form)

    def __exit__(self, *exc):
        self.ctx.set_block_gram_form(self.dualk.DK_BLOCK_TCGEN05)


def _ref_log(xr, xc, reps, b, entangler):
    from oracle import circuit
    n = xr.shape[1]
    out = np.zeros((xr.shape[0], xc.shape[0]))
    for s in range(0, n, b):
        e = min(s + b, n)
        a = np.stack([circuit.statevector(r[s:e].astype(np.float64), reps, entangler=entangler) for r in xr])
        c = np.stack([circuit.statevector(r[s:e].astype(np.float64), reps, entangler=entangler) for r in xc])
        with np.errstate(divide="ignore"):
            out += np.log(np.abs(a.conj() @ c.T) ** 2)
    return out


def _check(out, lref, kc_ref, w):
    kq = out["kq"].cpu().numpy().astype(np.float64)
    lkq = out["logkq"].cpu().numpy().astype(np.float64)
    kc = out["kc"].cpu().numpy().astype(np.float64)
    k = out["k"].cpu().numpy().astype(np.float64)
    kq_ref = np.exp(lref)
    assert np.max(np.abs(kq - kq_ref)) <= 1e-6
    assert np.max(np.abs(kc - kc_ref)) <= 1e-6
    assert np.max(np.abs(k - (w * kq_ref + (1 - w) * kc_ref))) <= 1e-6
    sel = lref > -700
    assert np.all(np.abs(lkq[sel] - lref[sel]) <= 1e-3 * np.maximum(1.0, np.abs(lref[sel])))


@pytest.mark.parametrize("n,b,reps,ent", [(40, 8, 2, "full"), (50, 7, 2, "chain"), (36, 12, 2, "full"),
                                          (9, 2, 3, "full"), (7, 1, 2, "full"), (30, 5, 1, "chain")])
def test_gram_blocks_vs_block_statevectors(dk, n, b, reps, ent):
    """Symmetric Gram of 70 samples (a full and a ragged tile) and 20 x 70 rows, element by
    element; blocks of 1, 2 (below the 16-amplitude chunk), 5, 7, 8 and 12 qubits, short
    last blocks (n = 50, 9, 7)."""
    dualk, ctx, torch = dk
    from oracle import gram as og
    from paper_2602_01330_gb300 import synthetic
    d = synthetic.fmnist_like(70, 20, n)
    xtr, xte = d["x_train"], d["x_test"]
    fm = dualk.FeatureMap(reps=reps, block=b)
    e = dualk.DK_ENT_FULL if ent == "full" else dualk.DK_ENT_CHAIN
    str_, ste = dualk.block_states(ctx, _dev(torch, xtr), fm, e), dualk.block_states(ctx, _dev(torch, xte), fm, e)
    g = dualk.gram_blocks(ctx, str_, w=0.5)
    r = dualk.gram_blocks(ctx, ste, str_, w=0.5)
    torch.cuda.synchronize()
    _check(g, _ref_log(xtr, xtr, reps, b, ent), og.rbf(xtr, xtr, 1.0 / n), 0.5)
    _check(r, _ref_log(xte, xtr, reps, b, ent), og.rbf(xte, xtr, 1.0 / n), 0.5)
    kq = g["kq"].cpu().numpy()
    assert np.all(np.diag(kq) == 1.0)
    assert np.array_equal(kq, kq.T)
    # positive semi-definite to the FP32 bound lambda_min >= -m 1e-6
    assert np.linalg.eigvalsh(kq.astype(np.float64)).min() >= -kq.shape[0] * 1e-6
    ctx.sync_status()


def test_gram_blocks_large_tiles(dk):
    """2000 samples, so that the 128 x 64 pair tile is the one chosen (2000 = 15 x 128 + 80
    leaves a ragged last row tile): the full 2000 x 2000 Gram of two all-to-all blocks of 8
    and 300 x 2000 rows (64 x 64 tiles), element by element."""
    dualk, ctx, torch = dk
    from oracle import gram as og
    from paper_2602_01330_gb300 import synthetic
    d = synthetic.fmnist_like(2000, 300, 16)
    xtr, xte = d["x_train"], d["x_test"]
    fm = dualk.FeatureMap(reps=2, block=8)
    st = dualk.block_states(ctx, _dev(torch, xtr), fm, dualk.DK_ENT_FULL)
    se = dualk.block_states(ctx, _dev(torch, xte), fm, dualk.DK_ENT_FULL)
    g = dualk.gram_blocks(ctx, st, w=0.5)
    r = dualk.gram_blocks(ctx, se, st, w=0.5)
    torch.cuda.synchronize()
    _check(g, _ref_log(xtr, xtr, 2, 8, "full"), og.rbf(xtr, xtr, 1.0 / 16), 0.5)
    _check(r, _ref_log(xte, xtr, 2, 8, "full"), og.rbf(xte, xtr, 1.0 / 16), 0.5)
    kq = g["kq"].cpu().numpy()
    assert np.all(np.diag(kq) == 1.0)
    assert np.array_equal(kq, kq.T)
    ctx.sync_status()


def test_gram_blocks_n784_log_kernel(dk):
    """All 784 pixels in blocks of 10 with all-to-all ZZ (exact bond up to 32 inside a block,
    beyond any bond-16 MPS): 48 images, every pair's log K_q against the oracle."""
    dualk, ctx, torch = dk
    from paper_2602_01330_gb300 import synthetic
    x = synthetic.fmnist_like(48, 0, 784)["x_train"]
    st = dualk.block_states(ctx, _dev(torch, x), dualk.FeatureMap(reps=2, block=10), dualk.DK_ENT_FULL)
    g = dualk.gram_blocks(ctx, st, w=1.0, want=("kq", "logkq"))
    torch.cuda.synchronize()
    ref = _ref_log(x, x, 2, 10, "full")
    lkq = g["logkq"].cpu().numpy().astype(np.float64)
    off = ~np.eye(48, dtype=bool)
    assert np.all(ref[off] < -100)
    assert np.max(np.abs(lkq[off] - ref[off]) / np.abs(ref[off])) <= 1e-4
    assert np.all(np.diag(g["kq"].cpu().numpy()) == 1.0)
    ctx.sync_status()


def test_gram_blocks_agrees_with_mps_paths(dk):
    """The same block-structured states through the MPS Gram: the closed-form chain build with
    blocks (bond 4) and the SVD build of all-to-all blocks of 8 (bond 16, exact at chi_max 32)."""
    dualk, ctx, torch = dk
    from paper_2602_01330_gb300 import synthetic
    x = _dev(torch, synthetic.fmnist_like(60, 0, 48)["x_train"])
    chain = dualk.gram_blocks(ctx, dualk.block_states(ctx, x, dualk.FeatureMap(reps=2, block=8), dualk.DK_ENT_CHAIN),
                              w=0.5)
    mchain = dualk.gram(ctx, dualk.mps_build(ctx, x, dualk.FeatureMap(reps=2, chi_max=4, block=8)), w=0.5)
    full = dualk.gram_blocks(ctx, dualk.block_states(ctx, x, dualk.FeatureMap(reps=2, block=8), dualk.DK_ENT_FULL),
                             w=0.5)
    mfull, _ = dualk.mps_build_blocks(ctx, x, dualk.FeatureMap(reps=2, chi_max=32, block=8), dualk.DK_ENT_FULL)
    gfull = dualk.gram(ctx, mfull, w=0.5)
    torch.cuda.synchronize()
    for a, b in ((chain, mchain), (full, gfull)):
        assert torch.max(torch.abs(a["kq"] - b["kq"])).item() <= 1e-6
        assert torch.max(torch.abs(a["k"] - b["k"])).item() <= 1e-6
        assert torch.equal(a["kc"], b["kc"])
    ctx.sync_status()


def _check_tol(out, lref, kc_ref, w, tol):
    kq = out["kq"].cpu().numpy().astype(np.float64)
    kq_ref = np.exp(lref)
    assert np.max(np.abs(kq - kq_ref)) <= tol
    assert np.max(np.abs(out["kc"].cpu().numpy() - kc_ref)) <= 1e-6
    assert np.max(np.abs(out["k"].cpu().numpy() - (w * kq_ref + (1 - w) * kc_ref))) <= tol
    lkq = out["logkq"].cpu().numpy().astype(np.float64)
    sel = lref > -700
    assert np.all(np.abs(lkq[sel] - lref[sel]) <= 1e-3 * np.maximum(1.0, np.abs(lref[sel])))


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("m,n,b,reps,ent", [(70, 40, 8, 2, "full"), (70, 50, 7, 2, "chain"), (70, 36, 12, 2, "full"),
                                            (70, 9, 2, 3, "full"), (300, 16, 8, 2, "full"), (2000, 16, 8, 2, "full"),
                                            (70, 27, 9, 3, "full"), (70, 25, 11, 2, "chain")])
def test_gram_blocks_bf16x3_tensor_cores(dk, m, n, b, reps, ent, form):
    """Split-BF16 tensor-core forms (tcgen05 and mma.sync) against the oracle with the
    mixed-precision tolerance 1e-4 on K_q and K (K_c stays FP32, 1e-6): one ragged tile (70
    samples), several (300) and a full-size Gram (2000 = 15 x 128 + 80); short last blocks
    (n = 50, 9, 25); blocks of 7 to 12 qubits (every register form of the state build) and
    of 2; rows; exact unit diagonal from the self-norms of the same MMA sequence; exact
    symmetry."""
    dualk, ctx, torch = dk
    from oracle import gram as og
    from paper_2602_01330_gb300 import synthetic
    d = synthetic.fmnist_like(m, 20, n)
    xtr, xte = d["x_train"], d["x_test"]
    fm = dualk.FeatureMap(reps=reps, block=b)
    e = dualk.DK_ENT_FULL if ent == "full" else dualk.DK_ENT_CHAIN
    p = dualk.DK_PREC_BF16X3
    with _form(dualk, ctx, form):
        str_ = dualk.block_states(ctx, _dev(torch, xtr), fm, e, prec=p)
        ste = dualk.block_states(ctx, _dev(torch, xte), fm, e, prec=p)
        g = dualk.gram_blocks(ctx, str_, w=0.5)
        r = dualk.gram_blocks(ctx, ste, str_, w=0.5)
        torch.cuda.synchronize()
    _check_tol(g, _ref_log(xtr, xtr, reps, b, ent), og.rbf(xtr, xtr, 1.0 / n), 0.5, 1e-4)
    _check_tol(r, _ref_log(xte, xtr, reps, b, ent), og.rbf(xte, xtr, 1.0 / n), 0.5, 1e-4)
    kq = g["kq"].cpu().numpy()
    assert np.all(np.diag(kq) == 1.0)
    assert np.array_equal(kq, kq.T)
    # positive semi-definite to the mixed-precision bound lambda_min >= -m 1e-4
    assert np.linalg.eigvalsh(kq.astype(np.float64)).min() >= -m * 1e-4
    ctx.sync_status()


@pytest.mark.parametrize("form", FORMS)
def test_gram_blocks_bf16x3_n784_matches_fp32(dk, form):
    """n = 784 in blocks of 10: the tensor-core log K_q against the FP32 form (and both
    against the oracle on a sample) to 1e-4 relative; 200 samples in 79 blocks give 158
    self-norm units, more than one per SM."""
    dualk, ctx, torch = dk
    from paper_2602_01330_gb300 import synthetic
    x = _dev(torch, synthetic.fmnist_like(200, 0, 784)["x_train"])
    fm = dualk.FeatureMap(reps=2, block=10)
    a = dualk.gram_blocks(ctx, dualk.block_states(ctx, x, fm, dualk.DK_ENT_FULL), w=1.0, want=("logkq",))
    with _form(dualk, ctx, form):
        b = dualk.gram_blocks(ctx, dualk.block_states(ctx, x, fm, dualk.DK_ENT_FULL, prec=dualk.DK_PREC_BF16X3),
                              w=1.0, want=("logkq",))
        torch.cuda.synchronize()
    assert np.all(np.diag(b["logkq"].cpu().numpy()) == 0.0)
    la, lb = a["logkq"].cpu().numpy().astype(np.float64), b["logkq"].cpu().numpy().astype(np.float64)
    off = ~np.eye(200, dtype=bool)
    assert np.max(np.abs(la[off] - lb[off]) / np.abs(la[off])) <= 1e-4
    ref = _ref_log(x[:12].cpu().numpy(), x[:12].cpu().numpy(), 2, 10, "full")
    o12 = ~np.eye(12, dtype=bool)
    assert np.max(np.abs(lb[:12, :12][o12] - ref[o12]) / np.abs(ref[o12])) <= 1e-4
    ctx.sync_status()


def test_gram_blocks_errors(dk):
    dualk, ctx, torch = dk
    x = torch.rand(8, 30, device="cuda")
    with pytest.raises(ValueError):
        dualk.block_states(ctx, x, dualk.FeatureMap(reps=2, block=13))
    with pytest.raises(ValueError):
        dualk.block_states(ctx, x, dualk.FeatureMap(reps=2, block=0))  # one block of 30 qubits
    st = dualk.block_states(ctx, x, dualk.FeatureMap(reps=2, block=6))
    lib = dualk._lib()
    out = torch.empty(8, 8, device="cuda")
    # symmetric with different row and column ranges
    assert lib.dk_gram_blocks(ctx.handle, dualk._ptr(st.data), 8, dualk._ptr(st.data), 8, 30, 6, 0, 4, 2, 4,
                              dualk._ptr(st.log_norm), dualk._ptr(st.log_norm), dualk._ptr(x), dualk._ptr(x),
                              0.1, 1.0, 0, None, dualk._ptr(out), None, None, 8, 1, None, 0, dualk._stream(None)) == 1
    # ld below ncols
    assert lib.dk_gram_blocks(ctx.handle, dualk._ptr(st.data), 8, dualk._ptr(st.data), 8, 30, 6, 0, 8, 0, 8,
                              dualk._ptr(st.log_norm), dualk._ptr(st.log_norm), dualk._ptr(x), dualk._ptr(x),
                              0.1, 1.0, 0, None, dualk._ptr(out), None, None, 4, 0, None, 0, dualk._stream(None)) == 1
    ctx.sync_status()


@pytest.mark.parametrize("prec", ["f32", "bf16x3", "bf16x3_mma_sync"])
def test_gram_blocks_edge_cases(dk, prec):
    """One sample (K = 1), one qubit (n = 1, block 1: the product form cos^2(x - y) at one
    repetition), a single block of 12 qubits (block 0 with n = 12), and an empty row range."""
    dualk, ctx, torch = dk
    with _form(dualk, ctx, "mma_sync" if prec == "bf16x3_mma_sync" else "tcgen05"):
        _edge_cases(dualk, ctx, torch, prec)


def _edge_cases(dualk, ctx, torch, prec):
    from paper_2602_01330_gb300 import synthetic
    p = dualk.DK_PREC_F32 if prec == "f32" else dualk.DK_PREC_BF16X3
    tol = 1e-6 if prec == "f32" else 1e-4
    x1 = _dev(torch, synthetic.uniform_angles(1, 7, 60))
    g1 = dualk.gram_blocks(ctx, dualk.block_states(ctx, x1, dualk.FeatureMap(reps=2, block=3), prec=p), w=0.5)
    xs = synthetic.uniform_angles(9, 1, 61)
    gs = dualk.gram_blocks(ctx, dualk.block_states(ctx, _dev(torch, xs), dualk.FeatureMap(reps=1, block=1), prec=p),
                           w=1.0, want=("kq",))
    x12 = synthetic.uniform_angles(10, 12, 62)
    g12 = dualk.gram_blocks(ctx, dualk.block_states(ctx, _dev(torch, x12), dualk.FeatureMap(reps=2, block=0),
                                                    dualk.DK_ENT_FULL, prec=p), w=1.0, want=("kq",))
    torch.cuda.synchronize()
    assert g1["k"].item() == 1.0 and g1["kq"].item() == 1.0
    prod = np.cos(xs[:, None, 0] - xs[None, :, 0]) ** 2
    assert np.max(np.abs(gs["kq"].cpu().numpy() - prod)) <= tol
    ref = np.exp(_ref_log(x12, x12, 2, 12, "full"))
    assert np.max(np.abs(g12["kq"].cpu().numpy() - ref)) <= tol
    st = dualk.block_states(ctx, x1, dualk.FeatureMap(reps=2, block=3), prec=p)
    out = torch.full((1, 1), -3.0, device="cuda")
    assert dualk._lib().dk_gram_blocks(ctx.handle, dualk._ptr(st.data), 1, dualk._ptr(st.data), 1, 7, 3, 0, 0, 0, 1,
                                       dualk._ptr(st.log_norm), dualk._ptr(st.log_norm), dualk._ptr(x1),
                                       dualk._ptr(x1), 0.1, 1.0, p, None, dualk._ptr(out), None, None, 1, 0,
                                       None, 0, dualk._stream(None)) == 0
    torch.cuda.synchronize()
    assert out.item() == -3.0  # nothing to compute, nothing written
    ctx.sync_status()


def _forms_agree(a, c):
    """The two forms multiply the same split-BF16 operands and accumulate in other orders
    (the tcgen05 form sums a_re b and a_im b separately, then combines): 99.9 % of the log K_q
    entries agree to 2e-5 relative, and every one to the mixed-precision log tolerance 1e-3
    (pairs with tiny block overlaps, log K_q ~ -24 at n = 16, are ~1e-3 off the oracle in
    both forms alike)."""
    rel = np.abs(a - c) / np.maximum(1.0, np.abs(c))
    assert np.quantile(rel, 0.999) <= 2e-5
    assert np.max(rel) <= 1e-3


def test_block_gram_forms_agree_and_persist(dk):
    """The tcgen05 and mma.sync kernels on the same split-BF16 states agree (_forms_agree) and
    both are within the mixed-precision tolerance of the oracle; a symmetric Gram of 4000
    samples (528 tiles of 128 x 128, several per CTA), a rectangular 2000 x 1900 block (128 x
    128 tiles, several per CTA) and 500 rows; rows and columns offset into the sample
    range."""
    dualk, ctx, torch = dk
    from paper_2602_01330_gb300 import synthetic
    n, b = 16, 8
    fm = dualk.FeatureMap(reps=2, block=b)
    p = dualk.DK_PREC_BF16X3
    x4 = synthetic.fmnist_like(4000, 500, n)
    xa, xt = x4["x_train"], x4["x_test"]
    res = {}
    for form in FORMS:
        with _form(dualk, ctx, form):
            sa = dualk.block_states(ctx, _dev(torch, xa), fm, dualk.DK_ENT_FULL, prec=p)
            st = dualk.block_states(ctx, _dev(torch, xt), fm, dualk.DK_ENT_FULL, prec=p)
            g = dualk.gram_blocks(ctx, sa, w=1.0, want=("logkq",))
            rect = torch.empty(2000, 1900, device="cuda")
            ws, nws = _ws(dualk, ctx, n, b, 2000, 1900, p, 0, 0)
            _check_call(dualk, dualk._lib().dk_gram_blocks(
                ctx.handle, dualk._ptr(sa.data), 4000, dualk._ptr(sa.data), 4000, n, b, 100, 2000, 2100, 1900,
                dualk._ptr(sa.log_norm), dualk._ptr(sa.log_norm), None, None, 0.0, 1.0, p, None, None, None,
                dualk._ptr(rect), 1900, 0, dualk._ptr(ws), nws, dualk._stream(None)))
            r = dualk.gram_blocks(ctx, st, sa, w=1.0, want=("logkq",))
            torch.cuda.synchronize()
            res[form] = (g["logkq"].cpu().numpy().astype(np.float64), rect.cpu().numpy().astype(np.float64),
                         r["logkq"].cpu().numpy().astype(np.float64))
            assert np.all(np.diag(res[form][0]) == 0.0)
    for a, c in zip(res["tcgen05"], res["mma_sync"]):
        _forms_agree(a, c)
    def near(lg, ref):
        assert np.max(np.abs(np.exp(lg) - np.exp(ref))) <= 1e-4
        assert np.max(np.abs(lg - ref) / np.maximum(1.0, np.abs(ref))) <= 1e-3

    gi, gj = np.arange(0, 4000, 97), np.arange(3, 4000, 89)
    near(res["tcgen05"][0][np.ix_(gi, gj)], _ref_log(xa[gi], xa[gj], 2, b, "full"))
    ri, rj = np.arange(100, 2100, 101), np.arange(2100, 4000, 93)
    near(res["tcgen05"][1][np.ix_(ri - 100, rj - 2100)], _ref_log(xa[ri], xa[rj], 2, b, "full"))
    ti = np.arange(0, 500, 25)
    near(res["tcgen05"][2][np.ix_(ti, gj)], _ref_log(xt[ti], xa[gj], 2, b, "full"))
    ctx.sync_status()


@pytest.mark.parametrize("case", ["split_n784", "one_block"])
def test_block_gram_rows_split_and_narrow_tiles(dk, case):
    """Rectangular blocks: 300 x 1000 at n = 784 in blocks of 10 (24 tiles of 128 x 128, so
    the 79 blocks are split over 6 work items per tile and the partial log sums added by the
    finishing kernel) and 300 x 700 with a single block of 10 qubits (no split possible: the
    128 x 64 tiles); tcgen05 against mma.sync (_forms_agree), K_c identical, and against the
    oracle on a sample."""
    dualk, ctx, torch = dk
    from oracle import gram as og
    from paper_2602_01330_gb300 import synthetic
    n, b, mr, mc = (784, 10, 300, 1000) if case == "split_n784" else (10, 10, 300, 700)
    d = synthetic.fmnist_like(mc, mr, n)
    xc, xr = d["x_train"], d["x_test"]
    fm = dualk.FeatureMap(reps=2, block=b)
    p = dualk.DK_PREC_BF16X3
    res = {}
    for form in FORMS:
        with _form(dualk, ctx, form):
            sc = dualk.block_states(ctx, _dev(torch, xc), fm, dualk.DK_ENT_FULL, prec=p)
            sr = dualk.block_states(ctx, _dev(torch, xr), fm, dualk.DK_ENT_FULL, prec=p)
            out = dualk.gram_blocks(ctx, sr, sc, w=0.5)
            torch.cuda.synchronize()
            res[form] = {k: v.cpu().numpy().astype(np.float64) for k, v in out.items()}
    a, c = res["tcgen05"], res["mma_sync"]
    _forms_agree(a["logkq"], c["logkq"])
    assert np.array_equal(a["kc"], c["kc"])
    ri, cj = np.arange(0, mr, 23), np.arange(0, mc, 41)
    ref = _ref_log(xr[ri], xc[cj], 2, b, "full")
    got = a["logkq"][np.ix_(ri, cj)]
    assert np.max(np.abs(np.exp(got) - np.exp(ref))) <= 1e-4
    assert np.max(np.abs(got - ref) / np.maximum(1.0, np.abs(ref))) <= 1e-3
    assert np.max(np.abs(a["kc"][np.ix_(ri, cj)] - og.rbf(xr[ri], xc[cj], 1.0 / n))) <= 1e-6
    ctx.sync_status()


@pytest.mark.parametrize("form", FORMS)
def test_block_gram_symmetric_offset_diagonal(dk, form):
    """A symmetric block starting at sample 50 (not a multiple of the 128-sample tile): each
    sample's diagonal element sits at another position of its Gram tile than of its
    self-norm tile, and K_q(x, x) = 1 must still hold exactly; off the diagonal the block
    equals the same entries of the full Gram to 1e-6 relative in log K_q."""
    dualk, ctx, torch = dk
    from paper_2602_01330_gb300 import synthetic
    x = _dev(torch, synthetic.fmnist_like(600, 0, 40)["x_train"])
    fm = dualk.FeatureMap(reps=2, block=10)
    with _form(dualk, ctx, form):
        s = dualk.block_states(ctx, x, fm, dualk.DK_ENT_FULL, prec=dualk.DK_PREC_BF16X3)
        # both blocks straight from the Gram kernels (no refinement pass on either side)
        full = dualk.gram_blocks(ctx, s, w=1.0, want=("logkq",), refine=None)["logkq"]
        sub = torch.full((300, 300), -7.0, device="cuda")
        ws, nws = _ws(dualk, ctx, 40, 10, 300, 300, dualk.DK_PREC_BF16X3, 1, 0)
        _check_call(dualk, dualk._lib().dk_gram_blocks(
            ctx.handle, dualk._ptr(s.data), 600, dualk._ptr(s.data), 600, 40, 10, 50, 300, 50, 300,
            dualk._ptr(s.log_norm), dualk._ptr(s.log_norm), None, None, 0.0, 1.0, dualk.DK_PREC_BF16X3, None,
            None, None, dualk._ptr(sub), 300, 1, dualk._ptr(ws), nws, dualk._stream(None)))
        torch.cuda.synchronize()
    sub, full = sub.cpu().numpy().astype(np.float64), full.cpu().numpy().astype(np.float64)
    assert np.all(np.diag(sub) == 0.0)
    ref = full[50:350, 50:350]
    assert np.max(np.abs(sub - ref) / np.maximum(1.0, np.abs(ref))) <= 1e-6
    ctx.sync_status()


def _check_call(dualk, status):
    assert status == 0, status


def _ws(dualk, ctx, n, b, nrows, ncols, prec, symmetric, with_kc):
    """Caller workspace of a direct dk_gram_blocks call: (tensor or None, bytes)."""
    import torch
    nbytes = int(dualk._lib().dk_gram_blocks_workspace_bytes(ctx.handle, n, b, nrows, ncols, prec, symmetric,
                                                             with_kc))
    return (torch.empty(nbytes, dtype=torch.uint8, device="cuda") if nbytes else None), nbytes


def test_svm_workflow_on_a_block_map(dk):
    """The §II-D workflow with the block-structured map (all-to-all ZZ in blocks of 8) from
    raw features: block Gram and rows, cross-validation, fit, test accuracy far above chance
    (0.1) on the synthetic classes; the quantum kernel alone (w = 1) is evaluated too."""
    dualk, ctx, torch = dk
    from paper_2602_01330_gb300 import svm
    out = svm.run_pipeline(ctx, n_train=300, n_test=100, d=32, Cs=(1.0, 10.0), ws=(0.5, 1.0), block=8,
                           entangler="full")
    assert out["test_accuracy"] > 0.5
    assert 0.0 <= out["cv_accuracy_by_w"]["1.0"] <= 1.0
    ctx.sync_status()


def test_tcgen05_block_calls_use_the_callers_workspace(dk):
    """The tcgen05 form takes its scratch from the caller: the queries give the sizes (the
    RBF distances, and partial sums of a rectangular block split over its blocks), a call
    with too small a workspace returns DK_ERR_WORKSPACE without launching, and a call with
    the queried size matches the binding's result bit for bit."""
    import ctypes
    dualk, ctx, torch = dk
    from paper_2602_01330_gb300 import synthetic
    lib = dualk._lib()
    d = synthetic.fmnist_like(300, 40, 60)
    fm = dualk.FeatureMap(reps=2, block=10)
    xtr, xte = _dev(torch, d["x_train"]), _dev(torch, d["x_test"])
    ws_states = int(lib.dk_block_states_workspace_bytes(ctx.handle, 300, 60, 10, dualk.DK_PREC_BF16X3))
    assert ws_states >= 6 * 300 * 4 and ws_states % 256 == 0
    assert int(lib.dk_block_states_workspace_bytes(ctx.handle, 300, 60, 10, dualk.DK_PREC_F32)) == 0
    s_tr = dualk.block_states(ctx, xtr, fm, dualk.DK_ENT_FULL, prec=dualk.DK_PREC_BF16X3)
    s_te = dualk.block_states(ctx, xte, fm, dualk.DK_ENT_FULL, prec=dualk.DK_PREC_BF16X3)
    # states with too small a workspace: rejected on the host
    out = torch.empty_like(s_tr.data)
    ln = torch.empty(300, device="cuda")
    small = torch.empty(ws_states - 256, dtype=torch.uint8, device="cuda")
    fmc = fm._c()
    st = dualk._stream(None)
    assert lib.dk_block_states(ctx.handle, dualk._ptr(xtr), 300, 60, ctypes.byref(fmc), dualk.DK_ENT_FULL,
                               dualk.DK_PREC_BF16X3, dualk._ptr(out), dualk._ptr(ln), dualk._ptr(small),
                               ws_states - 256, st) == 5
    # rows 40 x 300: 1 x 3 tiles of 128 x 128, fewer than the SMs, so the blocks are split
    ws_rows = int(lib.dk_gram_blocks_workspace_bytes(ctx.handle, 60, 10, 40, 300, dualk.DK_PREC_BF16X3, 0, 1))
    ws_rows_nokc = int(lib.dk_gram_blocks_workspace_bytes(ctx.handle, 60, 10, 40, 300, dualk.DK_PREC_BF16X3, 0, 0))
    ws_sym = int(lib.dk_gram_blocks_workspace_bytes(ctx.handle, 60, 10, 300, 300, dualk.DK_PREC_BF16X3, 1, 1))
    assert ws_rows > ws_rows_nokc > 0
    assert ws_rows - ws_rows_nokc == (40 * 300 * 4 + 255) // 256 * 256
    assert ws_sym == (300 * 300 * 4 + 255) // 256 * 256
    assert int(lib.dk_gram_blocks_workspace_bytes(ctx.handle, 60, 10, 300, 300, dualk.DK_PREC_F32, 1, 1)) == 0
    ref = dualk.gram_blocks(ctx, s_te, s_tr, w=0.5)
    k = torch.empty((40, 300), device="cuda")
    args = lambda ws, nb: (ctx.handle, dualk._ptr(s_te.data), 40, dualk._ptr(s_tr.data), 300, 60, 10, 0, 40, 0, 300,
                           dualk._ptr(s_te.log_norm), dualk._ptr(s_tr.log_norm), dualk._ptr(xte), dualk._ptr(xtr),
                           1.0 / 60, 0.5, dualk.DK_PREC_BF16X3, dualk._ptr(k), None, None, None, 300, 0,
                           dualk._ptr(ws), nb, st)
    tiny = torch.empty(ws_rows - 256, dtype=torch.uint8, device="cuda")
    assert lib.dk_gram_blocks(*args(tiny, ws_rows - 256)) == 5
    assert lib.dk_gram_blocks(*args(None, 0)) == 5
    ws = torch.full((ws_rows,), 0xAB, dtype=torch.uint8, device="cuda")  # stale contents must not matter
    assert lib.dk_gram_blocks(*args(ws, ws_rows)) == 0
    torch.cuda.synchronize()
    ctx.sync_status()
    assert torch.equal(k, ref["k"])


def _block_pair_logs(xa, xb, reps, b, entangler):
    """Oracle log K_q of the aligned pairs (xa[p], xb[p]): the sum over blocks of
    log |<psi_B(a)|psi_B(b)>|^2 from the oracle's dense block statevectors."""
    from oracle import circuit
    n = xa.shape[1]
    out = np.zeros(xa.shape[0])
    for s in range(0, n, b):
        e = min(s + b, n)
        for p in range(xa.shape[0]):
            u = circuit.statevector(xa[p, s:e].astype(np.float64), reps, entangler=entangler)
            v = circuit.statevector(xb[p, s:e].astype(np.float64), reps, entangler=entangler)
            out[p] += np.log(abs(np.vdot(u, v)) ** 2)
    return out


@pytest.mark.parametrize("prec", ["f32", "bf16x3"])
def test_block_gram_near_duplicates_n784(dk, prec):
    """n = 784 in all-to-all blocks of 10 (79 blocks), 300 samples of which 200..263 are near
    copies of 0..63 (K_q spread over about 1e-3 .. 1): the near pairs of the symmetric Gram
    against the oracle, 1e-6 on K_q in FP32 and 1e-4 in split BF16 (tcgen05 form), after the
    refinement pass (dk_gram_blocks_refine) the binding runs; without it the Gram kernels'
    sums of 79 block logs leave about 5e-5 (FP32) and 4e-4 (split BF16), printed too."""
    import json
    dualk, ctx, torch = dk
    from paper_2602_01330_gb300 import synthetic
    x = synthetic.fmnist_like(300, 0, 784)["x_train"].copy()
    x[200:264] = synthetic.near_copies(x[0:64], 3e-4, 3e-2, seed=71)
    p = dualk.DK_PREC_F32 if prec == "f32" else dualk.DK_PREC_BF16X3
    fm = dualk.FeatureMap(reps=2, block=10)
    s = dualk.block_states(ctx, _dev(torch, x), fm, dualk.DK_ENT_FULL, prec=p)
    g = dualk.gram_blocks(ctx, s, w=1.0, want=("kq", "logkq"))
    g0 = dualk.gram_blocks(ctx, s, w=1.0, want=("kq", "logkq"), refine=None)
    torch.cuda.synchronize()
    ctx.sync_status()
    ref = np.exp(_block_pair_logs(x[0:64], x[200:264], 2, 10, "full"))
    pick = lambda t: t.cpu().numpy().astype(np.float64)[np.arange(64), np.arange(200, 264)]
    got, got0 = pick(g["kq"]), pick(g0["kq"])
    err = np.abs(got - ref)
    big = ref > 1e-3
    print(json.dumps({"case": f"block gram n784 near pairs {prec}", "pairs_kq_gt_1e-3": int(big.sum()),
                      "max_abs_dkq": float(err.max()), "max_rel_dkq": float((err[big] / ref[big]).max()),
                      "max_abs_dkq_without_refinement": float(np.abs(got0 - ref).max())}))
    # entries at or below tau keep the Gram kernels' bits
    kq0 = g0["kq"].cpu().numpy()
    keep = ~(kq0 > dualk.REFINE_TAU) | np.eye(300, dtype=bool)
    assert np.array_equal(kq0[keep], g["kq"].cpu().numpy()[keep])
    assert np.all(np.diag(g["logkq"].cpu().numpy()) == 0.0)
    assert big.sum() >= 40
    assert err.max() <= (1e-6 if prec == "f32" else 1e-4)
