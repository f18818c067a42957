"""Split-BF16 operands of bond-32 MPS (dk_mps_split32, dtype DK_SPLIT_BF16).

The operands are a plain function of the complex64 site tensors (§II-C Eqs. 8-10 on tensor
cores): every value v of the transposed 16 x 16 blocks A_s[t] becomes hi = round(v) and
lo = round(v - hi) in BF16 (round to nearest even). The test writes that definition out in
NumPy on the stored tensors and asks for the same bytes, then checks that a Gram call on the
operands gives the bits of the same call on the complex64 tensors (the kernel that splits
for every tile), and the host-side rejections.
"""
import ctypes

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


def _bf16_rne(v):
    """float32 -> BF16 bits, round to nearest even (finite inputs)."""
    b = np.ascontiguousarray(v, dtype=np.float32).view(np.uint32).astype(np.uint64)
    return ((b + 0x7FFF + ((b >> 16) & 1)) >> 16).astype(np.uint16)


def _bf16_value(h):
    return (h.astype(np.uint32) << 16).view(np.float32)


def _split_reference(mps_c, m, n):
    """[n][m][4 blocks][2 planes][16][40] BF16 bits from the [n][m][2][16][32] site tensors."""
    out = np.zeros((n, m, 4, 2, 16, 40), dtype=np.uint16)
    for s in range(2):
        for t in range(2):
            blk = mps_c[:, :, s, :, 16 * t:16 * t + 16]       # [k][i][p = j][a]: A_s[t][a][p]
            x = np.concatenate([blk.real, blk.imag], axis=-1).astype(np.float32)  # row p: Re, Im over a
            hi = _bf16_rne(x)
            lo = _bf16_rne(x - _bf16_value(hi))
            out[:, :, 2 * s + t, 0, :, :32] = hi
            out[:, :, 2 * s + t, 1, :, :32] = lo
    return out


def test_split_operands_match_their_definition(dk):
    dualk, ctx, torch = dk
    from paper_2602_01330_gb300 import synthetic
    x = synthetic.fmnist_like(37, 0, 24)["x_train"]
    mps = dualk.mps_build(ctx, torch.from_numpy(x).cuda(), dualk.FeatureMap(reps=5, chi_max=32))
    ops = mps.split_for(ctx)
    torch.cuda.synchronize()
    got = ops.cpu().numpy().view(np.uint16).reshape(mps.n, mps.m, 4, 2, 16, 40)
    ref = _split_reference(mps.complex_view().cpu().numpy(), mps.m, mps.n)
    assert np.array_equal(got, ref)
    assert mps.split_for(ctx) is ops  # made once


@pytest.mark.parametrize("m_rows,m_cols,d", [(37, 37, 24), (13, 29, 40)])
def test_gram_on_split_operands_is_bit_identical(dk, m_rows, m_cols, d):
    dualk, ctx, torch = dk
    from paper_2602_01330_gb300 import synthetic
    data = synthetic.fmnist_like(m_cols, m_rows, d)
    fm = dualk.FeatureMap(reps=5, chi_max=32)
    cols = dualk.mps_build(ctx, torch.from_numpy(data["x_train"]).cuda(), fm)
    rows = cols if m_rows == m_cols else dualk.mps_build(ctx, torch.from_numpy(data["x_test"]).cuda(), fm)
    prec = dualk.DK_PREC_BF16X3
    symmetric = rows is cols
    split = dualk.gram_tile(ctx, rows, cols, w=0.5, symmetric=symmetric, prec=prec, refine=None)
    direct = dualk._gram_operands
    try:  # the same call on the complex64 tensors
        dualk._gram_operands = lambda c, mp, p, s=None: (mp.data, mp.dtype)
        whole = dualk.gram_tile(ctx, rows, cols, w=0.5, symmetric=symmetric, prec=prec, refine=None)
    finally:
        dualk._gram_operands = direct
    torch.cuda.synchronize()
    for key in ("k", "kq", "kc", "logkq"):
        assert torch.equal(split[key], whole[key]), key
    if symmetric:
        assert torch.all(torch.diagonal(split["kq"]) == 1.0)
    ctx.sync_status()


@pytest.mark.parametrize("m,d,row0,nrows,col0,ncols", [(23, 3, 5, 11, 3, 17), (9, 2, 0, 9, 2, 5), (41, 7, 37, 4, 0, 41)])
def test_split_operands_on_sub_blocks(dk, m, d, row0, nrows, col0, ncols):
    """Rectangular sub-blocks at offsets, ragged against the 4 x 4 pair tiles, short chains:
    the split-operand Gram gives the bits of the complex64 one."""
    dualk, ctx, torch = dk
    from paper_2602_01330_gb300 import synthetic
    x = synthetic.uniform_angles(m, d, seed=m + d)
    mps = dualk.mps_build(ctx, torch.from_numpy(x.astype(np.float32)).cuda(), dualk.FeatureMap(reps=5, chi_max=32))
    prec = dualk.DK_PREC_BF16X3
    kw = dict(row0=row0, nrows=nrows, col0=col0, ncols=ncols, w=0.25, prec=prec, refine=None)
    split = dualk.gram_tile(ctx, mps, mps, **kw)
    direct = dualk._gram_operands
    try:
        dualk._gram_operands = lambda c, mp, p, s=None: (mp.data, mp.dtype)
        whole = dualk.gram_tile(ctx, mps, mps, **kw)
    finally:
        dualk._gram_operands = direct
    torch.cuda.synchronize()
    for key in ("k", "kq", "kc", "logkq"):
        assert torch.equal(split[key], whole[key]), key
    kq = split["kq"].cpu().numpy()
    assert np.all(np.isfinite(kq)) and np.all(kq >= 0.0) and np.all(kq <= 1.0 + 1e-4)
    ctx.sync_status()


def test_split_rejections(dk):
    dualk, ctx, torch = dk
    from paper_2602_01330_gb300 import synthetic
    lib = dualk._lib()
    x = synthetic.fmnist_like(4, 0, 12)["x_train"]
    mps = dualk.mps_build(ctx, torch.from_numpy(x).cuda(), dualk.FeatureMap(reps=5, chi_max=32))
    need = int(lib.dk_mps_bytes(mps.m, mps.n, 32, dualk.DK_SPLIT_BF16))
    buf = torch.empty(need, dtype=torch.uint8, device="cuda")
    assert lib.dk_mps_split32(ctx.handle, dualk._ptr(mps.data), mps.m, mps.n, dualk._ptr(buf), need - 16,
                              None) == 5  # DK_ERR_WORKSPACE
    assert lib.dk_mps_split32(ctx.handle, dualk._ptr(mps.data), mps.m, mps.n, dualk._ptr(buf[1:]), need - 16,
                              None) == 1  # misaligned
    # a sweep refines from the complex64 tensors, so it does not take split operands
    out = torch.empty((mps.m, mps.m), dtype=torch.float32, device="cuda")
    item = dualk._SweepItem()
    item.mps = buf.data_ptr()
    item.log_norm = mps.log_norm.data_ptr()
    item.kq = out.data_ptr()
    item.ld, item.m, item.n = mps.m, mps.m, mps.n
    items = (dualk._SweepItem * 1)(item)
    assert lib.dk_gram_sweep(ctx.handle, items, 1, 32, dualk.DK_SPLIT_BF16, dualk.DK_PREC_BF16X3,
                             ctypes.c_float(1.0), 0, None, 0, None) == 2  # DK_ERR_UNSUPPORTED
