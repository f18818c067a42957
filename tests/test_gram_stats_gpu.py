"""dk_gram_stats (concentration diagnostics) against NumPy on the same float32 Gram outputs.

The sums are FP64 on both sides, in different orders: means and variances agree to 1e-9
relative. The symmetric form counts each pair of distinct samples once (the strict upper
triangle); the rectangular form counts every entry. On the synthetic set the mean
off-diagonal K_q falls as the qubit count grows (d = 8, 32, 128), the concentration the
diagnostic is there to show."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _np_stats(kq, lkq):
    lf = lkq[np.isfinite(lkq)].astype(np.float64)
    k = kq.astype(np.float64)
    return {"pairs": k.size, "kq_mean": k.mean(), "kq_var": k.var(),
            "finite_log_pairs": lf.size, "logkq_mean": lf.mean(), "logkq_var": lf.var()}


def _close(a, b):
    for key in ("pairs", "finite_log_pairs"):
        assert a[key] == b[key]
    for key in ("kq_mean", "kq_var", "logkq_mean", "logkq_var"):
        assert a[key] == pytest.approx(b[key], rel=1e-9, abs=1e-300)


def test_stats_match_numpy_and_show_concentration():
    import torch
    from paper_2602_01330_gb300 import build, dualk, synthetic
    build.build()
    ctx = dualk.Context(0)
    fm = dualk.FeatureMap(reps=2, chi_max=4)
    means = []
    for d in (8, 32, 128):
        data = synthetic.fmnist_like(300, 70, d)
        tr = dualk.mps_build(ctx, torch.from_numpy(data["x_train"]).cuda(), fm)
        te = dualk.mps_build(ctx, torch.from_numpy(data["x_test"]).cuda(), fm)
        g = dualk.gram(ctx, tr, w=1.0, want=("kq", "logkq"))
        r = dualk.dual_kernel_rows(ctx, te, tr, w=1.0, want=("kq", "logkq"))
        s = dualk.gram_stats(ctx, g["kq"], g["logkq"], symmetric=True)
        sr = dualk.gram_stats(ctx, r["kq"], r["logkq"], symmetric=False)
        kq, lkq = g["kq"].cpu().numpy(), g["logkq"].cpu().numpy()
        iu = np.triu_indices(300, 1)
        _close(s, _np_stats(kq[iu], lkq[iu]))
        _close(sr, _np_stats(r["kq"].cpu().numpy().ravel(), r["logkq"].cpu().numpy().ravel()))
        # a second call on the same output buffer restarts from zero
        again = dualk.gram_stats(ctx, g["kq"], g["logkq"], symmetric=True)
        _close(again, s)  # (the per-CTA partials are added atomically, in no fixed order)
        means.append(s["logkq_mean"])
    assert means[0] > means[1] > means[2]
    with pytest.raises(dualk.DualKError) as e:
        dualk.gram_stats(ctx, r["kq"], None, symmetric=True)  # a symmetric block must be square
    assert e.value.status == 1
    ctx.sync_status()
    ctx.close()
