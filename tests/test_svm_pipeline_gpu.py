"""The §II-D workflow through the library: the GPU Gram and rows of a small synthetic set,
5-fold cross-validation over C x w in one training and one prediction launch, the final fit
and the test predictions, each checked against the SVM oracle trained on the same kernel
values (copied from the GPU). Held-out and test predictions must equal the oracle's wherever
every class pair's oracle decision value exceeds 1e-3 in magnitude (at the SVM solver's
1e-3 stopping tolerance the two solutions differ by less than that), and the chosen (C, w)
must be one whose oracle accuracy is within one held-out sample per fold of the best."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_cv_fit_predict_against_oracle():
    import torch
    from oracle import svm as osvm
    from paper_2602_01330_gb300 import build, dualk, svm, synthetic
    build.build()
    ctx = dualk.Context(0)
    n_tr, n_te, d = 300, 80, 16
    data = synthetic.fmnist_like(n_tr, n_te, d)
    ytr, yte = np.asarray(data["y_train"]), np.asarray(data["y_test"])
    fm = dualk.FeatureMap(reps=2, chi_max=4)
    mtr = dualk.mps_build(ctx, torch.from_numpy(data["x_train"]).cuda(), fm)
    mte = dualk.mps_build(ctx, torch.from_numpy(data["x_test"]).cuda(), fm)
    g = dualk.gram(ctx, mtr, w=1.0, want=("kq", "kc"))
    r = dualk.dual_kernel_rows(ctx, mte, mtr, w=1.0, want=("kq", "kc"))
    clf = svm.DualKernelSVM(ctx, 10, Cs=(1.0, 10.0), ws=(0.5, 1.0), tol=1e-5)
    cv = clf.cross_validate(g["kq"], g["kc"], ytr)
    kq, kc = g["kq"].cpu().numpy(), g["kc"].cpu().numpy()
    kqr, kcr = r["kq"].cpu().numpy(), r["kc"].cpu().numpy()

    def mixed(a, b, w):
        return (np.float32(w) * a + np.float32(1 - w) * b).astype(np.float64)

    ref_acc = {}
    for j, (f, C, w) in enumerate(cv.job_list):
        tr, va = np.flatnonzero(cv.folds != f), np.flatnonzero(cv.folds == f)
        K = mixed(kq, kc, w)
        coef, bias = osvm.ovo_train(K[np.ix_(tr, tr)], ytr[tr], 10, C, tol=1e-6)
        dec = osvm.ovo_decision(K[np.ix_(va, tr)], coef, bias)
        ref = osvm.ovo_vote(dec, 10)
        clear = np.min(np.abs(dec), axis=1) > 1e-3
        np.testing.assert_array_equal(cv.pred[j, :va.size][clear], ref[clear])
        ref_acc.setdefault((C, w), []).append(np.mean(ref == ytr[va]))
    best_ref = max(np.mean(v) for v in ref_acc.values())
    assert np.mean(ref_acc[cv.best]) >= best_ref - 1.0 / 60
    C, w = cv.best
    clf.fit(g["kq"], g["kc"], ytr, C, w)
    out = clf.predict(r["kq"], r["kc"], want_decision=True)
    pred = out["pred"][0].cpu().numpy()
    coef, bias = osvm.ovo_train(mixed(kq, kc, w), ytr, 10, C, tol=1e-6)
    dec = osvm.ovo_decision(mixed(kqr, kcr, w), coef, bias)
    clear = np.min(np.abs(dec), axis=1) > 1e-3
    assert clear.sum() > n_te // 2
    np.testing.assert_array_equal(pred[clear], osvm.ovo_vote(dec, 10)[clear])
    ctx.sync_status()
    ctx.close()
