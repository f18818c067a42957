"""GPU parity of the one-against-one SVM (dk_svm_ovo_train / dk_svm_ovo_predict) against the
FP64 oracle (oracle/svm.py) on the same float32 kernel values.

Tolerance (written here, used below). Both solvers stop when the largest KKT violation is
below TOL_SMO = 1e-6, from the same kernel values, so both sit within that gap of the unique
optimum of the dual (Eqs. 1-2). The GPU solution's own KKT violation, evaluated in FP64 by
the oracle, is held to 1e-5; its dual objective to the oracle's within 1e-6 relative; the
decision values (Eq. 5) within 1e-4 absolute; the predicted classes exactly, wherever every
class pair's |f| exceeds 1e-3 (below that a vote may legitimately flip).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL_SMO = 1e-6
TOL_KKT = 1e-5
TOL_OBJ = 1e-6
TOL_DEC = 1e-4
MARGIN = 1e-3


@pytest.fixture(scope="module")
def dk():
    import torch
    from paper_2602_01330_gb300 import build, dualk
    build.build()
    ctx = dualk.Context(0)
    yield dualk, ctx, torch
    ctx.close()


def _blobs(seed, m, n_class, dim=5, spread=1.0):
    rng = np.random.Generator(np.random.PCG64(seed))
    centres = rng.normal(0, 1.4, size=(n_class, dim))
    labels = np.arange(m) % n_class
    rng.shuffle(labels)
    return centres[labels] + rng.normal(0, spread, size=(m, dim)), labels


def _rbf32(x, z, gamma):
    d2 = ((x[:, None, :] - z[None, :, :]) ** 2).sum(-1)
    return np.exp(-gamma * d2).astype(np.float32)


def _dev(torch, a, dt):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=dt)).cuda()


def _check_job(dualk, oracle_svm, K, labels, sel, C, n_class, coef, bias, iters, Krows=None, dec=None):
    """One job: the oracle trained on the samples `sel` of the (float64) kernel K."""
    Kj = K[np.ix_(sel, sel)]
    lj = labels[sel]
    pairs = oracle_svm.class_pairs(n_class)
    for p, (c1, c2) in enumerate(pairs):
        loc = np.flatnonzero((lj == c1) | (lj == c2))
        if loc.size == 0 or np.all(lj[loc] == lj[loc[0]]):
            assert iters[p] == 0 and bias[p] == 0.0 and np.all(coef[p] == 0.0)
            continue
        y = np.where(lj[loc] == c1, 1.0, -1.0)
        Kp = Kj[np.ix_(loc, loc)]
        a_gpu = coef[p, loc].astype(np.float64) * y
        assert iters[p] > 0
        assert np.all(a_gpu >= -1e-7) and np.all(a_gpu <= C * (1 + 1e-6))
        assert oracle_svm.kkt_violation(Kp, y, np.clip(a_gpu, 0, C), C) <= TOL_KKT
        a_ref, b_ref, _ = oracle_svm.smo(Kp, y, C, tol=TOL_SMO)
        o_gpu = oracle_svm.dual_objective(Kp, y, a_gpu)
        o_ref = oracle_svm.dual_objective(Kp, y, a_ref)
        assert abs(o_gpu - o_ref) <= TOL_OBJ * max(1.0, abs(o_ref))
        mask = np.ones(len(sel), dtype=bool)
        mask[loc] = False
        assert np.all(coef[p, :len(sel)][mask] == 0.0)
    if Krows is not None:
        coef_ref, bias_ref = oracle_svm.ovo_train(Kj, lj, n_class, C, tol=TOL_SMO)
        dec_ref = oracle_svm.ovo_decision(Krows, coef_ref, bias_ref)
        assert np.max(np.abs(dec - dec_ref)) <= TOL_DEC
        return dec_ref
    return None


@pytest.mark.parametrize("mix", [False, True])
def test_single_job_matches_oracle(dk, mix):
    """150 training samples in 4 classes (6 binary problems), 40 test samples; an RBF
    kernel, or a 0.3 / 0.7 mix of two RBF kernels of different widths."""
    dualk, ctx, torch = dk
    from oracle import svm as osvm
    x, labels = _blobs(1, 150, 4)
    xt, _ = _blobs(2, 40, 4)
    kq, kqt = _rbf32(x, x, 0.35), _rbf32(xt, x, 0.35)
    kc, kct = _rbf32(x, x, 0.08), _rbf32(xt, x, 0.08)
    w, C = (0.3 if mix else 1.0), 2.0
    K = (np.float32(w) * kq + np.float32(1 - w) * kc if mix else kq).astype(np.float64)
    Kt = (np.float32(w) * kqt + np.float32(1 - w) * kct if mix else kqt).astype(np.float64)
    m = 150
    idx = _dev(torch, np.arange(m)[None, :], np.int32)
    cnt = _dev(torch, [m], np.int32)
    wt, Ct = _dev(torch, [w], np.float32), _dev(torch, [C], np.float32)
    lab = _dev(torch, labels, np.int32)
    model = dualk.svm_ovo_train(ctx, _dev(torch, kq, np.float32), _dev(torch, kc, np.float32) if mix else None,
                                wt, Ct, idx, cnt, lab, 4, tol=TOL_SMO)
    out = dualk.svm_ovo_predict(ctx, _dev(torch, kqt, np.float32), _dev(torch, kct, np.float32) if mix else None,
                                wt, model, 4)
    torch.cuda.synchronize()
    coef = model["coef"].cpu().numpy()[0]
    bias = model["bias"].cpu().numpy()[0]
    iters = model["iters"].cpu().numpy()[0]
    dec = out["decision"].cpu().numpy()[0].astype(np.float64)
    pred = out["pred"].cpu().numpy()[0]
    dec_ref = _check_job(dualk, osvm, K, labels, np.arange(m), C, 4, coef, bias, iters, Kt, dec)
    clear = np.min(np.abs(dec_ref), axis=1) > MARGIN
    assert clear.sum() > 30
    np.testing.assert_array_equal(pred[clear], osvm.ovo_vote(dec_ref, 4)[clear])
    ctx.sync_status()


def test_cross_validation_grid_in_one_launch(dk):
    """5 folds x 2 values of C x 2 mixing weights = 20 jobs in one launch, 240 samples in 3
    classes; every job against the oracle trained on its own fold, and its held-out fold
    classified through the rows / idx lists of dk_svm_ovo_predict."""
    dualk, ctx, torch = dk
    from oracle import svm as osvm
    x, labels = _blobs(5, 240, 3)
    kq, kc = _rbf32(x, x, 0.3), _rbf32(x, x, 0.05)
    rng = np.random.Generator(np.random.PCG64(9))
    fold = rng.permutation(240) % 5
    jobs = [(f, C, w) for f in range(5) for C in (0.5, 4.0) for w in (0.25, 1.0)]
    m_max, r_max = 240, 240
    idx = np.zeros((len(jobs), m_max), np.int32)
    cnt = np.zeros(len(jobs), np.int32)
    rows = np.zeros((len(jobs), r_max), np.int32)
    rcnt = np.zeros(len(jobs), np.int32)
    for j, (f, C, w) in enumerate(jobs):
        tr, va = np.flatnonzero(fold != f), np.flatnonzero(fold == f)
        idx[j, :tr.size], cnt[j] = tr, tr.size
        rows[j, :va.size], rcnt[j] = va, va.size
    wt = _dev(torch, [w for _, _, w in jobs], np.float32)
    Ct = _dev(torch, [C for _, C, _ in jobs], np.float32)
    dq, dc = _dev(torch, kq, np.float32), _dev(torch, kc, np.float32)
    di, dn = _dev(torch, idx, np.int32), _dev(torch, cnt, np.int32)
    model = dualk.svm_ovo_train(ctx, dq, dc, wt, Ct, di, dn, _dev(torch, labels, np.int32), 3, tol=TOL_SMO)
    out = dualk.svm_ovo_predict(ctx, dq, dc, wt, model, 3, rows=_dev(torch, rows, np.int32),
                                row_count=_dev(torch, rcnt, np.int32), idx=di, count=dn)
    torch.cuda.synchronize()
    coef, bias = model["coef"].cpu().numpy(), model["bias"].cpu().numpy()
    iters, dec = model["iters"].cpu().numpy(), out["decision"].cpu().numpy().astype(np.float64)
    pred = out["pred"].cpu().numpy()
    for j, (f, C, w) in enumerate(jobs):
        K = (np.float32(w) * kq + np.float32(1 - w) * kc).astype(np.float64)
        tr, va = idx[j, :cnt[j]], rows[j, :rcnt[j]]
        assert np.all(coef[j][:, cnt[j]:] == 0.0)
        dec_ref = _check_job(dualk, osvm, K, labels, tr, C, 3, coef[j], bias[j], iters[j],
                             K[np.ix_(va, tr)], dec[j, :va.size])
        clear = np.min(np.abs(dec_ref), axis=1) > MARGIN
        np.testing.assert_array_equal(pred[j, :va.size][clear], osvm.ovo_vote(dec_ref, 3)[clear])
        assert np.all(pred[j, va.size:] == -1)  # rows past row_count are not written
    ctx.sync_status()


def test_absent_class_step_limit_and_errors(dk):
    dualk, ctx, torch = dk
    x, labels = _blobs(3, 60, 3)
    kq = _dev(torch, _rbf32(x, x, 0.3), np.float32)
    lab = _dev(torch, labels, np.int32)
    # job 0 has no sample of class 2: its pairs (0,2) and (1,2) are skipped
    no2 = np.flatnonzero(labels != 2).astype(np.int32)
    idx = np.zeros((2, 60), np.int32)
    idx[0, :no2.size] = no2
    idx[1] = np.arange(60)
    cnt = _dev(torch, [no2.size, 60], np.int32)
    w, C = _dev(torch, [1.0, 1.0], np.float32), _dev(torch, [1.0, 1.0], np.float32)
    model = dualk.svm_ovo_train(ctx, kq, None, w, C, _dev(torch, idx, np.int32), cnt, lab, 3, tol=TOL_SMO)
    it = model["iters"].cpu().numpy()
    assert it[0, 0] > 0 and it[0, 1] == 0 and it[0, 2] == 0
    assert np.all(model["coef"].cpu().numpy()[0, 1:] == 0.0) and np.all(model["bias"].cpu().numpy()[0, 1:] == 0.0)
    assert np.all(it[1] > 0)
    # a step limit below what the problem needs is reported as -1
    short = dualk.svm_ovo_train(ctx, kq, None, w, C, _dev(torch, idx, np.int32), cnt, lab, 3, tol=1e-9,
                                max_iter=2)
    assert np.all(short["iters"].cpu().numpy()[1] == -1)
    # host-side argument checks
    one = _dev(torch, np.arange(60)[None, :], np.int32)
    c1 = _dev(torch, [60], np.int32)
    w1, C1 = _dev(torch, [1.0], np.float32), _dev(torch, [1.0], np.float32)
    with pytest.raises(dualk.DualKError) as e:
        dualk.svm_ovo_train(ctx, kq, None, w1, C1, one, c1, lab, 33)
    assert e.value.status == 2
    with pytest.raises(dualk.DualKError) as e:
        dualk.svm_ovo_train(ctx, kq, None, w1, C1, one, c1, lab, 3, tol=0.0)
    assert e.value.status == 1
    big = _dev(torch, np.zeros((1, dualk.SVM_MAX_SAMPLES + 1)), np.int32)
    with pytest.raises(dualk.DualKError) as e:
        dualk.svm_ovo_train(ctx, kq, None, w1, C1, big, c1, lab, 3)
    assert e.value.status == 2
    ctx.sync_status()
