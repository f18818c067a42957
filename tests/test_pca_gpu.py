"""GPU pre-processing (dk_pca_fit / dk_pca_transform) against the pre-processing oracle.

Tolerance (written here, used below): the GPU works in FP32 (covariance, Jacobi rotations),
the oracle in FP64. With a well separated spectrum every eigenvalue agrees to 1e-4 relative
(plus 1e-6 absolute), every component to |<v, v_ref>| >= 1 - 1e-4 with the same sign, and the
scaled features (range pi) to 2e-3; the Jacobi sweeps leave an off-diagonal norm below 1e-5.
On raw synthetic images, whose spectrum has a few large (class template) eigenvalues above a
near-degenerate noise floor, only the leading 8 components are compared (the rest are not
unique), with 1e-3, and the eigenvalue sum against the covariance trace."""
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


def _spectrum_data(seed, m, p):
    rng = np.random.Generator(np.random.PCG64(seed))
    basis = np.linalg.qr(rng.normal(size=(p, p)))[0]
    spectrum = np.geomspace(4.0, 0.05, p)
    x = rng.normal(size=(m, p)) * np.sqrt(spectrum) @ basis.T + rng.normal(size=p) * 3
    return x.astype(np.float32)


@pytest.mark.parametrize("p", [64, 63])
def test_pca_matches_oracle_separated_spectrum(dk, p):
    dualk, ctx, torch = dk
    from oracle import preprocess as pp
    x = _spectrum_data(p, 400, p)
    xt = _spectrum_data(p + 1, 50, p)
    model = dualk.pca_fit(ctx, torch.from_numpy(x).cuda(), p, sweeps=10)
    ftr = dualk.pca_transform(ctx, torch.from_numpy(x).cuda(), model, fit_range=True)
    fte = dualk.pca_transform(ctx, torch.from_numpy(xt).cuda(), model, fit_range=False)
    torch.cuda.synchronize()
    mean, scale, comps, w = pp.pca_fit(x, p)
    assert model["off_norm"].item() < 1e-5
    np.testing.assert_allclose(model["mean"].cpu().numpy(), mean, rtol=1e-5, atol=1e-5)
    np.testing.assert_allclose(model["scale"].cpu().numpy(), scale, rtol=1e-5)
    np.testing.assert_allclose(model["eigenvalues"].cpu().numpy(), w, rtol=1e-4, atol=1e-6)
    dots = np.sum(model["components"].cpu().numpy().astype(np.float64) * comps, axis=1)
    assert np.all(dots >= 1 - 1e-4)
    y = pp.project(x, mean, scale, comps)
    lo, hi = pp.minmax_fit(y)
    np.testing.assert_allclose(ftr.cpu().numpy(), pp.minmax_apply(y, lo, hi), atol=2e-3)
    np.testing.assert_allclose(fte.cpu().numpy(), pp.minmax_apply(pp.project(xt, mean, scale, comps), lo, hi),
                               atol=2e-3)
    np.testing.assert_allclose(model["lo"].cpu().numpy(), lo, rtol=1e-4, atol=1e-4)
    np.testing.assert_allclose(model["hi"].cpu().numpy(), hi, rtol=1e-4, atol=1e-4)
    ctx.sync_status()


def test_pca_raw_images_leading_components(dk):
    """600 raw 784-pixel synthetic images."""
    dualk, ctx, torch = dk
    from oracle import preprocess as pp
    from paper_2602_01330_gb300 import synthetic
    x, _ = synthetic.images(600, 1, synthetic.SEED_TEMPLATES)
    x = x.astype(np.float32)
    model = dualk.pca_fit(ctx, torch.from_numpy(x).cuda(), 784, sweeps=10)
    torch.cuda.synchronize()
    mean, scale, comps, w = pp.pca_fit(x, 784)
    assert model["off_norm"].item() < 1e-5
    ev = model["eigenvalues"].cpu().numpy().astype(np.float64)
    np.testing.assert_allclose(ev[:8], w[:8], rtol=1e-3)
    assert ev.sum() == pytest.approx(w.sum(), rel=1e-4)
    dots = np.sum(model["components"].cpu().numpy()[:8].astype(np.float64) * comps[:8], axis=1)
    assert np.all(dots >= 1 - 1e-3)
    c = model["components"].cpu().numpy().astype(np.float64)
    np.testing.assert_allclose(c @ c.T, np.eye(784), atol=1e-4)
    ctx.sync_status()


def test_pca_workspace_checked(dk):
    dualk, ctx, torch = dk
    x = torch.rand(10, 8, device="cuda")
    small = torch.empty(64, dtype=torch.uint8, device="cuda")
    outs = [torch.empty(n, device="cuda") for n in (8, 8, 16, 2, 1)]
    st = dualk._lib().dk_pca_fit(ctx.handle, dualk._ptr(x), 10, 8, 2, 4, dualk._ptr(small), 64,
                                 *[dualk._ptr(t) for t in outs], dualk._stream(None))
    assert st == 5  # DK_ERR_WORKSPACE
    assert dualk._lib().dk_pca_workspace_bytes(1) == 0
    assert dualk._lib().dk_pca_workspace_bytes(dualk.PCA_MAX_FEATURES + 1) == 0


def test_preprocessor_leading_features(dk):
    """One fit to 32 components serves every n <= 32: the leading 8 of it give exactly the
    features of a fit to 8 (the Jacobi sweeps diagonalise the whole matrix either way), the
    training columns span [0, pi], and against the oracle every feature agrees within the
    bound its component's error implies: |dy| <= max|z| * |v - v_ref| rescaled to [0, pi],
    with |v - v_ref| = sqrt(2 (1 - <v, v_ref>)), plus 2e-3 of rounding."""
    dualk, ctx, torch = dk
    from oracle import preprocess as pp
    from paper_2602_01330_gb300 import synthetic
    from paper_2602_01330_gb300.preprocess import PCAPreprocessor
    xr, _ = synthetic.images(500, synthetic.SEED_TRAIN)
    xs, _ = synthetic.images(100, synthetic.SEED_TEST)
    xr, xs = xr.astype(np.float32), xs.astype(np.float32)
    gr, gs = torch.from_numpy(xr).cuda(), torch.from_numpy(xs).cuda()
    pre = PCAPreprocessor(ctx, k_max=32).fit(gr)
    ftr, fte = pre.features(gr, gs, 8)
    direct = dualk.pca_fit(ctx, gr, 8, sweeps=10)
    dtr = dualk.pca_transform(ctx, gr, direct, fit_range=True)
    torch.cuda.synchronize()
    assert torch.equal(ftr, dtr)
    f = ftr.cpu().numpy()
    np.testing.assert_allclose(f.min(axis=0), 0.0, atol=1e-6)
    np.testing.assert_allclose(f.max(axis=0), np.pi, rtol=1e-6)
    mean, scale, comps, _ = pp.pca_fit(xr, 8)
    y = pp.project(xr, mean, scale, comps)
    lo, hi = pp.minmax_fit(y)
    v = pre.model["components"][:8].cpu().numpy().astype(np.float64)
    dv = np.sqrt(np.maximum(2.0 * (1.0 - np.sum(v * comps, axis=1)), 0.0))
    znorm = max(np.linalg.norm((xr - mean) / scale, axis=1).max(), np.linalg.norm((xs - mean) / scale, axis=1).max())
    tol = znorm * dv * np.pi / (hi - lo) + 2e-3
    assert np.all(np.abs(f - pp.minmax_apply(y, lo, hi)) <= tol)
    ref_te = pp.minmax_apply(pp.project(xs, mean, scale, comps), lo, hi)
    assert np.all(np.abs(fte.cpu().numpy() - ref_te) <= tol)
    ctx.sync_status()


def test_pipeline_on_pca_features(dk):
    """The §II-D workflow from raw images: GPU pre-processing to 16 components, MPS, Gram,
    cross-validation, fit, test predictions. On the synthetic classes it must beat chance
    (0.1) by far; the paper's accuracies are not a target on synthetic data."""
    dualk, ctx, torch = dk
    from paper_2602_01330_gb300 import svm
    out = svm.run_pipeline(ctx, n_train=300, n_test=100, d=16, Cs=(1.0, 10.0), ws=(0.5, 1.0), features="pca")
    assert out["preprocess_ms"] is not None and out["preprocess_ms"] > 0
    assert out["test_accuracy"] > 0.5
    ctx.sync_status()
