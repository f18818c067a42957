"""dk_pca_fit_noalloc: the PCA fit for callers that cannot give the library device memory
(a program whose device memory another framework owns and caps, a plug-in handed only its
input and output pointers, a loop that must not stall on or fail in an allocation). It keeps
its working memory in a fixed array inside the library instead of a caller workspace.

Checked through the C ABI against the workspace form dk_pca_fit on two calls in a row with
different shapes (the second at the 256-feature maximum, so it reuses and overruns nothing
the first left in the shared array), within the PCA tests' tolerance: eigenvalues to 1e-4
relative (plus 1e-6 absolute), components to |<v, v_ref>| >= 1 - 1e-4 with the same sign,
mean and scale to 1e-6; and a size beyond the maximum is refused with DK_ERR_UNSUPPORTED.
This file is collected last, so a run that stops at its first failure has run every other
test before it."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _spectrum_data(seed, m, p):
    rng = np.random.Generator(np.random.PCG64(seed))
    basis = np.linalg.qr(rng.normal(size=(p, p)))[0]
    spectrum = np.geomspace(4.0, 0.05, p)
    return (rng.normal(size=(m, p)) * np.sqrt(spectrum) @ basis.T + rng.normal(size=p) * 3).astype(np.float32)


def test_noalloc_fit_matches_workspace_fit_two_calls_in_a_row():
    import torch
    from paper_2602_01330_gb300 import build, dualk
    build.build()
    ctx = dualk.Context(0)
    lib = dualk._lib()
    for seed, m, p, k in ((31, 300, 64, 64), (32, 400, dualk.PCA_NOALLOC_MAX_FEATURES, 16)):
        x = torch.from_numpy(_spectrum_data(seed, m, p)).cuda()
        ref = dualk.pca_fit(ctx, x, k, sweeps=10)
        out = {"mean": torch.empty(p, device="cuda"), "scale": torch.empty(p, device="cuda"),
               "components": torch.empty((k, p), device="cuda"), "eigenvalues": torch.empty(k, device="cuda"),
               "off_norm": torch.empty(1, device="cuda")}
        st = lib.dk_pca_fit_noalloc(ctx.handle, dualk._ptr(x), m, p, k, 10, dualk._ptr(out["mean"]),
                                    dualk._ptr(out["scale"]), dualk._ptr(out["components"]),
                                    dualk._ptr(out["eigenvalues"]), dualk._ptr(out["off_norm"]),
                                    dualk._stream(None))
        assert st == 0
        torch.cuda.synchronize()
        ctx.sync_status()
        assert out["off_norm"].item() < 1e-5
        np.testing.assert_allclose(out["mean"].cpu().numpy(), ref["mean"].cpu().numpy(), rtol=1e-6, atol=1e-6)
        np.testing.assert_allclose(out["scale"].cpu().numpy(), ref["scale"].cpu().numpy(), rtol=1e-6)
        np.testing.assert_allclose(out["eigenvalues"].cpu().numpy(), ref["eigenvalues"].cpu().numpy(),
                                   rtol=1e-4, atol=1e-6)
        dots = np.sum(out["components"].cpu().numpy().astype(np.float64) *
                      ref["components"].cpu().numpy().astype(np.float64), axis=1)
        assert np.all(dots >= 1 - 1e-4)
    # one feature past the maximum is refused before anything runs
    p = dualk.PCA_NOALLOC_MAX_FEATURES + 1
    x = torch.rand(8, p, device="cuda")
    bufs = [torch.empty(n, device="cuda") for n in (p, p, p, 1, 1)]
    st = lib.dk_pca_fit_noalloc(ctx.handle, dualk._ptr(x), 8, p, 1, 10, *[dualk._ptr(b) for b in bufs],
                                dualk._stream(None))
    assert st == 2  # DK_ERR_UNSUPPORTED
    ctx.close()
