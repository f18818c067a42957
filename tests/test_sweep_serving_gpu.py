"""GPU: the graph-captured feature-dimension sweep and the continuous-batching server.

Tolerance as in test_parity_gpu: |dK| <= 1e-6 against the FP64 oracle.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL_K = 1e-6


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_2602_01330_gb300 import build, dualk
    build.build()
    ctx = dualk.Context(0)
    yield dualk, ctx, torch
    ctx.close()


def test_sweep_graph_equals_eager_and_oracle(env):
    dualk, ctx, torch = env
    from oracle import gram, mps
    from paper_2602_01330_gb300 import synthetic
    from paper_2602_01330_gb300.sweep import Autotuner, GramSweep
    dims = (2, 5, 16, 64)
    feats = {d: synthetic.fmnist_like(90, 0, d)["x_train"] for d in dims}
    tuner = Autotuner(ctx, probe_sites=8, reps=1)
    sw = GramSweep(ctx, feats, dualk.FeatureMap(reps=2, chi_max=4), w=0.5, autotuner=tuner)
    sw.run_eager()
    torch.cuda.synchronize()
    eager = {mt.d: {k: v.clone() for k, v in mt.out.items()} for mt in sw.mats}
    for mt in sw.mats:
        for v in mt.out.values():
            v.fill_(-1.0)
    sw.capture()
    sw.replay()
    torch.cuda.synchronize()
    ctx.sync_status()
    for mt in sw.mats:
        for k in mt.out:
            assert torch.equal(mt.out[k], eager[mt.d][k]), (mt.d, k)
    # the library's own sweep call (dk_gram_sweep), recorded into a graph and replayed
    side = torch.cuda.Stream()
    for rnd in range(2):
        for mt in sw.mats:
            for v in mt.out.values():
                v.fill_(-1.0)
        torch.cuda.synchronize()
        with torch.cuda.stream(side):
            sw.run_native(graph=True, stream=side)
        side.synchronize()
        for mt in sw.mats:
            for k in mt.out:
                assert torch.equal(mt.out[k], eager[mt.d][k]), (rnd, mt.d, k)
    ctx.sync_status()
    for mt in sw.mats:
        x = feats[mt.d].astype(np.float64)
        sites, _ = mps.build_mps(x, 2)
        kq, _ = gram.gram_from_mps(sites, sites)
        k_ref = gram.dual_kernel(kq, gram.rbf(x, x, 1.0 / mt.d), 0.5)
        assert np.max(np.abs(mt.out["k"].cpu().numpy() - k_ref)) <= TOL_K
        assert 1 <= mt.cfg <= dualk.gram_config_count()


def test_serving_same_alone_and_in_mix(env):
    dualk, ctx, torch = env
    from oracle import gram, mps
    from paper_2602_01330_gb300 import synthetic
    from paper_2602_01330_gb300.serving import KernelServer, latency_stats, poisson_requests
    dims = (8, 32, 96)
    train = {n: synthetic.fmnist_like(150, 0, n)["x_train"] for n in dims}
    pool = {n: synthetic.fmnist_like(8, 64, n)["x_test"] for n in dims}
    srv = KernelServer(ctx, train, dualk.FeatureMap(reps=2, chi_max=4), w=0.5, slots=4, reserve_bytes=1 << 28)
    rng = np.random.Generator(np.random.PCG64(4))
    reqs = poisson_requests(rng, 24, 2000.0, dims, pool, b_max=20)
    srv.run(reqs)
    st = latency_stats(reqs)
    assert st["served"] == 24 and st["rejected"] == 0
    for r in reqs[:6]:
        assert np.array_equal(srv.solve_alone(r), r.result)
    # a burst: every request waits at once, so launches of all three qubit counts (each a
    # merged batch) are on the device together, on their own streams
    burst = poisson_requests(rng, 24, 1e9, dims, pool, b_max=20)
    srv.max_launches_in_flight = srv.max_in_flight = 0
    srv.run(burst)
    assert srv.max_launches_in_flight >= 2 and srv.max_in_flight >= 3
    for r in burst[:6]:
        assert np.array_equal(srv.solve_alone(r), r.result)
    for r in reqs[:3]:
        xt = train[r.n].astype(np.float64)
        xs = r.x.astype(np.float64)
        a, _ = mps.build_mps(xs, 2)
        b, _ = mps.build_mps(xt, 2)
        kq, _ = gram.gram_from_mps(a, b)
        ref = gram.dual_kernel(kq, gram.rbf(xs, xt, 1.0 / r.n), 0.5)
        assert np.max(np.abs(r.result - ref)) <= TOL_K
