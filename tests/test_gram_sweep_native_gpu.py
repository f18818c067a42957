"""dk_gram_sweep: the feature-dimension sweep as one native call, eager or replayed from a
CUDA graph kept by the context.

Every item must be bit-identical to the same Gram computed alone by dk_gram_tile (same tile
shape, same arithmetic), both eagerly and from the graph; a replay must read the buffers'
current contents (new inputs written in place give the new results, not stale ones); the
graph cache must survive eviction; bad arguments are refused."""
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


def _items(dualk, torch, ctx, specs, fm, seed=0, tiles=None):
    from paper_2602_01330_gb300 import synthetic
    items = []
    for t, (m, d) in enumerate(specs):
        x = torch.from_numpy(synthetic.uniform_angles(m, d, seed + t).astype(np.float32)).cuda()
        mps = dualk.mps_build(ctx, x, fm)
        out = {k: torch.full((m, m), -7.0, device="cuda") for k in ("k", "kq", "kc", "logkq")}
        items.append((mps, out, 0 if tiles is None else tiles[t]))
    torch.cuda.synchronize()  # the builds and fills ran on the current stream; sweeps may use another
    return items


def _alone(dualk, ctx, mps, tile, w):
    ctx.set_gram_config(tile)
    try:
        return dualk.gram(ctx, mps, w=w)
    finally:
        ctx.set_gram_config(0)


def _assert_same(torch, items, refs):
    for (mps, out, _), ref in zip(items, refs):
        for key in ("k", "kq", "kc", "logkq"):
            assert torch.equal(out[key], ref[key]), (mps.n, key)


def test_native_sweep_eager_and_graph_match_single_grams(dk):
    dualk, ctx, torch = dk
    fm = dualk.FeatureMap(reps=2, chi_max=4)
    items = _items(dualk, torch, ctx, [(30, 2), (50, 7), (70, 16), (40, 64), (33, 200)], fm,
                   tiles=[0, 14, 17, 0, 19])
    refs = [_alone(dualk, ctx, mps, tile, 0.5) for mps, _, tile in items]
    dualk.gram_sweep(ctx, items, w=0.5)
    torch.cuda.synchronize()
    _assert_same(torch, items, refs)
    side = torch.cuda.Stream()
    for _, out, _ in items:
        for v in out.values():
            v.fill_(-7.0)
    torch.cuda.synchronize()
    for _ in range(3):  # record, then replay twice
        dualk.gram_sweep(ctx, items, w=0.5, graph=True, stream=side)
        side.synchronize()
        _assert_same(torch, items, refs)
    ctx.sync_status()


def test_graph_replay_reads_current_inputs(dk):
    """New features written into the same buffers, MPS rebuilt in place: the replayed graph
    gives the new Gram matrices."""
    dualk, ctx, torch = dk
    from paper_2602_01330_gb300 import synthetic
    fm = dualk.FeatureMap(reps=2, chi_max=4)
    items = _items(dualk, torch, ctx, [(40, 12), (60, 30)], fm, seed=10)
    side = torch.cuda.Stream()
    dualk.gram_sweep(ctx, items, w=0.25, graph=True, stream=side)
    side.synchronize()
    for t, (mps, out, _) in enumerate(items):
        mps.x.copy_(torch.from_numpy(synthetic.uniform_angles(mps.m, mps.n, 99 + t).astype(np.float32)))
        dualk.mps_build(ctx, mps.x, fm, out=mps.data, bond=mps.bond_dims, log_norm=mps.log_norm)
    torch.cuda.synchronize()
    refs = [_alone(dualk, ctx, mps, 0, 0.25) for mps, _, _ in items]
    dualk.gram_sweep(ctx, items, w=0.25, graph=True, stream=side)
    side.synchronize()
    _assert_same(torch, items, refs)
    ctx.sync_status()


def test_graph_cache_eviction_and_bond8(dk):
    """More distinct sweeps than the cache holds (here by the mix weight), then the newest
    again; a bond-8 sweep (reps = 3) through the same call."""
    dualk, ctx, torch = dk
    side = torch.cuda.Stream()
    items = _items(dualk, torch, ctx, [(20, 5)], dualk.FeatureMap(reps=2, chi_max=4), seed=20)
    ws = [i / 20.0 for i in range(20)]
    for w in ws:
        dualk.gram_sweep(ctx, items, w=w, graph=True, stream=side)
    dualk.gram_sweep(ctx, items, w=ws[-1], graph=True, stream=side)
    side.synchronize()
    _assert_same(torch, items, [_alone(dualk, ctx, items[0][0], 0, ws[-1])])
    torch.cuda.synchronize()
    items8 = _items(dualk, torch, ctx, [(24, 9), (31, 20)], dualk.FeatureMap(reps=3, chi_max=8), seed=30)
    refs8 = [_alone(dualk, ctx, mps, 0, 0.5) for mps, _, _ in items8]
    torch.cuda.synchronize()
    dualk.gram_sweep(ctx, items8, w=0.5, graph=True, stream=side)
    dualk.gram_sweep(ctx, items8, w=0.5, graph=True, stream=side)
    side.synchronize()
    _assert_same(torch, items8, refs8)
    ctx.sync_status()


def test_native_sweep_errors(dk):
    dualk, ctx, torch = dk
    items = _items(dualk, torch, ctx, [(20, 5)], dualk.FeatureMap(reps=2, chi_max=4), seed=40)
    default = torch.cuda.default_stream()
    with pytest.raises(dualk.DualKError):  # graphs need a non-default stream
        dualk.gram_sweep(ctx, items, graph=True, stream=default)
    with pytest.raises(dualk.DualKError):  # tile shape out of range
        dualk.gram_sweep(ctx, [(items[0][0], items[0][1], 999)])
    ctx.sync_status()
