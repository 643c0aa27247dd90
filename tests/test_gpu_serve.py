"""Serving: requests of many models arriving open-loop, batched continuously, with models spilled
and re-admitted under an HBM budget.  Each model's final layers and each query's result must equal
(a) the plain definition -- the CPU oracle applying that model's requests alone, in arrival order
(Section 4.3.1 / Fig. 3 per request): bit-exact, except lasso texels the oracle flags as ambiguous,
whose differences must stay below 1e-5 of the texels touched -- and (b) the library's own
single-stroke calls applied alone, bit for bit (the same result alone and in the mix)."""
import numpy as np
import pytest
import torch

import synth
from serve_replay import replay_alone, replay_oracle

pytestmark = pytest.mark.gpu

from paper_2501_14807_gb300 import lcl, serve  # noqa: E402


def served_models(n, seed=300):
    out, pools = [], []
    for i in range(n):
        kind = ["vessel", "sphere", "torus"][i % 3]
        bm = synth.batch_model(kind, [4000, 12000, 30000][i % 3], seed + i, n_sphere=32, n_lasso=8, depth_side=256)
        side = 256 if bm.mesh.n_tri < 10000 else 512
        out.append(serve.ServedModel(bm.mesh, side, bm.cams, n_layers=2))
        pools.append(bm)
    return out, pools


def trace(pools, rate, duration, seed):
    def sphere_of(m, rng):
        st = pools[m].strokes
        k = int(rng.integers(0, len(st.radius)))
        return (st.centre[k], float(st.radius[k]), int(rng.integers(1, 256)))

    def lasso_of(m, rng):
        L = pools[m].lassos[int(rng.integers(0, len(pools[m].lassos)))]
        return (L.cam, L.poly, int(rng.integers(1, 256)))

    return serve.poisson_requests(len(pools), rate, duration, seed, sphere_of=sphere_of, lasso_of=lasso_of)


@pytest.mark.parametrize("layer_pool", [False, True])
def test_served_results_equal_requests_applied_alone(layer_pool):
    models, pools = served_models(8)
    probe = serve.Server(models[:1], hbm_budget_bytes=1 << 40, layer_pool=layer_pool)
    one = probe.slots[0].bytes
    probe.close()
    del probe
    torch.cuda.empty_cache()
    srv = serve.Server(models, hbm_budget_bytes=int(3.5 * one), layer_pool=layer_pool)   # only a few models fit
    reqs = trace(pools, rate=4000.0, duration=0.3, seed=11)
    srv.run(reqs)
    assert all(r.t_done >= r.t_arrive for r in reqs)
    assert srv.spills > 0 and srv.admissions > 0 and srv.epochs > 1
    oracle_layers, oracle_results = replay_oracle(models, reqs)
    for mi, (ls, amb, touched) in oracle_layers.items():
        got = srv.layers_of(mi)
        for li, (exp, g) in enumerate(zip(ls, got)):
            diff = g.cpu().numpy() != exp
            assert not (diff & ~amb[li]).any(), f"model {mi} layer {li}: differs from the oracle off ambiguous texels"
            assert diff.sum() <= 1e-5 * max(touched[li], 1), f"model {mi} layer {li}: too many ambiguous differences"
    for i, r in enumerate(reqs):
        if r.kind == serve.QUERY:
            ec, ea, n_amb = oracle_results[i]
            if n_amb == 0:
                assert np.array_equal(r.result[0], ec) and np.array_equal(r.result[1], ea), f"query {i} differs"
            else:   # each differing texel moves one count from one label to another
                assert np.abs(r.result[0].astype(np.int64) - ec.astype(np.int64)).sum() <= 2 * n_amb
    alone_layers, alone_results = replay_alone(models, reqs)
    for mi, ls in alone_layers.items():
        got = srv.layers_of(mi)
        for a, b in zip(ls, got):
            assert torch.equal(a, b), f"model {mi}: served layers differ from the requests applied alone"
    n_q = 0
    for i, r in enumerate(reqs):
        if r.kind == serve.QUERY:
            n_q += 1
            ec, ea = alone_results[i]
            assert np.array_equal(r.result[0], ec) and np.array_equal(r.result[1], ea)
    assert n_q > 0
    if layer_pool:
        st = srv.pool.stats()
        resident_layers = sum(len(sl.layers) for sl in srv.slots if sl.resident)
        assert st["layers"] == resident_layers < sum(m.n_layers for m in models)
    srv.close()


@pytest.mark.parametrize("layer_pool", [False, True])
def test_models_spilled_as_they_are_built_keep_complete_depth_maps(layer_pool):
    """A model over the budget is spilled right after it is built: the copy to its host image runs on
    the copy stream and must wait for the depth maps rendered on the build's stream (an image taken
    too early holds a partly rendered map, and every later lasso on the model reads it)."""
    models, _ = served_models(6)
    probe = serve.Server(models[:1], hbm_budget_bytes=1 << 40, layer_pool=layer_pool)
    one = probe.slots[0].bytes
    probe.close()
    del probe
    torch.cuda.empty_cache()
    srv = serve.Server(models, hbm_budget_bytes=one, layer_pool=layer_pool)   # one model fits
    assert srv.spills >= len(models) - 1
    dev = torch.device("cuda")
    for spec, sl in zip(models, srv.slots):
        if sl.resident:
            continue
        mesh = lcl.Mesh.from_host(spec.mesh, dev)
        a = lcl.Atlas(spec.side, spec.side, spec.tile, spec.mesh.n_tri, dev)
        lcl.lcl_atlas_build(mesh, a)
        _, _, _, offs_d, _ = sl.lay
        for o, c in zip(offs_d, spec.cams):
            d = torch.empty((c.height, c.width), dtype=torch.float32, device=dev)
            lcl.lcl_depth_render(mesh, a, lcl.lcl_camera_from_vp(a, c.vp, c.width, c.height), d)
            stored = sl.host["image"][o:o + 4 * c.width * c.height].view(torch.float32).view(c.height, c.width)
            assert torch.equal(stored.view(torch.int32), d.cpu().view(torch.int32))
    srv.close()
