"""The native request server (lcl_serve_*: admission by HBM footprint, per-model FIFO queues,
continuous batching, queries, all in a host thread of the library): the same open-loop trace as the
Python scheduler's test, with only a few models fitting the arena, so models are spilled and
re-admitted.  Each model's final layers and each query's result must equal the CPU oracle applying
that model's requests alone in arrival order (bit-exact; lasso texels the oracle flags as ambiguous
may differ, below 1e-5 of the texels touched) and the library's single-stroke calls alone."""
import numpy as np
import pytest
import torch

from serve_replay import replay_alone, replay_oracle
from test_gpu_serve import served_models, trace

pytestmark = pytest.mark.gpu

from paper_2501_14807_gb300 import lcl, serve  # noqa: E402


def test_native_server_results_equal_the_oracle_and_requests_alone():
    models, pools = served_models(8)
    one = max(serve.model_image_layout(s)[3] for s in models)
    srv = serve.NativeServer(models, hbm_budget_bytes=int(3.5 * one))   # only a few models fit
    reqs = trace(pools, rate=4000.0, duration=0.3, seed=11)
    srv.run(reqs)
    st = srv.stats()
    assert st["done"] == st["submitted"] == len(reqs)
    assert all(r.t_done >= r.t_arrive for r in reqs)
    # each completion carries its epoch's GPU time: the epoch's work starts after the request arrived and
    # ends before the host sees it complete
    assert all(0.0 <= r.t_gpu <= r.t_done - r.t_arrive + 1e-4 for r in reqs)
    assert st["spills"] > 0 and st["admissions"] > len(models) // 2 and st["epochs"] > 1
    served = {mi: srv.layers_of(mi) for mi in range(len(models))}
    oracle_layers, oracle_results = replay_oracle(models, reqs)
    for mi, (ls, amb, touched) in oracle_layers.items():
        for li, (exp, g) in enumerate(zip(ls, served[mi])):
            diff = g.cpu().numpy() != exp
            assert not (diff & ~amb[li]).any(), f"model {mi} layer {li}: differs from the oracle off ambiguous texels"
            assert diff.sum() <= 1e-5 * max(touched[li], 1)
    n_q = 0
    for i, r in enumerate(reqs):
        if r.kind == serve.QUERY:
            n_q += 1
            ec, ea, n_amb = oracle_results[i]
            if n_amb == 0:
                assert np.array_equal(r.result[0], ec) and np.array_equal(r.result[1], ea), f"query {i}"
            else:
                assert np.abs(r.result[0].astype(np.int64) - ec.astype(np.int64)).sum() <= 2 * n_amb
    assert n_q > 0
    alone_layers, alone_results = replay_alone(models, reqs)
    for mi, ls in alone_layers.items():
        for a, b in zip(ls, served[mi]):
            assert torch.equal(a, b), f"model {mi}: served layers differ from the requests applied alone"
    for i, r in enumerate(reqs):
        if r.kind == serve.QUERY:
            ec, ea = alone_results[i]
            assert np.array_equal(r.result[0], ec) and np.array_equal(r.result[1], ea)
    srv.close()


def test_native_server_rejects_bad_requests():
    models, _ = served_models(2)
    srv = serve.NativeServer(models, hbm_budget_bytes=1 << 30)
    bad = [serve.Request(0.0, 5, serve.SPHERE, sphere=((0.0, 0.0, 0.0), 0.1, 3)),        # no model 5
           serve.Request(0.0, 0, serve.SPHERE, layer=2, sphere=((0.0, 0.0, 0.0), 0.1, 3)),  # no layer 2
           serve.Request(0.0, 0, serve.SPHERE, sphere=((0.0, 0.0, 0.0), 0.1, 300)),       # label above u8
           serve.Request(0.0, 0, serve.LASSO, lasso=(9, np.zeros((3, 2), np.float32), 1))]  # no camera 9
    for r in bad:
        with pytest.raises(lcl.LclError) as e:
            srv.run([r])
        assert e.value.status == 1
    srv.run([serve.Request(0.0, 0, serve.SPHERE, sphere=(models[0].mesh.pos[0].astype(np.float64), 0.2, 9))])
    assert int((srv.layers_of(0)[0] == 9).sum()) > 0
    srv.close()
