"""Host logic of the serving loop, on the CPU: the open-loop request generator, the latency
statistics and the victim heap that picks which resident model to spill (its keys must order the
models by their current decayed request rate at any later time without ever being refreshed)."""
import math

import numpy as np

from paper_2501_14807_gb300 import serve


def _requests(n_models=16, rate=20000.0, duration=1.0, seed=3):
    return serve.poisson_requests(n_models, rate, duration, seed, sphere_of=lambda m, rng: ("sphere", m),
                                  lasso_of=lambda m, rng: ("lasso", m))


def test_poisson_requests_follow_rate_mix_and_zipf_law():
    reqs = _requests()
    t = np.array([r.t_arrive for r in reqs])
    assert len(reqs) == 20000
    assert (np.diff(t) > 0).all()
    assert abs(t[-1] - 1.0) < 0.03                      # 20000 exponential gaps of mean 50 us
    kinds = np.bincount([r.kind for r in reqs], minlength=3) / len(reqs)
    assert np.abs(kinds - np.array([0.7, 0.2, 0.1])).max() < 0.02
    freq = np.bincount([r.model for r in reqs], minlength=16) / len(reqs)
    w = 1.0 / np.arange(1, 17) ** 1.1
    assert np.abs(freq - w / w.sum()).max() < 0.01
    for r in reqs:
        assert r.layer in (0, 1)
        if r.kind == serve.SPHERE:
            assert r.sphere == ("sphere", r.model) and r.lasso is None and r.query is None
        elif r.kind == serve.LASSO:
            assert r.lasso == ("lasso", r.model) and r.sphere is None
        else:
            op, la, lb, n_labels = r.query
            assert op in ("and", "or", "xor") and (la, lb) == (0, 1) and n_labels == 256


def test_poisson_requests_are_reproducible():
    a, b, c = _requests(seed=9), _requests(seed=9), _requests(seed=10)
    key = lambda rs: [(r.t_arrive, r.model, r.kind, r.layer) for r in rs]
    assert key(a) == key(b)
    assert key(a) != key(c)


def test_latency_stats_match_numpy():
    rng = np.random.default_rng(4)
    arrive = np.sort(rng.uniform(0.0, 2.0, 999))
    lat = rng.exponential(0.01, 999)
    reqs = []
    for ta, l in zip(arrive, lat):
        r = serve.Request(float(ta), 0, serve.SPHERE)
        r.t_done = float(ta + l)
        reqs.append(r)
    st = serve.latency_stats(reqs)
    span = (arrive + lat).max() - arrive.min()
    assert st["requests"] == 999
    assert math.isclose(st["throughput_rps"], 999 / span, rel_tol=1e-12)
    assert math.isclose(st["p50_ms"], 1e3 * np.percentile(lat, 50), rel_tol=1e-9)
    assert math.isclose(st["p99_ms"], 1e3 * np.percentile(lat, 99), rel_tol=1e-9)
    assert math.isclose(st["max_ms"], 1e3 * lat.max(), rel_tol=1e-9)


def _bare_server(n):
    """A Server with slots and a victim heap only (no device state): enough for _touch/_score."""
    srv = object.__new__(serve.Server)
    srv.slots = [serve._Slot(spec=None, idx=i) for i in range(n)]
    srv._heap = []
    return srv


def _touch_randomly(srv, n_touch, seed):
    rng = np.random.default_rng(seed)
    n = len(srv.slots)
    w = 1.0 / np.arange(1, n + 1) ** 1.1
    t = np.cumsum(rng.exponential(0.01, n_touch))
    for now, i in zip(t, rng.choice(n, size=n_touch, p=w / w.sum())):
        srv._touch(srv.slots[int(i)], float(now))
    return float(t[-1])


def test_score_is_the_decayed_request_count():
    srv = _bare_server(1)
    s = srv.slots[0]
    for now in (0.5, 0.7, 2.0):
        srv._touch(s, now)
    tau = serve.TAU_S
    exp = (math.exp(-0.2 / tau) + 1.0) * math.exp(-1.3 / tau) + 1.0   # touches at 0.5, 0.7, 2.0
    assert math.isclose(serve.Server._score(s, 2.0), exp, rel_tol=1e-12)
    assert math.isclose(serve.Server._score(s, 3.0), exp * math.exp(-1.0 / tau), rel_tol=1e-12)


def test_victim_keys_order_models_by_current_rate():
    srv = _bare_server(24)
    last = _touch_randomly(srv, 3000, 5)
    touched = [s for s in srv.slots if s.score > 0]
    assert len(touched) > 10
    for now in (last, last + 0.3, last + 5.0):
        by_key = sorted(touched, key=lambda s: s.key)
        rates = [serve.Server._score(s, now) for s in by_key]
        assert all(a <= b * (1 + 1e-9) for a, b in zip(rates, rates[1:]))
        for s in touched:   # key = log(current rate) + now / tau at any time after the last touch
            assert math.isclose(s.key, math.log(serve.Server._score(s, now)) + now / serve.TAU_S, rel_tol=1e-9)


def test_victim_heap_pops_each_live_model_once_in_rate_order():
    import heapq
    srv = _bare_server(16)
    _touch_randomly(srv, 20000, 6)          # far more touches than the heap keeps: it is compacted
    assert len(srv._heap) <= 8 * len(srv.slots) + 1024 + 1
    live = []
    heap = list(srv._heap)
    while heap:
        key, i = heapq.heappop(heap)
        if key == srv.slots[i].key:          # stale entries (key changed since) are skipped
            live.append(i)
    touched = {s.idx for s in srv.slots if s.score > 0}
    assert sorted(live) == sorted(touched)           # each touched model exactly once
    keys = [srv.slots[i].key for i in live]
    assert keys == sorted(keys)
