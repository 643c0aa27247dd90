"""Batched edits (many models, queued sphere and lasso strokes, one cull and one persistent apply
launch) against the same strokes applied one call at a time, in queue order, through the
single-stroke entry points -- and, for some models, against the oracle.  Results must be
identical bit for bit: the batch only changes the schedule."""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import DEV, to_dev, to_np

pytestmark = pytest.mark.gpu

from paper_2501_14807_gb300 import lcl  # noqa: E402

BIAS = lcl.DEFAULT_BIAS


def build(models, tiles, dtypes, seed=0):
    """GPU atlases, initial layers, depth maps and per-model queues for a list of BatchModel."""
    out = []
    rng = np.random.default_rng(seed)
    for bm, T, dt in zip(models, tiles, dtypes):
        mesh = lcl.Mesh.from_host(bm.mesh, DEV)
        a = lcl.Atlas(bm.side, bm.side, T, bm.mesh.n_tri, DEV)
        lcl.lcl_atlas_build(mesh, a)
        init = rng.integers(0, 5, size=(bm.side, bm.side)).astype(dt)
        cams = [lcl.lcl_camera_from_vp(a, c.vp, c.width, c.height) for c in bm.cams]
        depths = []
        for c in cams:
            d = torch.empty((c.height, c.width), dtype=torch.float32, device=DEV)
            lcl.lcl_depth_render(mesh, a, c, d)
            depths.append(d)
        top = int(np.iinfo(dt).max)
        queue = []
        for e in bm.order:
            if e >= 0:
                rec = lcl.lcl_quantize_sphere(a, bm.strokes.centre[e], bm.strokes.radius[e],
                                              min(int(bm.strokes.label[e]) * 131 % top + 1, top))
                queue.append(("sphere", rec))
            else:
                L = bm.lassos[-1 - e]
                queue.append(("lasso", (cams[L.cam], depths[L.cam], L.poly, min(L.label * 7 % top + 1, top), BIAS)))
        out.append(dict(bm=bm, mesh=mesh, atlas=a, init=init, queue=queue, dtype=dt))
    return out


def run_sequential(models):
    layers = []
    for m in models:
        layer = to_dev(m["init"])
        for kind, payload in m["queue"]:
            if kind == "sphere":
                lcl.lcl_select_sphere(m["atlas"], layer, np.array([payload], lcl.SPHERE_DTYPE))
            else:
                cam, depth, poly, label, bias = payload[:5]
                flags = payload[5] if len(payload) > 5 else 0
                lcl.lcl_select_lasso(m["atlas"], layer, cam, depth, poly, label, bias, flags=flags)
        layers.append(layer)
    return layers


def with_padding(models, seed=7):
    """The same models with texture padding on about a third of their strokes (radius and
    thickness 1..8), spheres and lassos alike."""
    rng = np.random.default_rng(seed)
    out = []
    for m in models:
        q = []
        for kind, payload in m["queue"]:
            pad = lcl.pad_flags(int(rng.integers(1, 9)), int(rng.integers(1, 9))) if rng.random() < 0.35 else 0
            if kind == "sphere":
                rec = payload.copy()
                rec["flags"] = pad
                q.append(("sphere", rec))
            else:
                q.append(("lasso", tuple(payload[:5]) + (pad,)))
        out.append(dict(m, queue=q))
    return out


def make_batch(models):
    layers = [to_dev(m["init"]) for m in models]
    b = lcl.Batch([(m["atlas"], l) for m, l in zip(models, layers)], [m["queue"] for m in models])
    return b, layers


@pytest.fixture(scope="module")
def models():
    kinds = ["vessel", "sphere", "torus", "vessel", "torus", "sphere"]
    tris = [3000, 9000, 20000, 40000, 6000, 15000]
    bms = [synth.batch_model(k, t, 50 + i, n_sphere=40, n_lasso=12, depth_side=320) for i, (k, t) in
           enumerate(zip(kinds, tris))]
    for bm in bms:
        bm.side = 256 if bm.mesh.n_tri < 10000 else 512
    return build(bms, [16, 32, 64, 32, 128, 32], [np.uint8, np.uint16, np.uint8, np.uint8, np.uint16, np.uint8])


def test_batch_equals_sequential_single_stroke_calls(models):
    seq = run_sequential(models)
    b, layers = make_batch(models)
    lcl.lcl_batch_edit(b)
    torch.cuda.synchronize()
    for m, s, l in zip(models, seq, layers):
        assert torch.equal(s, l), "batched layer differs from sequential calls"
        assert not torch.equal(l, to_dev(m["init"]))


def test_batch_matches_oracle_on_two_models(models):
    b, layers = make_batch(models)
    lcl.lcl_batch_edit(b)
    torch.cuda.synchronize()
    for mi in (0, 1):
        m = models[mi]
        bm = m["bm"]
        o = oracle.Atlas(bm.mesh, bm.side, bm.side, tile=m["atlas"].tile)
        exp = m["init"].copy()
        amb = np.zeros(exp.shape, bool)
        for kind, payload in m["queue"]:
            if kind == "sphere":
                oracle.select_sphere(o, exp, np.array([payload], oracle.SPHERE_DTYPE))
            else:
                cam, depth, poly, label, bias = payload
                M = np.array(list(cam.m), np.float32)
                dm = oracle.depth(bm.mesh, o.mn, o.S, M, cam.width, cam.height)
                _, a = oracle.select_lasso(o, exp, M, dm, poly, label, bias)
                amb |= a.astype(bool)
        d = to_np(layers[mi], m["dtype"]) != exp
        assert not (d & ~amb).any()


def test_batch_relaunch_and_cuda_graph_replay(models):
    seq = run_sequential(models)
    b, layers = make_batch(models)
    lcl.lcl_batch_edit(b)
    torch.cuda.synchronize()
    # the same queue again on its own result changes nothing
    lcl.lcl_batch_launch(b)
    torch.cuda.synchronize()
    for s, l in zip(seq, layers):
        assert torch.equal(s, l)
    # capture the launch in a CUDA graph, reset the layers, replay
    g = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        with torch.cuda.graph(g, stream=side):
            lcl.lcl_batch_launch(b)
    torch.cuda.current_stream().wait_stream(side)
    for m, l in zip(models, layers):
        l.copy_(to_dev(m["init"]))
    g.replay()
    torch.cuda.synchronize()
    for s, l in zip(seq, layers):
        assert torch.equal(s, l)


def test_batch_rejects_long_queues(models):
    m = models[0]
    rec = m["queue"][0]
    with pytest.raises(ValueError):
        lcl.Batch([(m["atlas"], to_dev(m["init"]))], [[rec] * 65])


def test_batch_back_to_back_edits_reuse_staging_safely(models):
    """Three edits in a row on one Batch without synchronising: each call must wait until the
    previous upload from the shared pinned staging has run before rewriting it."""
    seq = run_sequential(models)
    b, layers = make_batch(models)
    for _ in range(3):
        lcl.lcl_batch_edit(b)
    torch.cuda.synchronize()
    for s, l in zip(seq, layers):
        assert torch.equal(s, l)


def run_sequential_queues(models, queues, inits):
    layers = []
    for m, q, init in zip(models, queues, inits):
        layer = to_dev(init)
        for kind, payload in q:
            if kind == "sphere":
                lcl.lcl_select_sphere(m["atlas"], layer, np.array([payload], lcl.SPHERE_DTYPE))
            else:
                cam, depth, poly, label, bias = payload
                lcl.lcl_select_lasso(m["atlas"], layer, cam, depth, poly, label, bias)
        layers.append(layer)
    return layers


@pytest.mark.parametrize("threads,ctas,split", [(64, 0, 1), (128, 0, 2), (256, 2, 4), (64, 1, 8), (256, 0, 8),
                                                (128, 3, 1)])
def test_batch_launch_shapes_give_identical_results(models, threads, ctas, split):
    seq = run_sequential(models)
    b, layers = make_batch(models)
    b.config = lcl.batch_config(threads, ctas, split)
    lcl.lcl_batch_edit(b)
    torch.cuda.synchronize()
    for s, l in zip(seq, layers):
        assert torch.equal(s, l)


def test_batch_autotuner_keeps_results(models):
    seq = run_sequential(models)
    b, layers = make_batch(models)
    lcl.lcl_batch_upload(b)
    cfg, ms = lcl.lcl_batch_tune(b, reps=1)
    assert cfg.threads in (64, 128, 256) and cfg.split in (1, 2, 4, 8) and 0 <= cfg.ctas_per_sm <= 32
    assert ms > 0
    torch.cuda.synchronize()
    for s, l in zip(seq, layers):  # the tuner re-ran the strokes many times: same labels
        assert torch.equal(s, l)
    for l, m in zip(layers, models):
        l.copy_(to_dev(m["init"]))
    lcl.lcl_batch_edit(b)  # with the tuned shape
    torch.cuda.synchronize()
    for s, l in zip(seq, layers):
        assert torch.equal(s, l)


def test_one_graph_serves_different_batches_within_limits(models):
    """Capture the launch once for limits covering every model; upload two different batches
    (different models, queue orders and lengths) and replay the same graph for each."""
    full, _ = make_batch(models)
    limits = full.own_limits
    ws = lcl.batch_workspace(limits, DEV)
    graph = lcl.BatchGraph(limits, lcl.batch_config(128, 0, 2), ws)
    picks = [(list(range(0, 3)), lambda q: q), (list(range(2, 6)), lambda q: q[::-1][:50])]
    for idx, reorder in picks:
        sub = [models[i] for i in idx]
        queues = [reorder(m["queue"]) for m in sub]
        inits = [m["init"] for m in sub]
        seq = run_sequential_queues(sub, queues, inits)
        layers = [to_dev(x) for x in inits]
        b = lcl.Batch([(m["atlas"], l) for m, l in zip(sub, layers)], queues, workspace=ws, limits=limits)
        assert b.workspace is ws
        lcl.lcl_batch_upload(b)
        graph.replay()
        torch.cuda.synchronize()
        for s, l in zip(seq, layers):
            assert torch.equal(s, l)


def test_batch_rejects_batches_above_the_limits(models):
    small = lcl.batch_limits(1, 64, 16, 1 << 20, 1 << 24)
    with pytest.raises(ValueError):
        lcl.Batch([(m["atlas"], to_dev(m["init"])) for m in models[:2]], [m["queue"] for m in models[:2]],
                  limits=small)


@pytest.fixture(scope="module")
def chart_models():
    """Models whose atlases have gutters (rectangular charts shelf-packed with 2-texel gaps), so that
    texture padding has uncovered texels to write: three chart vessels with different tiles, label
    widths and queues of 40 spheres and 12 lassos."""
    bms = []
    for i, (nt, nh, side) in enumerate([(60, 30, 256), (120, 60, 512), (80, 40, 384)]):
        m = synth.vessel_charts(nt, nh, 10 if nt % 20 else 20, 10, side, seed=60 + i)
        rng = np.random.default_rng(70 + i)
        st = synth.sphere_strokes(m, 40, 80 + i, 0.01, 0.2, 1, 255)
        cams = [synth.orbit_camera(m, 320, 320, rng) for _ in range(2)]
        las = synth.lassos(m, cams, 12, 90 + i, 1, 255, 1)
        order = np.concatenate([np.arange(40), -1 - np.arange(12)])
        rng.shuffle(order)
        bms.append(synth.BatchModel(m, side, st, cams, las, order))
    return build(bms, [16, 32, 16], [np.uint8, np.uint16, np.uint8], seed=3)


def test_batch_with_texture_padding_equals_sequential_calls(chart_models):
    """Padded sphere and lasso strokes in a batch: identical to the single-stroke calls in queue order,
    and to the oracle's padded edits except on flagged texels."""
    pm = with_padding(chart_models)
    seq = run_sequential(pm)
    b, layers = make_batch(pm)
    lcl.lcl_batch_edit(b)
    torch.cuda.synchronize()
    for s, l in zip(seq, layers):
        assert torch.equal(s, l), "padded batched layer differs from sequential calls"
    m = pm[0]
    bm = m["bm"]
    o = oracle.Atlas(bm.mesh, bm.side, bm.side, tile=m["atlas"].tile)
    exp = m["init"].copy()
    amb = np.zeros(exp.shape, bool)
    n_pad = 0
    for kind, payload in m["queue"]:
        if kind == "sphere":
            _, p = oracle.select_sphere_2d(o, exp, np.array([payload], oracle.SPHERE_DTYPE))
            n_pad += int(p.sum())
        else:
            cam, depth, poly, label, bias, flags = payload
            M = np.array(list(cam.m), np.float32)
            dm = oracle.depth(bm.mesh, o.mn, o.S, M, cam.width, cam.height)
            _, p, a = oracle.select_lasso_2d(o, exp, M, dm, poly, label, bias, flags)
            n_pad += p
            amb |= a.astype(bool)
    d = to_np(layers[0], m["dtype"]) != exp
    assert not (d & ~amb).any()
    assert n_pad > 100
