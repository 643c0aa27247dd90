"""Row-band partition of one texture (one band per rank), on CPU: the band arithmetic of
paper_2501_14807_gb300.shard, and two gloo ranks that each run the oracle on their band -- atlas,
sphere strokes, a lasso, an overlay and per-label areas -- then sum the area tables with
shard.reduce_tables.  The union of the bands must equal the single-rank oracle bit for bit: every
texel is edited from its own atlas entry and the stroke (Section 4.3.1), so no rank needs another's
rows, and the per-label sums add up exactly."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2501_14807_gb300 import shard

W, H, T = 160, 150, 16   # 10 tile rows, the last one ragged (150 = 9 * 16 + 6)


def test_band_rows_cover_the_texture_in_tile_aligned_disjoint_bands():
    for height, tile in ((150, 16), (16384, 32), (33, 8), (64, 64)):
        tiles_y = -(-height // tile)
        for world in range(1, min(tiles_y, 9) + 1):
            bands = [shard.band_rows(height, tile, world, r) for r in range(world)]
            assert bands[0][0] == 0 and bands[-1][1] == height
            for (a0, a1), (b0, b1) in zip(bands, bands[1:]):
                assert a1 == b0
            assert all(y0 % tile == 0 and y1 > y0 for y0, y1 in bands)
            sizes = [-(-(y1 - y0) // tile) for y0, y1 in bands]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard.band_rows(150, 16, 11, 0)         # 10 tile rows, 11 ranks
    with pytest.raises(ValueError):
        shard.band_rows(150, 16, 2, 2)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _workload():
    import oracle
    import synth
    mesh = synth.vessel_cylindrical(48, 24, noise_amp=0.02, seed=7)
    mn, S = oracle.quant_params(mesh.pos)
    st = synth.sphere_strokes(mesh, 30, 5, 0.02, 0.25, 1, 200)
    recs = oracle.sphere_records(mn, S, st.centre, st.radius, st.label)
    cam = synth.orbit_camera(mesh, 120, 90, np.random.default_rng(3))
    m = oracle.camera_mq(cam.vp, mn, S)
    dm = oracle.depth(mesh, mn, S, m, 120, 90)
    poly = synth.star_lasso((60.0, 45.0), 24, 40.0, np.random.default_rng(4))
    return mesh, recs, m, dm, poly


def _run_band(y0, y1):
    """The oracle on rows [y0, y1): two layers edited, their XOR, per-label tables of both."""
    import oracle
    mesh, recs, m, dm, poly = _workload()
    o = oracle.Atlas(mesh, W, H, tile=T, y0=y0, y1=y1)
    layers = [np.zeros((y1 - y0, W), np.uint8) for _ in range(2)]
    oracle.select_sphere(o, layers[0], recs[:20])
    oracle.select_sphere(o, layers[1], recs[10:])
    oracle.select_lasso(o, layers[0], m, dm, poly, 77)
    x = oracle.overlay(o, layers[0], layers[1], "xor")
    tables = [oracle.label_area(o, L, 256) for L in (layers[0], x)]
    return o, layers, x, tables


def _rank(rank, world, port, q):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    y0, y1 = shard.band_rows(H, T, world, rank)
    o, layers, x, tables = _run_band(y0, y1)
    flat = [torch.from_numpy(t.view(np.int64).copy()) for pair in tables for t in pair]
    shard.reduce_tables(flat)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, (y0, y1), layers, x, [t.numpy().view(np.uint64) for t in flat], o.tile_aabb(), o.area_w))


def test_two_gloo_ranks_bands_equal_the_single_rank_oracle():
    import oracle
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = {}
    for _ in procs:
        r = q.get(timeout=180)
        res[r[0]] = r[1:]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    o, layers, x, tables = _run_band(0, H)
    full_tables = [t for pair in tables for t in pair]
    full_boxes = o.tile_aabb().reshape(-(-H // T), -(-W // T), 8)
    assert res[0][0][0] == 0 and res[0][0][1] == res[1][0][0] and res[1][0][1] == H
    for li in range(2):
        assert np.array_equal(np.vstack([res[r][1][li] for r in (0, 1)]), layers[li])
    assert np.array_equal(np.vstack([res[r][2] for r in (0, 1)]), x)
    for r in (0, 1):
        (y0, y1), _, _, sums, boxes, area_w = res[r]
        for got, exp in zip(sums, full_tables):       # every rank holds the reduced tables
            assert np.array_equal(got, exp)
        assert np.array_equal(boxes.reshape(-1, full_boxes.shape[1], 8), full_boxes[y0 // T: -(-y1 // T)])
        assert np.array_equal(area_w, o.area_w)
    assert full_tables[0][77] > 0 and full_tables[0][1:].sum() > 0     # the lasso and strokes hit texels
    # a rank's own (unreduced) table is a strict part of the whole
    _, _, _, own = _run_band(*shard.band_rows(H, T, 2, 0))
    assert own[0][0].sum() < full_tables[0].sum()
    assert oracle is not None
