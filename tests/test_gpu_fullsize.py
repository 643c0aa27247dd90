"""GPU parity at the benchmark's full size: the 16384^2 atlas of the ~8M-triangle vessel, 4 uint8
layers, 1000 sphere strokes, 4 depth maps of 2048^2 and 20 lassos, XOR/OR overlays and per-label
areas -- the same workload and launch configuration bench.py times.  The oracle cannot redo the
whole texture in seconds, so it computes three 32-row bands (top, middle, bottom) of every result
and the GPU's rows there must match: bit for bit for the atlas, the sphere edits, overlays and
areas; within the lasso tolerance for lassos.  Depth maps and all 8M area weights are compared
whole, and the full-texture area sums are checked against the coverage counts."""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import DEV, to_np

pytestmark = pytest.mark.gpu

from paper_2501_14807_gb300 import lcl  # noqa: E402

BANDS = [(0, 32), (8192, 8224), (16352, 16384)]


@pytest.fixture(scope="module")
def run():
    w = synth.config_roofline()
    W, H = w.width, w.height
    mesh = lcl.Mesh.from_host(w.mesh, DEV)
    atlas = lcl.Atlas(W, H, w.tile, w.mesh.n_tri, DEV)
    lcl.lcl_atlas_build(mesh, atlas)
    layers = [torch.zeros((H, W), dtype=torch.uint8, device=DEV) for _ in range(w.n_layers)]
    recs = []
    for li in range(w.n_layers):
        sel = np.nonzero(w.strokes.layer == li)[0]
        r = np.ascontiguousarray(np.stack([lcl.lcl_quantize_sphere(atlas, w.strokes.centre[k], w.strokes.radius[k],
                                                                   w.strokes.label[k]) for k in sel]),
                                 dtype=lcl.SPHERE_DTYPE)
        recs.append(r)
        lcl.lcl_select_sphere(atlas, layers[li], r)
    after_sphere = [[to_np(l[y0:y1], np.uint8) for (y0, y1) in BANDS] for l in layers]
    cams = [lcl.lcl_camera_from_vp(atlas, c.vp, c.width, c.height) for c in w.cams]
    depths = [torch.empty((c.height, c.width), dtype=torch.float32, device=DEV) for c in w.cams]
    for c, d in zip(cams, depths):
        lcl.lcl_depth_render(mesh, atlas, c, d)
    for L in w.lassos:
        lcl.lcl_select_lasso(atlas, layers[L.layer], cams[L.cam], depths[L.cam], L.poly, L.label)
    after_lasso = [[to_np(l[y0:y1], np.uint8) for (y0, y1) in BANDS] for l in layers]
    torch.cuda.synchronize()
    return w, atlas, layers, recs, cams, depths, after_sphere, after_lasso


def test_fullsize_atlas_bands_and_area_weights(run):
    w, atlas, *_ = run
    for bi, (y0, y1) in enumerate(BANDS):
        o = oracle.Atlas(w.mesh, w.width, w.height, tile=w.tile, y0=y0, y1=y1)
        if bi == 0:
            assert np.array_equal(atlas.bbox_min, o.mn) and atlas.scale == o.S
            assert np.array_equal(to_np(atlas.area_w(), np.uint64), o.area_w)
        for name, plane in (("tri", o.tri), ("pos_x", o.px), ("pos_y", o.py), ("pos_z", o.pz)):
            got = to_np(atlas.plane(name)[y0:y1], plane.dtype)
            assert np.array_equal(got, plane), f"{name} differs in rows [{y0}, {y1})"
        # the band is exactly one row of tiles: their boxes follow from the band alone
        ob = oracle.lib()
        box = np.empty((w.width // w.tile, 8), np.int32)
        import ctypes as C
        ob.orc_tile_aabb(C.c_int32(w.width), C.c_int32(y1 - y0), C.c_int32(w.tile), o.px.ctypes.data_as(C.c_void_p),
                         o.py.ctypes.data_as(C.c_void_p), o.pz.ctypes.data_as(C.c_void_p),
                         o.tri.ctypes.data_as(C.c_void_p), box.ctypes.data_as(C.c_void_p))
        row = y0 // w.tile
        got_box = to_np(atlas.tile_box(), np.int32).reshape(-1, w.width // w.tile, 8)[row]
        assert np.array_equal(got_box, box)


def test_fullsize_sphere_bands(run):
    w, atlas, layers, recs, cams, depths, after_sphere, _ = run
    for bi, (y0, y1) in enumerate(BANDS):
        o = oracle.Atlas(w.mesh, w.width, w.height, tile=w.tile, y0=y0, y1=y1)
        for li in range(w.n_layers):
            exp = np.zeros((y1 - y0, w.width), np.uint8)
            orecs = oracle.sphere_records(o.mn, o.S, w.strokes.centre[w.strokes.layer == li],
                                          w.strokes.radius[w.strokes.layer == li],
                                          w.strokes.label[w.strokes.layer == li])
            assert np.array_equal(orecs, recs[li].view(orecs.dtype))
            oracle.select_sphere(o, exp, orecs)
            assert np.array_equal(after_sphere[li][bi], exp), f"layer {li} rows [{y0}, {y1})"


def test_fullsize_depth_maps(run):
    w, atlas, layers, recs, cams, depths, *_ = run
    mn, S = oracle.quant_params(w.mesh.pos)
    for c, cam, d in zip(w.cams, cams, depths):
        M = oracle.camera_mq(c.vp, mn, S)
        assert np.array_equal(np.array(list(cam.m), np.float32), M)
        exp = oracle.depth(w.mesh, mn, S, M, c.width, c.height)
        assert np.array_equal(d.cpu().numpy().view(np.uint32), exp.view(np.uint32))


def test_fullsize_lasso_bands(run):
    w, atlas, layers, recs, cams, depths, after_sphere, after_lasso = run
    mn, S = oracle.quant_params(w.mesh.pos)
    Ms = [oracle.camera_mq(c.vp, mn, S) for c in w.cams]
    dms = [d.cpu().numpy() for d in depths]   # equal to the oracle's maps (checked above)
    touched, diffs = 0, 0
    for bi, (y0, y1) in enumerate(BANDS):
        o = oracle.Atlas(w.mesh, w.width, w.height, tile=w.tile, y0=y0, y1=y1)
        exp = [after_sphere[li][bi].copy() for li in range(w.n_layers)]
        amb = [np.zeros_like(e, dtype=bool) for e in exp]
        for L in w.lassos:
            h, a = oracle.select_lasso(o, exp[L.layer], Ms[L.cam], dms[L.cam], L.poly, L.label)
            touched += h
            amb[L.layer] |= a.astype(bool)
        for li in range(w.n_layers):
            d = after_lasso[li][bi] != exp[li]
            assert not (d & ~amb[li]).any(), f"lasso differs outside ambiguous texels, layer {li} band {bi}"
            diffs += int(d.sum())
    assert touched > 0
    assert diffs <= 1e-5 * touched


def test_fullsize_overlay_and_area(run):
    w, atlas, layers, *_ = run
    outs = []
    for op, ia, ib in w.overlays:
        out = torch.empty_like(layers[0])
        lcl.lcl_overlay(atlas, layers[ia], layers[ib], out, op)
        outs.append((op, ia, ib, out))
    for y0, y1 in BANDS:
        o = oracle.Atlas(w.mesh, w.width, w.height, tile=w.tile, y0=y0, y1=y1)
        v = lcl.lcl_atlas_rows(atlas, y0, y1)
        host = [to_np(l[y0:y1], np.uint8) for l in layers]
        for op, ia, ib, out in outs:
            assert np.array_equal(to_np(out[y0:y1], np.uint8), oracle.overlay(o, host[ia], host[ib], op))
        for li in range(w.n_layers):
            c, a = lcl.lcl_label_area(v, layers[li][y0:y1], w.n_labels)
            ec, ea = oracle.label_area(o, host[li], w.n_labels)
            assert np.array_equal(to_np(c, np.uint64), ec) and np.array_equal(to_np(a, np.uint64), ea)
    # whole texture: with 256 labels every covered texel is counted once
    covered = int(to_np(atlas.tile_box(), np.int32)[:, 3].astype(np.int64).sum())
    for li in range(w.n_layers):
        c, a = lcl.lcl_label_area(atlas, layers[li], 256)
        assert int(to_np(c, np.uint64).sum()) == covered
