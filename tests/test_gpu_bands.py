"""Row bands of one texture on the GPU (the partition one GPU per band would use): band atlases
built by the library hold exactly the rows of the whole atlas -- planes, coverage bits, tile and
super-tile boxes against the oracle's band -- and every edit, overlay and per-label table on the
bands gives the rows (and, summed, the tables) of the same calls on the whole atlas, bit for bit.
Padded edits on a band are refused (padding reads rows beyond the band)."""
import numpy as np
import pytest
import torch

import oracle
import synth
from paper_2501_14807_gb300 import lcl, shard

pytestmark = pytest.mark.gpu


def _bits(t):
    return t.cpu().numpy().view(np.uint32)


@pytest.mark.parametrize("W,H,T,world", [(512, 384, 32, 3), (256, 300, 16, 4), (192, 200, 64, 2)])
def test_band_atlases_and_edits_equal_the_whole_texture(W, H, T, world):
    dev = "cuda"
    mesh = synth.vessel_cylindrical(90, 40, noise_amp=0.02, seed=21)
    m = lcl.Mesh.from_host(mesh, dev)
    full = lcl.lcl_atlas_build(m, lcl.Atlas(W, H, T, mesh.n_tri, dev))
    bands = [shard.band_rows(H, T, world, r) for r in range(world)]
    atl = [lcl.lcl_atlas_build(m, lcl.Atlas(W, H, T, mesh.n_tri, dev, band=b)) for b in bands]
    for (y0, y1), a in zip(bands, atl):
        assert (a.row0, a.height, a.tex_height) == (y0, y1 - y0, H)
        for name in ("pos_x", "pos_y", "pos_z", "tri"):
            assert torch.equal(a.plane(name), full.plane(name)[y0:y1]), name
        o = oracle.Atlas(mesh, W, H, tile=T, y0=y0, y1=y1)
        assert np.array_equal(_bits(a.cover()), o.cover_bits())
        box = o.tile_aabb()
        assert np.array_equal(a.tile_box().cpu().numpy(), box)
        assert np.array_equal(a.super_box().cpu().numpy(), o.super_aabb(box))
        assert torch.equal(a.area_w(), full.area_w())
        assert a.scale == full.scale and np.array_equal(a.bbox_min, full.bbox_min)

    st = synth.sphere_strokes(mesh, 40, 8, 0.02, 0.3, 1, 250)
    recs = np.stack([lcl.lcl_quantize_sphere(full, st.centre[k], st.radius[k], st.label[k]) for k in range(40)])
    recs = np.ascontiguousarray(recs, lcl.SPHERE_DTYPE)
    cam_h = synth.orbit_camera(mesh, 160, 120, np.random.default_rng(5))
    cam = lcl.lcl_camera_from_vp(full, cam_h.vp, 160, 120)
    depth = torch.empty((120, 160), dtype=torch.float32, device=dev)
    lcl.lcl_depth_render(m, full, cam, depth)
    poly = synth.star_lasso((80.0, 60.0), 20, 55.0, np.random.default_rng(6))
    tool = lcl.make_tool((70.0, 50.0), (60.0, 44.0))

    def edits(atlas, rows):
        a = torch.zeros((rows, W), dtype=torch.uint8, device=dev)
        b = torch.zeros((rows, W), dtype=torch.uint8, device=dev)
        hits = torch.zeros(40, dtype=torch.int64, device=dev)
        lcl.lcl_select_sphere(atlas, a, recs[:25], hits_out=hits[:25])
        lcl.lcl_select_sphere(atlas, b, recs[15:], hits_out=hits[25:])
        lcl.lcl_select_lasso(atlas, a, cam, depth, poly, 201)
        lcl.lcl_select_tool(atlas, b, cam, depth, tool, 202)
        x = torch.empty_like(a)
        lcl.lcl_overlay(atlas, a, b, x, "xor")
        c, ar = lcl.lcl_label_area(atlas, x, 256)
        return a, b, x, c, ar, hits

    fa, fb, fx, fc, far, fh = edits(full, H)
    sums = [torch.zeros_like(fc), torch.zeros_like(far), torch.zeros_like(fh)]
    for (y0, y1), a in zip(bands, atl):
        ba, bb, bx, bc, bar, bh = edits(a, y1 - y0)
        assert torch.equal(ba, fa[y0:y1]) and torch.equal(bb, fb[y0:y1]) and torch.equal(bx, fx[y0:y1])
        for s, t in zip(sums, (bc, bar, bh)):
            s += t
    assert torch.equal(sums[0], fc) and torch.equal(sums[1], far) and torch.equal(sums[2], fh)
    assert int(fc[1:].sum()) > 0 and int((fa == 201).sum()) > 0 and int((fb == 202).sum()) > 0

    # padding reads rows beyond a band: refused there, accepted on the whole texture
    padded = recs[:1].copy()
    padded["flags"] = oracle.pad_flags(2, 2)
    layer = torch.zeros((atl[0].height, W), dtype=torch.uint8, device=dev)
    with pytest.raises(lcl.LclError) as e:
        lcl.lcl_select_sphere(atl[0], layer, padded)
    assert e.value.status == 4
    lcl.lcl_select_sphere(full, torch.zeros((H, W), dtype=torch.uint8, device=dev), padded)
    torch.cuda.synchronize()
