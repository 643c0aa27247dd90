"""GPU parity: the CUDA library through its C ABI against the CPU oracle, element by
element, on the same seeded inputs.  Atlas, sphere edits, depth map, overlays and areas
must match bit for bit; lasso labels may differ only on texels the oracle flags as
ambiguous (within 1e-4 px of an edge or 1e-6 of the depth test), and those must stay
below 1e-5 of the texels touched."""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import DEV, assert_atlas_equal, atlas_planes, gpu_atlas, sphere_recs, to_dev, to_np

pytestmark = pytest.mark.gpu

from paper_2501_14807_gb300 import lcl  # noqa: E402

LASSO_TOL = 1e-5


def lattice_soup(seed, W, H, n=40):
    rng = np.random.default_rng(seed)
    c = rng.integers(-2, 2 * max(W, H) + 3, size=(n, 3, 2)) / 2.0
    uv = (c / np.array([W, H])).reshape(-1, 2).astype(np.float32)
    pos = rng.uniform(-1, 1, size=(3 * n, 3)).astype(np.float32)
    idx = np.arange(3 * n, dtype=np.uint32).reshape(n, 3)
    return synth.Mesh(pos, uv, idx.copy(), idx.copy()).check()


ATLAS_CASES = [
    ("vessel-small-1024", lambda: synth.config_small().mesh, 1024, 1024, 32),
    ("vessel-ragged", lambda: synth.vessel_cylindrical(60, 20, seed=4), 300, 170, 32),
    ("charts-512", lambda: synth.vessel_charts(200, 100, 25, 10, 512, seed=5), 512, 512, 64),
    ("soup-t8", lambda: synth.random_soup(200, 6), 100, 70, 8),
    ("soup-t16", lambda: synth.random_soup(300, 7, uv_size=0.5), 64, 48, 16),
    ("lattice-ties", lambda: lattice_soup(8, 48, 40), 48, 40, 16),
    ("square-big-tris", lambda: synth.uv_square_patch(512, 384, 3), 512, 384, 128),
    ("grid-jitter", lambda: synth.grid_patch(37, 23, 256, 200, seed=9, jitter=0.4), 256, 200, 32),
    # big overlapping UV triangles: ~15,800 16x16 blocks against a list of 4096, so most triangles
    # find the list full and are rasterised by their own thread
    ("soup-list-full", lambda: synth.random_soup(400, 11), 512, 384, 32),
]


@pytest.mark.parametrize("name,make,W,H,T", ATLAS_CASES, ids=[c[0] for c in ATLAS_CASES])
def test_atlas_bit_exact(name, make, W, H, T):
    mesh = make()
    o = oracle.Atlas(mesh, W, H, tile=T)
    _, a = gpu_atlas(mesh, W, H, T)
    assert np.array_equal(a.bbox_min, o.mn) and a.scale == o.S
    assert_atlas_equal(a, o)
    assert np.array_equal(to_np(a.cover(), np.uint32), o.cover_bits())
    box = o.tile_aabb()
    assert np.array_equal(to_np(a.tile_box(), np.int32), box)
    assert np.array_equal(to_np(a.super_box(), np.int32), o.super_aabb(box))
    assert np.array_equal(to_np(a.area_w(), np.uint64), o.area_w)


def test_atlas_rejects_bad_inputs():
    mesh = synth.random_soup(10, 1)
    bad = synth.Mesh(mesh.pos, mesh.uv.copy(), mesh.tri_pos, mesh.tri_uv)
    bad.uv[4, 0] = 2.5
    with pytest.raises(lcl.LclError, match="INVALID_ARG"):
        gpu_atlas(bad, 64, 64, 16)
    bad2 = synth.Mesh(mesh.pos, mesh.uv, mesh.tri_pos.copy(), mesh.tri_uv)
    bad2.tri_pos[3, 1] = 10 ** 6
    with pytest.raises(lcl.LclError, match="index out of range"):
        gpu_atlas(bad2, 64, 64, 16)
    flat = synth.Mesh(np.zeros_like(mesh.pos), mesh.uv, mesh.tri_pos, mesh.tri_uv)
    with pytest.raises(lcl.LclError, match="zero extent"):
        gpu_atlas(flat, 64, 64, 16)


SPHERE_CASES = [
    ("small-1024-u8", lambda: synth.config_small().mesh, 1024, 1024, 32, np.uint8, 100, 0.02, 0.02),
    ("ragged-u16", lambda: synth.vessel_cylindrical(60, 20, seed=4), 300, 170, 16, np.uint16, 60, 0.01, 0.4),
    ("charts-u8-t64", lambda: synth.vessel_charts(200, 100, 25, 10, 512, seed=5), 512, 512, 64, np.uint8, 80,
     0.001, 0.3),
    ("t128-u16", lambda: synth.vessel_cylindrical(50, 30, seed=2), 384, 256, 128, np.uint16, 40, 0.05, 0.6),
    # tiles inside big spheres: whole-row handling (W a multiple of 32) and per-quad handling (not)
    ("t32-big-u16", lambda: synth.vessel_charts(160, 80, 20, 10, 1024, seed=6), 1024, 512, 32, np.uint16, 40,
     0.1, 0.6),
    ("t32-odd-width-u8", lambda: synth.vessel_cylindrical(60, 30, seed=6), 1000, 600, 32, np.uint8, 40, 0.05, 0.5),
]


@pytest.mark.parametrize("name,make,W,H,T,dt,n,rlo,rhi", SPHERE_CASES, ids=[c[0] for c in SPHERE_CASES])
def test_sphere_bit_exact(name, make, W, H, T, dt, n, rlo, rhi):
    mesh = make()
    o = oracle.Atlas(mesh, W, H, tile=T)
    _, a = gpu_atlas(mesh, W, H, T)
    st = synth.sphere_strokes(mesh, n, 77, rlo, rhi, 1, int(np.iinfo(dt).max))
    recs = sphere_recs(o, st)
    # a few extreme strokes: everything, nothing, a single exact position
    extra = np.zeros(3, oracle.SPHERE_DTYPE)
    extra[0] = (1 << 20, 1 << 20, 1 << 20, 0, 1 << 62, 3, 0)
    extra[1] = (-(1 << 22), -(1 << 22), -(1 << 22), 0, 0, 4, 0)
    j, i = np.argwhere(o.covered())[len(np.argwhere(o.covered())) // 3]
    extra[2] = (o.px[j, i], o.py[j, i], o.pz[j, i], 0, 0, 5, 0)
    recs = np.concatenate([recs[: n // 2], extra, recs[n // 2:]])
    init = np.random.default_rng(3).integers(0, 9, size=(H, W)).astype(dt)
    exp = init.copy()
    exp_hits = oracle.select_sphere(o, exp, recs)
    layer = to_dev(init)
    hits = torch.zeros(len(recs), dtype=torch.int64, device=DEV)
    lcl.lcl_select_sphere(a, layer, recs, hits_out=hits)
    assert np.array_equal(to_np(layer, dt), exp)
    assert np.array_equal(to_np(hits, np.uint64), exp_hits)
    # the same strokes applied one call at a time give the same layer
    layer2 = to_dev(init)
    for k in range(len(recs)):
        lcl.lcl_select_sphere(a, layer2, recs[k:k + 1])
    assert torch.equal(layer, layer2)
    # in one call without hit counts (the apply may stop at a texel's newest selecting stroke), and
    # in calls of 2 and of 33 strokes (group boundaries)
    layer3 = to_dev(init)
    lcl.lcl_select_sphere(a, layer3, recs)
    assert torch.equal(layer, layer3)
    layer4 = to_dev(init)
    for k0 in range(0, len(recs), 35):
        lcl.lcl_select_sphere(a, layer4, recs[k0:k0 + 2])
        lcl.lcl_select_sphere(a, layer4, recs[k0 + 2:k0 + 35])
    assert torch.equal(layer, layer4)


def test_sphere_host_helper_matches_oracle():
    mesh = synth.config_small().mesh
    o = oracle.Atlas(mesh, 256, 256, tile=32)
    _, a = gpu_atlas(mesh, 256, 256, 32)
    st = synth.sphere_strokes(mesh, 50, 5, 0.001, 0.5, 1, 200)
    for k in range(50):
        got = lcl.lcl_quantize_sphere(a, st.centre[k], st.radius[k], st.label[k])
        exp = oracle.sphere_stroke(o.mn, o.S, st.centre[k], st.radius[k], st.label[k])
        assert tuple(got) == tuple(exp)
    with pytest.raises(lcl.LclError):
        lcl.lcl_quantize_sphere(a, [1e7, 0, 0], 1.0, 1)


def test_camera_helper_matches_oracle():
    mesh = synth.config_small().mesh
    o = oracle.Atlas(mesh, 64, 64, tile=32)
    _, a = gpu_atlas(mesh, 64, 64, 32)
    rng = np.random.default_rng(2)
    for _ in range(5):
        cam = synth.orbit_camera(mesh, 640, 480, rng)
        got = np.array(list(lcl.lcl_camera_from_vp(a, cam.vp, 640, 480).m), np.float32)
        assert np.array_equal(got, oracle.camera_mq(cam.vp, o.mn, o.S))


DEPTH_CASES = [
    ("vessel-orbit", lambda: synth.config_small().mesh, 512, 384, 0),
    ("vessel-orbit-2", lambda: synth.vessel_cylindrical(120, 40, noise_amp=0.05, seed=3), 333, 211, 1),
    ("charts-orbit", lambda: synth.vessel_charts(200, 100, 25, 10, 512, seed=5), 256, 256, 2),
    # triangles spanning most of the screen: far more 16x16 blocks than the list holds
    ("soup-list-full", lambda: synth.random_soup(400, 11), 512, 512, 3),
]


@pytest.mark.parametrize("name,make,Ws,Hs,seed", DEPTH_CASES, ids=[c[0] for c in DEPTH_CASES])
def test_depth_bit_exact(name, make, Ws, Hs, seed):
    mesh = make()
    o = oracle.Atlas(mesh, 64, 64, tile=32, y0=0, y1=1)
    m, a = gpu_atlas(mesh, 64, 64, 32)
    rng = np.random.default_rng(100 + seed)
    for _ in range(3):
        cam = synth.orbit_camera(mesh, Ws, Hs, rng)
        M = oracle.camera_mq(cam.vp, o.mn, o.S)
        exp = oracle.depth(mesh, o.mn, o.S, M, Ws, Hs)
        d = torch.empty((Hs, Ws), dtype=torch.float32, device=DEV)
        lcl.lcl_depth_render(m, a, lcl.camera(M, Ws, Hs), d)
        got = d.cpu().numpy()
        assert np.isfinite(exp).sum() > 0
        assert np.array_equal(got.view(np.uint32), exp.view(np.uint32))


def test_depth_big_triangles_bit_exact():
    W = H = 64
    mesh = synth.uv_square_patch(W, H, k=1000)
    o = oracle.Atlas(mesh, 64, 64, tile=32)
    m, a = gpu_atlas(mesh, 64, 64, 32)
    view = synth.look_at((30000, 20000, 5e5), (32000, 32000, 0), up=(0, 1, 0))
    proj = synth.perspective01(20.0, 1.3, 1e5, 1e6)
    M = oracle.camera_mq(proj @ view, o.mn, o.S)
    exp = oracle.depth(mesh, o.mn, o.S, M, 520, 400)
    d = torch.empty((400, 520), dtype=torch.float32, device=DEV)
    lcl.lcl_depth_render(m, a, lcl.camera(M, 520, 400), d)
    assert np.isfinite(exp).sum() > 1000
    assert np.array_equal(d.cpu().numpy().view(np.uint32), exp.view(np.uint32))


LASSO_CASES = [
    ("vessel-u8", lambda: synth.config_small().mesh, 512, 512, 32, np.uint8, 400, 300),
    ("ragged-u16", lambda: synth.vessel_cylindrical(90, 30, noise_amp=0.03, seed=6), 300, 170, 16, np.uint16,
     257, 199),
    ("charts-u8", lambda: synth.vessel_charts(200, 100, 25, 10, 512, seed=5), 512, 512, 64, np.uint8, 640, 480),
]


@pytest.mark.parametrize("name,make,W,H,T,dt,Ws,Hs", LASSO_CASES, ids=[c[0] for c in LASSO_CASES])
def test_lasso_within_tolerance(name, make, W, H, T, dt, Ws, Hs):
    mesh = make()
    o = oracle.Atlas(mesh, W, H, tile=T)
    m, a = gpu_atlas(mesh, W, H, T)
    rng = np.random.default_rng(55)
    cams = [synth.orbit_camera(mesh, Ws, Hs, rng) for _ in range(3)]
    las = synth.lassos(mesh, cams, 12, 66, 1, int(min(np.iinfo(dt).max, 900)), 1)
    exp = np.zeros((H, W), dt)
    layer = to_dev(exp)
    hits = torch.zeros(1, dtype=torch.int64, device=DEV)
    touched = 0
    amb_all = np.zeros((H, W), bool)
    depths = {}
    for ci, cam in enumerate(cams):
        M = oracle.camera_mq(cam.vp, o.mn, o.S)
        dm = oracle.depth(mesh, o.mn, o.S, M, Ws, Hs)
        d = torch.empty((Hs, Ws), dtype=torch.float32, device=DEV)
        lcl.lcl_depth_render(m, a, lcl.camera(M, Ws, Hs), d)
        assert np.array_equal(d.cpu().numpy().view(np.uint32), dm.view(np.uint32))
        depths[ci] = (M, dm, d)
    for L in las:
        M, dm, d = depths[L.cam]
        h, amb = oracle.select_lasso(o, exp, M, dm, L.poly, L.label)
        touched += h
        amb_all |= amb.astype(bool)
        lcl.lcl_select_lasso(a, layer, lcl.camera(M, Ws, Hs), d, L.poly, L.label, hits_out=hits)
        got_h = int(hits.item())
        assert abs(got_h - h) <= amb.sum()
    got = to_np(layer, dt)
    diff = got != exp
    assert touched > 1000
    assert not (diff & ~amb_all).any(), "lasso labels differ outside the ambiguous texels"
    assert diff.sum() <= LASSO_TOL * touched


def _star(cx, cy, r, n, step):
    k = (np.arange(n) * step) % n
    a = 2.0 * np.pi * k / n + 0.1
    return np.stack([cx + r * np.cos(a), cy + r * np.sin(a)], 1)


ODD_POLYGONS = {
    "off-screen": [(-200, -200), (-100, -200), (-150, -100)],
    "collinear": [(10, 10), (200, 150), (390, 290)],
    "single-point": [(200.5, 150.5)] * 3,
    "pentagram": _star(200, 150, 130, 5, 2),            # even-odd: the centre pentagon is outside
    "bow-tie": [(60, 40), (340, 260), (340, 40), (60, 260)],
    "repeated-vertices": [(100, 100), (100, 100), (300, 100), (300, 220), (300, 220), (100, 220), (100, 100)],
    "horizontal-edges": [(50, 60.5), (150, 60.5), (150, 120.5), (250, 120.5), (250, 60.5), (350, 60.5),
                         (350, 240.5), (50, 240.5)],
    "full-screen": [(-10, -10), (410, -10), (410, 310), (-10, 310)],
    "past-the-edges": [(-80, 150), (200, -90), (480, 150), (200, 390)],
    "triangle": [(50, 50), (350, 80), (200, 280)],
    "64-gon": _star(210, 140, 110, 64, 1),
    "64-star": _star(190, 160, 140, 64, 29),             # heavily self-intersecting
}


@pytest.mark.parametrize("kind", list(ODD_POLYGONS))
def test_lasso_odd_polygons_within_tolerance(kind):
    """Degenerate and self-intersecting lassos (no area, off screen, repeated vertices, horizontal
    edges, a pentagram and a 64-vertex star under the even-odd rule, the 3- and 64-vertex limits,
    polygons past the screen edges) against the oracle."""
    mesh = synth.config_small().mesh
    W = H = 512
    o = oracle.Atlas(mesh, W, H, tile=32)
    m, a = gpu_atlas(mesh, W, H, 32)
    Ws, Hs = 400, 300
    cam = synth.orbit_camera(mesh, Ws, Hs, np.random.default_rng(12))
    M = oracle.camera_mq(cam.vp, o.mn, o.S)
    dm = oracle.depth(mesh, o.mn, o.S, M, Ws, Hs)
    d = torch.empty((Hs, Ws), dtype=torch.float32, device=DEV)
    lcl.lcl_depth_render(m, a, lcl.camera(M, Ws, Hs), d)
    poly = np.asarray(ODD_POLYGONS[kind], np.float32)
    exp = np.zeros((H, W), np.uint8)
    h, amb = oracle.select_lasso(o, exp, M, dm, poly, 7)
    layer = to_dev(np.zeros((H, W), np.uint8))
    hits = torch.zeros(1, dtype=torch.int64, device=DEV)
    lcl.lcl_select_lasso(a, layer, lcl.camera(M, Ws, Hs), d, poly, 7, hits_out=hits)
    got = to_np(layer, np.uint8)
    diff = got != exp
    assert not (diff & ~amb.astype(bool)).any(), "lasso labels differ outside the ambiguous texels"
    assert abs(int(hits.item()) - h) <= amb.sum()
    if kind in ("off-screen", "collinear", "single-point"):
        assert h == 0 and int(hits.item()) == 0
    else:
        assert h > 100


@pytest.mark.parametrize("name,make,W,H,T,dt,Ws,Hs", LASSO_CASES, ids=[c[0] for c in LASSO_CASES])
def test_tool_within_tolerance(name, make, W, H, T, dt, Ws, Hs):
    """The paper's editing tool: circles of the paper's radii (10-200 px), ellipses, random shape
    masks, windows half off screen; labels equal to the oracle's except on flagged texels."""
    mesh = make()
    o = oracle.Atlas(mesh, W, H, tile=T)
    m, a = gpu_atlas(mesh, W, H, T)
    rng = np.random.default_rng(77)
    cams = [synth.orbit_camera(mesh, Ws, Hs, rng) for _ in range(2)]
    centres = [(L.cam, L.poly.mean(0)) for L in synth.lassos(mesh, cams, 8, 78, 1, 2, 1)]
    top = int(min(np.iinfo(dt).max, 900))
    tools = []
    for k, (ci, c) in enumerate(centres):
        r = [10, 40, 70, 100, 200][k % 5]
        tools.append((ci, (float(c[0]), float(c[1])), (2.0 * r, 2.0 * r), None))
        mask = (rng.random((int(rng.integers(1, 24)), int(rng.integers(1, 24)))) < 0.5).astype(np.uint8)
        tools.append((ci, (float(c[0]) + 0.37, float(c[1]) - 0.61), (float(rng.uniform(20, 140)),
                                                                     float(rng.uniform(20, 140))), mask))
    tools.append((0, (3.0, Hs - 2.0), (90.0, 60.0), None))                 # mostly off screen
    tools.append((1, (Ws / 2, Hs / 2), (1.5 * Ws, 1.5 * Hs), np.ones((3, 5), np.uint8)))  # whole screen
    exp = np.zeros((H, W), dt)
    layer = to_dev(exp)
    hits = torch.zeros(1, dtype=torch.int64, device=DEV)
    touched, amb_all = 0, np.zeros((H, W), bool)
    depths = {}
    for ci, cam in enumerate(cams):
        M = oracle.camera_mq(cam.vp, o.mn, o.S)
        dm = oracle.depth(mesh, o.mn, o.S, M, Ws, Hs)
        d = torch.empty((Hs, Ws), dtype=torch.float32, device=DEV)
        lcl.lcl_depth_render(m, a, lcl.camera(M, Ws, Hs), d)
        depths[ci] = (M, dm, d)
    for i, (ci, centre, size, mask) in enumerate(tools):
        M, dm, d = depths[ci]
        label = 1 + (i * 37) % top
        h, amb = oracle.select_tool(o, exp, M, dm, centre, size, mask, label)
        touched += h
        amb_all |= amb.astype(bool)
        shape = None if mask is None else torch.from_numpy(mask).to(DEV)
        tool = lcl.make_tool(centre, size, shape)
        lcl.lcl_select_tool(a, layer, lcl.camera(M, Ws, Hs), d, tool, label, hits_out=hits)
        assert abs(int(hits.item()) - h) <= amb.sum()
    got = to_np(layer, dt)
    diff = got != exp
    assert touched > 1000
    assert not (diff & ~amb_all).any(), "tool labels differ outside the ambiguous texels"
    assert diff.sum() <= LASSO_TOL * touched


@pytest.mark.parametrize("dt", [np.uint8, np.uint16])
def test_tool_padding_within_tolerance(dt):
    """Tool edits with texture padding on a chart atlas (islands with gutters): circle and mask
    tools, radius / thickness 1..8, labels equal to the oracle's except on flagged texels."""
    mesh = synth.vessel_charts(120, 60, 20, 10, 384, seed=8)
    W = H = 384
    o = oracle.Atlas(mesh, W, H, tile=16)
    m, a = gpu_atlas(mesh, W, H, 16)
    Ws, Hs = 320, 240
    rng = np.random.default_rng(21)
    cam = synth.orbit_camera(mesh, Ws, Hs, rng)
    M = oracle.camera_mq(cam.vp, o.mn, o.S)
    dm = oracle.depth(mesh, o.mn, o.S, M, Ws, Hs)
    d = torch.empty((Hs, Ws), dtype=torch.float32, device=DEV)
    lcl.lcl_depth_render(m, a, lcl.camera(M, Ws, Hs), d)
    exp = np.zeros((H, W), dt)
    layer = to_dev(exp)
    hits = torch.zeros(1, dtype=torch.int64, device=DEV)
    touched, padded, amb_all = 0, 0, np.zeros((H, W), bool)
    centres = [L.poly.mean(0) for L in synth.lassos(mesh, [cam], 6, 31, 1, 2, 1)]
    for i, c in enumerate(centres):
        rad, thick = [(1, 1), (2, 1), (3, 4), (8, 8), (5, 2), (1, 6)][i]
        mask = None if i % 2 == 0 else (rng.random((9, 7)) < 0.6).astype(np.uint8)
        size = (float(rng.uniform(40, 160)), float(rng.uniform(40, 160)))
        label = 3 + 11 * i
        h, npad, amb = oracle.select_tool_2d(o, exp, M, dm, (float(c[0]), float(c[1])), size, mask, label,
                                             flags=oracle.pad_flags(rad, thick))
        touched += h + npad
        padded += npad
        amb_all |= amb.astype(bool)
        shape = None if mask is None else torch.from_numpy(mask).to(DEV)
        tool = lcl.make_tool((float(c[0]), float(c[1])), size, shape, lcl.pad_flags(rad, thick))
        lcl.lcl_select_tool(a, layer, lcl.camera(M, Ws, Hs), d, tool, label, hits_out=hits)
        assert abs(int(hits.item()) - h) <= amb.sum()
    got = to_np(layer, dt)
    diff = got != exp
    assert touched > 1000 and padded > 50
    assert not (diff & ~amb_all).any(), "padded tool labels differ outside the ambiguous texels"


@pytest.mark.parametrize("dt", [np.uint8, np.uint16])
def test_lasso_padding_within_tolerance(dt):
    """Lasso edits with texture padding on a chart atlas (islands with gutters), radius / thickness
    1..8: labels equal to the oracle's except on flagged texels (and padded texels next to them)."""
    mesh = synth.vessel_charts(120, 60, 20, 10, 384, seed=8)
    W = H = 384
    o = oracle.Atlas(mesh, W, H, tile=16)
    m, a = gpu_atlas(mesh, W, H, 16)
    Ws, Hs = 320, 240
    rng = np.random.default_rng(23)
    cam = synth.orbit_camera(mesh, Ws, Hs, rng)
    M = oracle.camera_mq(cam.vp, o.mn, o.S)
    dm = oracle.depth(mesh, o.mn, o.S, M, Ws, Hs)
    d = torch.empty((Hs, Ws), dtype=torch.float32, device=DEV)
    lcl.lcl_depth_render(m, a, lcl.camera(M, Ws, Hs), d)
    exp = np.zeros((H, W), dt)
    layer = to_dev(exp)
    hits = torch.zeros(1, dtype=torch.int64, device=DEV)
    touched, padded, amb_all = 0, 0, np.zeros((H, W), bool)
    for i, L in enumerate(synth.lassos(mesh, [cam], 6, 37, 1, 2, 1)):
        rad, thick = [(1, 1), (2, 1), (3, 4), (8, 8), (5, 2), (1, 6)][i]
        label = 5 + 13 * i
        h, npad, amb = oracle.select_lasso_2d(o, exp, M, dm, L.poly, label, flags=oracle.pad_flags(rad, thick))
        touched += h + npad
        padded += npad
        amb_all |= amb.astype(bool)
        lcl.lcl_select_lasso(a, layer, lcl.camera(M, Ws, Hs), d, L.poly, label, hits_out=hits,
                             flags=lcl.pad_flags(rad, thick))
        assert abs(int(hits.item()) - h) <= amb.sum()
    got = to_np(layer, dt)
    diff = got != exp
    assert touched > 1000 and padded > 50
    assert not (diff & ~amb_all).any(), "padded lasso labels differ outside the ambiguous texels"


@pytest.mark.parametrize("dt", [np.uint8, np.uint16])
def test_overlay_bit_exact(dt):
    mesh = synth.vessel_cylindrical(60, 20, seed=4)
    W, H = 300, 170                      # W*H*s not a multiple of 16: exercises the tail
    o = oracle.Atlas(mesh, W, H, tile=32)
    _, a = gpu_atlas(mesh, W, H, 32)
    rng = np.random.default_rng(1)
    A = rng.integers(0, np.iinfo(dt).max + 1, size=(H, W)).astype(dt)
    B = rng.integers(0, np.iinfo(dt).max + 1, size=(H, W)).astype(dt)
    B[::4] = 0
    dA, dB = to_dev(A), to_dev(B)
    out = torch.empty_like(dA)
    for op in ("and", "or", "xor", "mask"):
        for flags in range(8):
            lcl.lcl_overlay(a, dA, dB, out, op, flags)
            assert np.array_equal(to_np(out, dt), oracle.overlay(o, A, B, op, flags)), (op, flags)
    # aliasing: out = a
    dA2 = dA.clone()
    lcl.lcl_overlay(a, dA2, dB, dA2, "xor")
    assert np.array_equal(to_np(dA2, dt), oracle.overlay(o, A, B, "xor"))


@pytest.mark.parametrize("dt,n_labels,W,H", [(np.uint8, 256, 512, 508), (np.uint8, 37, 512, 508),
                                             (np.uint16, 1000, 512, 508), (np.uint16, 5000, 512, 508),
                                             (np.uint16, 65536, 512, 508),
                                             (np.uint8, 256, 1040, 300),
                                             (np.uint16, 300, 1040, 77),
                                             (np.uint8, 256, 300, 201),     # width not a multiple of 16
                                             (np.uint16, 3000, 484, 97)])
def test_label_area_bit_exact(dt, n_labels, W, H):
    mesh = synth.vessel_charts(200, 100, 25, 10, 512, seed=5)
    o = oracle.Atlas(mesh, W, H, tile=32)
    _, a = gpu_atlas(mesh, W, H, 32)
    rng = np.random.default_rng(n_labels)
    L = rng.integers(0, min(np.iinfo(dt).max, n_labels + 30) + 1, size=(H, W)).astype(dt)
    L[min(100, H // 3):min(300, H), 50:400] = 7          # long runs of one label
    if n_labels <= np.iinfo(dt).max:
        L[min(30, H // 5):min(90, H), 100:460] = n_labels   # long runs of a label the query ignores
    ec, ea = oracle.label_area(o, L, n_labels)
    c, ar = lcl.lcl_label_area(a, to_dev(L), n_labels)
    assert np.array_equal(to_np(c, np.uint64), ec)
    assert np.array_equal(to_np(ar, np.uint64), ea)


def test_row_views_match_oracle_bands():
    mesh = synth.vessel_cylindrical(60, 20, seed=4)
    W, H = 256, 200
    _, a = gpu_atlas(mesh, W, H, 32)
    rng = np.random.default_rng(4)
    A = rng.integers(0, 256, size=(H, W)).astype(np.uint8)
    B = rng.integers(0, 256, size=(H, W)).astype(np.uint8)
    for y0, y1 in ((0, 40), (37, 121), (160, 200)):
        if (y0 * W) % 32:
            continue
        o = oracle.Atlas(mesh, W, H, tile=32, y0=y0, y1=y1)
        v = lcl.lcl_atlas_rows(a, y0, y1)
        dA, dB = to_dev(A[y0:y1]), to_dev(B[y0:y1])
        out = torch.empty_like(dA)
        lcl.lcl_overlay(v, dA, dB, out, "or")
        assert np.array_equal(to_np(out, np.uint8), oracle.overlay(o, A[y0:y1], B[y0:y1], "or"))
        c, ar = lcl.lcl_label_area(v, dA, 256)
        ec, ea = oracle.label_area(o, A[y0:y1], 256)
        assert np.array_equal(to_np(c, np.uint64), ec) and np.array_equal(to_np(ar, np.uint64), ea)
    with pytest.raises(lcl.LclError, match="row view"):
        lcl.lcl_select_sphere(lcl.lcl_atlas_rows(a, 0, 40), torch.zeros((40, W), dtype=torch.uint8, device=DEV),
                              np.zeros(1, lcl.SPHERE_DTYPE))


def test_empty_inputs():
    mesh = synth.vessel_cylindrical(20, 8, seed=1)
    m, a = gpu_atlas(mesh, 64, 64, 16)
    layer = torch.zeros((64, 64), dtype=torch.uint8, device=DEV)
    lcl.lcl_select_sphere(a, layer, np.zeros(0, lcl.SPHERE_DTYPE))        # no strokes: nothing happens
    assert int(layer.sum()) == 0
    # a mesh whose triangles all have zero UV area covers nothing
    flat = synth.Mesh(mesh.pos, np.zeros_like(mesh.uv) + 0.5, mesh.tri_pos, mesh.tri_uv)
    o = oracle.Atlas(flat, 64, 64, tile=16)
    _, a2 = gpu_atlas(flat, 64, 64, 16)
    assert (o.tri == oracle.NONE).all()
    assert_atlas_equal(a2, o)
    assert (to_np(a2.tile_box(), np.int32)[:, 3] == 0).all()
    hits = torch.zeros(1, dtype=torch.int64, device=DEV)
    rec = np.array([(1 << 20, 1 << 20, 1 << 20, 0, 1 << 50, 9, 0)], lcl.SPHERE_DTYPE)
    lcl.lcl_select_sphere(a2, layer, rec, hits_out=hits)
    assert int(hits.item()) == 0 and int(layer.sum()) == 0


@pytest.mark.parametrize("T,dt", [(16, np.uint8), (32, np.uint16), (64, np.uint8)])
def test_sphere_with_texture_padding_bit_exact(T, dt):
    """Texture padding (Section 4.3.2) requested per stroke: radius and thickness from 1 to 8, mixed
    with unpadded strokes in one call, on a chart atlas whose gutters leave uncovered texels."""
    mesh = synth.vessel_charts(200, 100, 25, 10, 512, seed=5)
    W = H = 512
    o = oracle.Atlas(mesh, W, H, tile=T)
    _, a = gpu_atlas(mesh, W, H, T)
    st = synth.sphere_strokes(mesh, 24, 41, 0.01, 0.3, 1, int(np.iinfo(dt).max))
    recs = sphere_recs(o, st)
    pads = [(1, 1), (0, 0), (2, 1), (1, 3), (8, 8), (3, 0), (0, 5), (1, 2)]
    for k in range(len(recs)):
        r, t = pads[k % len(pads)]
        recs[k]["flags"] = oracle.pad_flags(r, t)
    init = np.random.default_rng(4).integers(0, 7, size=(H, W)).astype(dt)
    exp = init.copy()
    exp_hits, padded = oracle.select_sphere_2d(o, exp, recs)
    assert padded.sum() > 0
    layer = to_dev(init)
    hits = torch.zeros(len(recs), dtype=torch.int64, device=DEV)
    lcl.lcl_select_sphere(a, layer, recs, hits_out=hits)
    assert np.array_equal(to_np(layer, dt), exp)
    assert np.array_equal(to_np(hits, np.uint64), exp_hits)
    # short calls (one launch per stroke) and long calls (one launch for all) give the same layer
    layer2 = to_dev(init)
    for k in range(0, len(recs), 3):
        lcl.lcl_select_sphere(a, layer2, recs[k:k + 3])
    assert np.array_equal(to_np(layer2, dt), exp)


def test_library_division_equals_ieee_division():
    """The projections divide with the library's own correctly rounded binary32 division (a fast
    route for operands in [2^-30, 2^31), IEEE division elsewhere); it must equal __fdiv_rn bit for
    bit: random operands across and beyond the window, quotients next to rounding midpoints, the
    window's edges, zeros, subnormals, infinities and NaN.  The depth test's exact decisions on the
    quotient (q >= 0, q <= t without dividing where an FMA settles them) are checked on the same
    pairs against __fdiv_rn's quotient, at thresholds on it and one ulp either side."""
    for seed in (1, 2, 3):
        compared, mismatches = lcl.lcl_check_division(1 << 28, seed=seed)
        assert compared > 2 * (1 << 28)   # the divisions plus the decisions of the pairs with b > 0
        assert mismatches == 0
