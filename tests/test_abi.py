"""The C ABI without a GPU: liblcl.so loads, exports every function include/lcl.h declares,
lays out atlas buffers as documented, and rejects bad arguments on the host before anything
is enqueued.  Every call here is built to fail a host-side check, so no device memory is
ever touched (the pointers are placeholders)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lcl.h")


@pytest.fixture(scope="module")
def lcl():
    from paper_2501_14807_gb300 import build, lcl as binding
    if not os.path.exists(binding.LIB_PATH):
        build.build()
    binding.library()
    return binding


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(lcl_[a-z_0-9]+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_path_entry_points():
    names = declared_functions()
    for n in ("lcl_atlas_build", "lcl_depth_render", "lcl_select_sphere", "lcl_select_lasso", "lcl_overlay",
              "lcl_label_area"):
        assert n in names


def test_library_exports_every_declared_function(lcl):
    lib = C.CDLL(lcl.LIB_PATH)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing
    assert sorted(lcl.EXPORTS) == declared_functions()


def test_status_strings(lcl):
    assert lcl.lcl_status_str(0) == "LCL_OK" and lcl.lcl_status_str(4) == "LCL_ERR_UNSUPPORTED"
    assert lcl.lcl_status_str(99) == "LCL_ERR_UNKNOWN"


def test_atlas_layout(lcl):
    lib = lcl.library()
    assert lib.lcl_atlas_bytes(1000, 70, 32, 10) > 0
    assert lib.lcl_atlas_bytes(1002, 70, 32, 10) == 0        # width not a multiple of 4
    assert lib.lcl_atlas_bytes(64, 64, 24, 10) == 0          # tile not a power of two in [8, 128]
    assert lib.lcl_atlas_bytes(20000, 64, 32, 10) == 0       # too wide
    W, H, T, n = 100, 70, 32, 123
    nb = lib.lcl_atlas_bytes(W, H, T, n)
    a = lcl.lcl_atlas()
    base = 1 << 40                                           # placeholder address, never dereferenced
    assert lib.lcl_atlas_bind(C.c_void_p(base), nb, W, H, T, n, C.byref(a)) == 0
    assert (a.tiles_x, a.tiles_y, a.supers_x, a.supers_y) == (4, 3, 1, 1)
    planes = [a.pos_x, a.pos_y, a.pos_z, a.tri, a.cover, a.tile_box, a.super_box, a.area_w]
    assert all(p % 256 == 0 for p in planes)
    assert planes == sorted(planes)
    assert a.pos_y - a.pos_x >= W * H * 4 and a.cover - a.tri >= W * H * 4
    assert a.area_w + n * 8 <= base + nb
    # too small, misaligned
    assert lib.lcl_atlas_bind(C.c_void_p(base), nb - 1, W, H, T, n, C.byref(a)) == 2
    assert lib.lcl_atlas_bind(C.c_void_p(base + 16), nb, W, H, T, n, C.byref(a)) == 1
    # row views
    v = lcl.lcl_atlas()
    assert lib.lcl_atlas_rows(C.byref(a), 8, 40, C.byref(v)) == 0
    assert v.height == 32 and v.row0 == 8 and v.tri == a.tri + 8 * W * 4 and v.cover == a.cover + 8 * W // 32 * 4
    assert v.tile_box is None and v.super_box is None
    assert lib.lcl_atlas_rows(C.byref(a), 3, 40, C.byref(v)) == 1   # 3 * 100 not a multiple of 32
    assert lib.lcl_atlas_rows(C.byref(a), 0, 71, C.byref(v)) == 1


def test_band_atlas_binding(lcl):
    """lcl_atlas_bind_band: rows [y0, y1) of a texture, laid out as an atlas of y1 - y0 rows with its
    own boxes; texture padding is refused on it (host-side checks only)."""
    lib = lcl.library()
    W, TH, T, n = 128, 300, 32, 50
    a = lcl.lcl_atlas()
    nb = lib.lcl_atlas_bytes(W, 300 - 192, T, n)
    assert lib.lcl_atlas_bind_band(C.c_void_p(1 << 40), nb, W, TH, 192, 300, T, n, C.byref(a)) == 0
    assert (a.height, a.row0, a.tex_height, a.tiles_y, a.tiles_x) == (108, 192, 300, 4, 4)
    assert a.tile_box is not None and a.super_box is not None
    w = lcl.lcl_atlas()
    assert lib.lcl_atlas_bind(C.c_void_p(1 << 40), lib.lcl_atlas_bytes(W, TH, T, n), W, TH, T, n, C.byref(w)) == 0
    assert (w.row0, w.tex_height) == (0, TH)
    for y0, y1 in ((-1, 10), (10, 10), (200, 301)):
        assert lib.lcl_atlas_bind_band(C.c_void_p(1 << 40), nb, W, TH, y0, y1, T, n, C.byref(a)) == 1
    assert lib.lcl_atlas_bind_band(C.c_void_p(1 << 40), nb - 1, W, TH, 192, 300, T, n, C.byref(a)) == 2
    assert lib.lcl_atlas_bind_band(C.c_void_p(1 << 40), nb, W, TH, 192, 300, T, n, C.byref(a)) == 0
    recs = np.zeros(2, lcl.SPHERE_DTYPE)
    recs[1]["flags"] = 1                                     # padding radius 1
    wsb = lib.lcl_select_workspace_bytes(C.byref(a), 2)
    P = lambda r: r.ctypes.data_as(C.c_void_p)  # noqa: E731
    st = lib.lcl_select_sphere(C.byref(a), C.c_void_p(1 << 41), 1, P(recs), 2, None, C.c_void_p(1 << 42), wsb, None)
    assert st == 4 and "band" in lcl.lcl_last_error()
    cam = lcl.lcl_camera()
    cam.width, cam.height = 64, 48
    poly = np.zeros((3, 2), np.float32)
    st = lib.lcl_select_lasso(C.byref(a), C.c_void_p(1 << 41), 1, C.byref(cam), C.c_void_p(1 << 43), P(poly), 3, 5,
                              0x22, C.c_float(0.001), None, C.c_void_p(1 << 42), wsb, None)
    assert st == 4
    bad = lcl.lcl_atlas.from_buffer_copy(a)
    bad.row0 = 250                                           # rows past the texture
    st = lib.lcl_overlay(C.byref(bad), C.c_void_p(1 << 41), C.c_void_p(1 << 41), C.c_void_p(1 << 41), 1, 0, 0, None)
    assert st == 1


def _bound(lcl, W=64, H=64, T=16, n=10):
    lib = lcl.library()
    a = lcl.lcl_atlas()
    nb = lib.lcl_atlas_bytes(W, H, T, n)
    assert lib.lcl_atlas_bind(C.c_void_p(1 << 40), nb, W, H, T, n, C.byref(a)) == 0
    return lib, a


def test_select_sphere_rejects_bad_arguments(lcl):
    lib, a = _bound(lcl)
    layer = C.c_void_p(1 << 41)
    ws = C.c_void_p(1 << 42)
    wsb = lib.lcl_select_workspace_bytes(C.byref(a), 4)
    good = np.zeros(4, lcl.SPHERE_DTYPE)
    P = lambda r: r.ctypes.data_as(C.c_void_p)  # noqa: E731

    def call(recs, dtype=1, lay=layer, n=None, ws_bytes=wsb, wsp=ws, hits=None):
        n = len(recs) if n is None else n
        return lib.lcl_select_sphere(C.byref(a), lay, dtype, P(recs), n, hits, wsp, ws_bytes, None)

    bad = good.copy(); bad[2]["label"] = 256
    assert call(bad) == 1                                     # label does not fit uint8
    bad = good.copy(); bad[1]["r2"] = -1
    assert call(bad) == 1
    bad = good.copy(); bad[0]["flags"] = 9                     # padding radius above 8
    assert call(bad) == 1
    bad = good.copy(); bad[0]["flags"] = 1 << 8                # undefined flag bit
    assert call(bad) == 1
    bad = good.copy(); bad[3]["cx"] = 1 << 23
    assert call(bad) == 1                                     # centre outside the accepted range
    assert call(good, dtype=3) == 1                           # bad dtype
    assert call(good, lay=C.c_void_p((1 << 41) + 4)) == 1     # layer not 16-byte aligned
    assert call(good, ws_bytes=wsb - 1) == 2                  # workspace too small
    assert call(good, wsp=C.c_void_p((1 << 42) + 8)) == 1     # workspace misaligned
    assert call(good, n=-1) == 1
    assert call(good, hits=C.c_void_p((1 << 43) + 4)) == 1    # hits not 8-byte aligned
    assert "aligned" in lcl.lcl_last_error()


def test_static_sphere_checks_arguments_like_the_workspace_entry_point(lcl):
    """lcl_select_sphere_static runs lcl_select_sphere's argument checks before its own size limits:
    a bad atlas, label or layer gives the same status from both, and only valid calls beyond the
    scratch array's limits get LCL_ERR_UNSUPPORTED (host-side checks only, nothing is launched)."""
    lib, a = _bound(lcl)
    layer, ws = C.c_void_p(1 << 41), C.c_void_p(1 << 42)
    wsb = lib.lcl_select_workspace_bytes(C.byref(a), 4)
    good = np.zeros(4, lcl.SPHERE_DTYPE)
    P = lambda r: r.ctypes.data_as(C.c_void_p)  # noqa: E731

    def both(atlas, recs, dtype=1, lay=layer):
        ws_st = lib.lcl_select_sphere(C.byref(atlas), lay, dtype, P(recs), len(recs), None, ws, wsb, None)
        st_st = lib.lcl_select_sphere_static(C.byref(atlas), lay, dtype, P(recs), len(recs), None, None)
        return ws_st, st_st

    bad = good.copy(); bad[2]["label"] = 256
    assert both(a, bad) == (1, 1)
    assert both(a, good, dtype=3) == (1, 1)
    assert both(a, good, lay=C.c_void_p((1 << 41) + 4)) == (1, 1)
    # an unbound atlas whose tile counts exceed the array: the atlas check answers first
    junk = lcl.lcl_atlas()
    junk.tiles_x, junk.tiles_y = 4096, 4096
    assert lib.lcl_select_sphere_static(C.byref(junk), layer, 1, P(good), 4, None, None) == 1
    assert lib.lcl_select_sphere_static(C.byref(a), layer, 1, P(good), 0, None, None) == 0   # nothing to do
    many = np.zeros(4097, lcl.SPHERE_DTYPE)
    assert lib.lcl_select_sphere_static(C.byref(a), layer, 1, P(many), 4097, None, None) == 4
    assert "4096" in lcl.lcl_last_error()


def test_lasso_and_layer_ops_reject_bad_arguments(lcl):
    lib, a = _bound(lcl)
    cam = lcl.lcl_camera()
    cam.width, cam.height = 64, 48
    for i in range(16):
        cam.m[i] = 1.0 if i % 5 == 0 else 0.0
    poly = np.zeros((3, 2), np.float32)
    P = lambda r: r.ctypes.data_as(C.c_void_p)  # noqa: E731
    dptr, lay, ws = C.c_void_p(1 << 41), C.c_void_p(1 << 42), C.c_void_p(1 << 43)
    wsb = lib.lcl_select_workspace_bytes(C.byref(a), 1)
    args = lambda p, n, label=5, dt=1, bias=0.001, c=cam, fl=0: (C.byref(a), lay, dt, C.byref(c), dptr, P(p), n,  # noqa
                                                                 label, fl, C.c_float(bias), None, ws, wsb, None)
    assert lib.lcl_select_lasso(*args(np.zeros((2, 2), np.float32), 2)) == 4       # too few vertices
    assert lib.lcl_select_lasso(*args(np.zeros((65, 2), np.float32), 65)) == 4     # too many
    nanp = poly.copy(); nanp[1, 0] = np.nan
    assert lib.lcl_select_lasso(*args(nanp, 3)) == 1
    assert lib.lcl_select_lasso(*args(poly, 3, label=300)) == 1
    assert lib.lcl_select_lasso(*args(poly, 3, bias=float("inf"))) == 1
    assert lib.lcl_select_lasso(*args(poly, 3, fl=9)) == 1                          # padding radius above 8
    assert lib.lcl_select_lasso(*args(poly, 3, fl=1 << 8)) == 1                     # undefined flag bit
    badcam = lcl.lcl_camera.from_buffer_copy(cam); badcam.m[3] = float("nan")
    assert lib.lcl_select_lasso(*args(poly, 3, c=badcam)) == 1
    badcam = lcl.lcl_camera.from_buffer_copy(cam); badcam.width = 0
    assert lib.lcl_select_lasso(*args(poly, 3, c=badcam)) == 1
    # overlay / area
    assert lib.lcl_overlay(C.byref(a), lay, lay, lay, 1, 7, 0, None) == 1             # unknown op
    assert lib.lcl_overlay(C.byref(a), lay, lay, lay, 1, 0, 8, None) == 1             # unknown flag
    assert lib.lcl_overlay(C.byref(a), C.c_void_p((1 << 42) + 1), lay, lay, 1, 0, 0, None) == 1
    assert lib.lcl_label_area(C.byref(a), lay, 1, 0, dptr, dptr, None) == 1          # n_labels = 0
    assert lib.lcl_label_area(C.byref(a), lay, 1, 65537, dptr, dptr, None) == 1
    assert lib.lcl_label_area(C.byref(a), lay, 2, 16, C.c_void_p((1 << 41) + 4), dptr, None) == 1


def test_atlas_build_and_helpers_reject_bad_arguments(lcl):
    lib, a = _bound(lcl, n=10)
    m = lcl.lcl_mesh(1 << 40, 30, 1 << 41, 30, 1 << 42, 1 << 43, 11)   # triangle count differs from the atlas
    ws = C.c_void_p(1 << 44)
    assert lib.lcl_atlas_build(C.byref(m), C.byref(a), ws, 1 << 30, None) == 1
    m.n_tri = 10
    m.n_pos = 0
    assert lib.lcl_atlas_build(C.byref(m), C.byref(a), ws, 1 << 30, None) == 1
    m.n_pos = 30
    assert lib.lcl_atlas_build(C.byref(m), C.byref(a), C.c_void_p((1 << 44) + 64), 1 << 30, None) == 1
    v = lcl.lcl_atlas()
    assert lib.lcl_atlas_rows(C.byref(a), 0, 32, C.byref(v)) == 0
    assert lib.lcl_atlas_build(C.byref(m), C.byref(v), ws, 1 << 30, None) == 1       # a view
    # helpers need a built atlas (scale > 0)
    s = lcl.lcl_sphere()
    c3 = (C.c_double * 3)(0, 0, 0)
    assert lib.lcl_quantize_sphere(C.byref(a), c3, 1.0, 1, C.byref(s)) == 1
    a.scale = 1000.0
    assert lib.lcl_quantize_sphere(C.byref(a), c3, 0.5, 7, C.byref(s)) == 0
    assert (s.cx, s.r2, s.label) == (0, 250000, 7)
    assert lib.lcl_quantize_sphere(C.byref(a), c3, -1.0, 1, C.byref(s)) == 1
    assert lib.lcl_quantize_sphere(C.byref(a), (C.c_double * 3)(1e5, 0, 0), 1.0, 1, C.byref(s)) == 1
    vp = (C.c_double * 16)(*np.eye(4).ravel())
    cam = lcl.lcl_camera()
    assert lib.lcl_camera_from_vp(C.byref(a), vp, 0, 10, C.byref(cam)) == 1
    assert lib.lcl_camera_from_vp(C.byref(a), vp, 10, 10, C.byref(cam)) == 0
    assert cam.m[0] == np.float32(1e-3) and cam.m[15] == 1.0


def test_host_helpers_match_oracle_without_gpu(lcl):
    """The library's host-only helpers (stroke quantisation, camera composition) against the
    oracle's independent ones, on a bbox/scale taken from the oracle."""
    import oracle
    import synth
    mesh = synth.config_small().mesh
    mn, S = oracle.quant_params(mesh.pos)
    lib, a = _bound(lcl)
    for i in range(3):
        a.bbox_min[i] = float(mn[i])
    a.scale = S
    st = synth.sphere_strokes(mesh, 100, 9, 0.001, 0.5, 1, 255)
    for k in range(100):
        s = lcl.lcl_sphere()
        c3 = (C.c_double * 3)(*st.centre[k])
        assert lib.lcl_quantize_sphere(C.byref(a), c3, float(st.radius[k]), int(st.label[k]), C.byref(s)) == 0
        e = oracle.sphere_stroke(mn, S, st.centre[k], st.radius[k], st.label[k])
        assert (s.cx, s.cy, s.cz, s.r2, s.label) == (e["cx"], e["cy"], e["cz"], e["r2"], e["label"])
    rng = np.random.default_rng(1)
    for _ in range(10):
        cam = synth.orbit_camera(mesh, 800, 600, rng)
        out = lcl.lcl_camera()
        vp = (C.c_double * 16)(*cam.vp.ravel())
        assert lib.lcl_camera_from_vp(C.byref(a), vp, 800, 600, C.byref(out)) == 0
        assert np.array_equal(np.array(list(out.m), np.float32), oracle.camera_mq(cam.vp, mn, S))


def test_tool_rejects_bad_arguments(lcl):
    lib, a = _bound(lcl)
    cam = lcl.lcl_camera()
    cam.width, cam.height = 64, 48
    for i in range(16):
        cam.m[i] = 1.0 if i % 5 == 0 else 0.0
    dptr, lay, ws = C.c_void_p(1 << 41), C.c_void_p(1 << 42), C.c_void_p(1 << 43)
    wsb = lib.lcl_select_workspace_bytes(C.byref(a), 1)

    def call(tool, label=5, bias=0.001, wsb=wsb):
        return lib.lcl_select_tool(C.byref(a), lay, 1, C.byref(cam), dptr, C.byref(tool) if tool else None, label,
                                   C.c_float(bias), None, ws, wsb, None)

    def tool(px=10.0, py=10.0, tw=8.0, th=8.0, shape=None, sw=0, sh=0):
        t = lcl.lcl_tool()
        t.px, t.py, t.tw, t.th, t.shape, t.shape_w, t.shape_h = px, py, tw, th, shape, sw, sh
        return t

    assert call(None) == 1                                         # no tool
    for bad in (tool(tw=0.0), tool(th=-2.0), tool(px=float("nan")), tool(tw=float("inf")), tool(py=2e7)):
        assert call(bad) == 1                                      # window not finite / positive / bounded
    assert call(tool(shape=1 << 40, sw=0, sh=4)) == 1              # shape sizes
    assert call(tool(shape=1 << 40, sw=4, sh=5000)) == 1
    for f in (9, 9 << 4, 1 << 8):
        bad = tool()
        bad.flags = f
        assert call(bad) == 1                                      # padding flags out of range
    assert call(tool(), label=256) == 1                            # label too wide for uint8
    assert call(tool(), bias=float("nan")) == 1
    assert call(tool(), wsb=16) == 2                               # workspace too small


def test_batch_rejects_bad_arguments_on_host(lcl):
    lib, a = _bound(lcl, W=128, H=128, T=32)
    ws, stg = C.c_void_p(1 << 42), (C.c_uint8 * 4096)()
    models = (lcl.lcl_batch_model * 1)()
    models[0].atlas = C.pointer(a)
    models[0].layer = 1 << 41
    models[0].dtype = 1
    models[0].first_stroke = 0
    models[0].n_strokes = 65
    strokes = (lcl.lcl_batch_stroke * 65)()
    lassos = (lcl.lcl_batch_lasso * 1)()
    lim = lcl.batch_limits(models=1, strokes=65, lassos=1, supers=a.supers_x * a.supers_y, tiles=a.tiles_x * a.tiles_y)
    call = lambda n_strokes=65, n_lassos=0, limits=lim: lib.lcl_batch_upload(  # noqa
        C.byref(limits), models, 1, strokes, n_strokes, lassos, n_lassos, ws, 1 << 30, stg, 4096, None)
    assert call() == 4                                   # more than 64 strokes for one model
    models[0].n_strokes = 10
    assert call(n_strokes=5) == 1                        # stroke range outside the array
    strokes[3].kind = 7
    assert call() == 1                                   # unknown stroke kind
    strokes[3].kind = 1
    strokes[3].lasso = 0
    assert call() == 1                                   # lasso index with no lassos
    strokes[3].kind = 0
    strokes[4].sphere.label = 300
    assert call() == 1                                   # label too wide for uint8
    strokes[4].sphere.label = 3
    strokes[5].sphere.flags = 9
    assert call() == 1                                   # padding radius above 8
    strokes[5].sphere.flags = 1 << 8
    assert call() == 1                                   # undefined flag bit
    strokes[5].sphere.flags = 0
    models[0].layer = (1 << 41) + 8
    assert call() == 1                                   # layer misaligned
    models[0].layer = 1 << 41
    small = lcl.batch_limits(models=1, strokes=8, lassos=1, supers=lim.supers, tiles=lim.tiles)
    assert call(limits=small) == 1                       # more strokes than the workspace limits
    tiny = lcl.batch_limits(models=1, strokes=65, lassos=1, supers=lim.supers, tiles=lim.tiles - 1)
    assert call(limits=tiny) == 1                        # more tiles than the limits
    assert call() == 2                                   # staging too small for the descriptors
    assert lib.lcl_batch_workspace_bytes(C.byref(lim)) > lib.lcl_batch_staging_bytes(C.byref(lim)) > 4096
    bad = lcl.batch_limits(models=-1)
    assert lib.lcl_batch_workspace_bytes(C.byref(bad)) == 0
    own = lcl.lcl_batch_limits()
    assert lib.lcl_batch_limits_of(models, 1, 65, 0, C.byref(own)) == 0
    assert (own.models, own.strokes, own.lassos, own.supers, own.tiles) == (1, 65, 0, lim.supers, lim.tiles)
    # launch shapes are checked before anything is enqueued
    for cfg in (lcl.batch_config(threads=96), lcl.batch_config(split=3), lcl.batch_config(ctas_per_sm=33),
                lcl.batch_config(threads=0, split=0)):
        assert lib.lcl_batch_launch(C.byref(lim), C.byref(cfg), ws, 1 << 30, None) == 1
    assert lib.lcl_batch_launch(C.byref(lim), None, ws, 16, None) == 1      # workspace smaller than the limits
    best, ms = lcl.lcl_batch_config(), C.c_float()
    assert lib.lcl_batch_tune(C.byref(lim), ws, 1 << 30, 0, None, C.byref(best), C.byref(ms)) == 1  # reps < 1


def test_numeric_layers_reject_bad_arguments(lcl):
    lib, a = _bound(lcl)
    P = lambda r: r.ctypes.data_as(C.c_void_p)  # noqa: E731
    data, mask = 1 << 41, 1 << 42
    ws = C.c_void_p(1 << 43)
    wsb = lib.lcl_select_workspace_bytes(C.byref(a), 4)

    def layer(t, d=data, m=mask):
        return lcl.lcl_numeric_layer(d, m, t, 0)

    i16, f32 = layer(lcl.NUM_TYPES["i16"]), layer(lcl.NUM_TYPES["f32"])
    good = np.zeros(4, lcl.SPHERE_DTYPE)

    def sphere(recs, lay=i16):
        return lib.lcl_numeric_sphere(C.byref(a), C.byref(lay), P(recs), len(recs), None, ws, wsb, None)

    bad = good.copy(); bad[0]["label"] = 1 << 16
    assert sphere(bad) == 1                                           # value wider than int16
    bad = good.copy(); bad[1]["flags"] = 0x200
    assert sphere(bad) == 1                                           # unknown flag bit
    assert sphere(good, layer(0x13)) == 1                             # unknown type
    assert sphere(good, layer(lcl.NUM_TYPES["i16"], d=data + 4)) == 1  # data misaligned
    assert sphere(good, layer(lcl.NUM_TYPES["i16"], m=0)) == 1        # no mask
    # arithmetic
    ar = lambda x, y, o, op, s=0: lib.lcl_numeric_arith(C.byref(a), C.byref(x), None if y is None else C.byref(y),  # noqa
                                                        s, C.byref(o), op, None)
    assert ar(i16, f32, i16, 0) == 1                                  # types differ
    assert ar(i16, i16, i16, 3) == 4                                  # integer division
    assert ar(i16, i16, i16, 6) == 1                                  # unknown op
    assert ar(i16, None, i16, 0, 1 << 16) == 1                        # scalar wider than the type
    # selection by value and statistics
    lay = C.c_void_p(1 << 44)
    assert lib.lcl_numeric_select(C.byref(a), C.byref(f32), 6, 0, lay, 1, 1, None, None) == 1   # unknown cmp
    assert lib.lcl_numeric_select(C.byref(a), C.byref(i16), 0, 1 << 16, lay, 1, 1, None, None) == 1
    assert lib.lcl_numeric_select(C.byref(a), C.byref(f32), 0, 0, lay, 1, 256, None, None) == 1  # label > u8
    out = C.c_void_p(1 << 45)
    assert lib.lcl_numeric_stats(C.byref(a), C.byref(f32), None, 0, 2, out, None) == 1   # no zones, 2 labels
    assert lib.lcl_numeric_stats(C.byref(a), C.byref(f32), lay, 1, 0, out, None) == 1    # n_labels 0
    assert lib.lcl_numeric_stats(C.byref(a), C.byref(f32), lay, 3, 4, out, None) == 1    # zone dtype


def test_pool_rejects_bad_arguments_on_host(lcl):
    lib = lcl.library()
    p = C.c_void_p()
    assert lib.lcl_pool_create(0, C.byref(p)) == 1                  # no slots
    assert lib.lcl_pool_create(1 << 21, C.byref(p)) == 1            # too many slots
    assert lib.lcl_pool_create(4, None) == 1
    rec = lcl.lcl_pool_layer()
    assert lib.lcl_pool_acquire(None, 64, 64, 1, None, C.byref(rec)) == 1
    assert lib.lcl_pool_release(None, 0, None) == 1
    st = lcl.lcl_pool_stats()
    assert lib.lcl_pool_stats_get(None, C.byref(st)) == 1
    assert lib.lcl_pool_destroy(None) == 0


def _site(name, line):
    """A bounds-check site as the kernels record it: 16-bit fold of the FNV-1a hash of the file
    name (after the last '/') above the line number."""
    h = 2166136261
    for c in name.encode():
        h = ((h ^ c) * 16777619) & 0xFFFFFFFF
    return (((h ^ (h >> 16)) & 0xFFFF) << 16) | (line & 0xFFFF)


def test_device_status_sites_decode_to_file_and_line(lcl):
    names = ["atlas.cu", "batch.cu", "depth.cu", "layers.cu", "numeric.cu", "select.cu", "noalloc.cu",
             "lcl_api.cu", "pool.cu", "select_common.cuh", "lcl_impl.cuh"]
    assert len({_site(n, 0) for n in names}) == len(names)          # no two files share a hash
    for i, n in enumerate(names):
        assert lcl.lcl_describe_site(_site(n, 17 + i)) == f"{n}:{17 + i}"
    unknown = _site("elsewhere.cu", 9)
    assert lcl.lcl_describe_site(unknown) == f"file#{unknown >> 16:04x}:9"
    lib = lcl.library()
    assert lib.lcl_describe_site(_site("select.cu", 123), None, 0) == len("select.cu:123")
    buf = C.create_string_buffer(5)
    lib.lcl_describe_site(_site("select.cu", 123), buf, 5)
    assert buf.value == b"sele"                                        # truncated, NUL-terminated


def test_debug_build_reports_bounds_checks(lcl):
    """liblcl.so has no bounds checks; liblcl_debug.so (built by the same build()) has them."""
    from paper_2501_14807_gb300 import build
    assert lcl.lcl_build_flags() & lcl.LCL_BUILD_BOUNDS_CHECKS == 0
    if not os.path.exists(lcl.DEBUG_LIB_PATH):
        build.build(debug=True)
    dbg = C.CDLL(lcl.DEBUG_LIB_PATH)
    dbg.lcl_build_flags.restype = C.c_uint32
    assert dbg.lcl_build_flags() == lcl.LCL_BUILD_BOUNDS_CHECKS
    missing = [n for n in declared_functions() if not hasattr(dbg, n)]
    assert not missing


def test_device_status_without_a_gpu_is_a_cuda_error(lcl):
    import torch
    if torch.cuda.is_available():
        pytest.skip("checks the no-device answer")
    assert lcl.library().lcl_last_device_status(None) == 3           # LCL_ERR_CUDA: nothing to synchronise
    assert "lcl_last_device_status" in lcl.lcl_last_error()
