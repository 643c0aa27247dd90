"""Pins of the oracle's edits: sphere brush, camera composition, depth map and lasso,
against brute force in exact rationals, closed forms and invariants.  CPU only."""
from fractions import Fraction as F

import numpy as np
import pytest

import brute
import oracle
import synth

BIAS = 2.0 ** -10


@pytest.fixture(scope="module")
def small():
    m = synth.vessel_cylindrical(48, 16, noise_amp=0.02, seed=3)
    return m, oracle.Atlas(m, 96, 64, tile=32)


def last_hit_labels(a, layer0, recs):
    """Final labels as 'label of the last stroke whose ball holds the texel', vectorised."""
    q = np.stack([a.px, a.py, a.pz], -1).astype(np.int64)
    cov = a.covered()
    out = layer0.copy()
    best = np.full(layer0.shape, -1)
    for k, s in enumerate(recs):
        d2 = ((q - np.array([s["cx"], s["cy"], s["cz"]], np.int64)) ** 2).sum(-1)
        best[(d2 <= s["r2"]) & cov] = k
    sel = best >= 0
    out[sel] = recs["label"][best[sel]]
    return out


@pytest.mark.parametrize("dtype", [np.uint8, np.uint16])
def test_sphere_strokes_last_hit_wins(small, dtype):
    m, a = small
    st = synth.sphere_strokes(m, 40, 5, 0.03, 0.3, 1, 200 if dtype == np.uint8 else 60000)
    recs = oracle.sphere_records(a.mn, a.S, st.centre, st.radius, st.label)
    layer = np.random.default_rng(1).integers(0, 50, size=a.tri.shape).astype(dtype)
    exp = last_hit_labels(a, layer, recs)
    hits = oracle.select_sphere(a, layer, recs)
    assert np.array_equal(layer, exp)
    q = np.stack([a.px, a.py, a.pz], -1).astype(np.int64)
    for k, s in enumerate(recs):
        d2 = ((q - np.array([s["cx"], s["cy"], s["cz"]])) ** 2).sum(-1)
        assert hits[k] == ((d2 <= s["r2"]) & a.covered()).sum()


def test_sphere_outside_unchanged_and_uncovered_untouched(small):
    m, a = small
    layer = np.full(a.tri.shape, 7, np.uint8)
    big = np.zeros(1, oracle.SPHERE_DTYPE)
    big["cx"], big["cy"], big["cz"], big["r2"], big["label"] = 1 << 20, 1 << 20, 1 << 20, 1 << 50, 9
    h = oracle.select_sphere(a, layer, big)
    assert h[0] == a.covered().sum()
    assert (layer[a.covered()] == 9).all() and (layer[~a.covered()] == 7).all()


def test_sphere_zero_radius_hits_exact_position(small):
    m, a = small
    cov = np.argwhere(a.covered())
    j, i = cov[len(cov) // 2]
    s = np.zeros(1, oracle.SPHERE_DTYPE)
    s["cx"], s["cy"], s["cz"], s["r2"], s["label"] = a.px[j, i], a.py[j, i], a.pz[j, i], 0, 3
    layer = np.zeros(a.tri.shape, np.uint8)
    oracle.select_sphere(a, layer, s)
    same = (a.px == a.px[j, i]) & (a.py == a.py[j, i]) & (a.pz == a.pz[j, i]) & a.covered()
    assert np.array_equal(layer == 3, same) and same[j, i]


def test_sphere_stroke_quantisation(small):
    m, a = small
    q = oracle.quantize(m.pos, a.mn, a.S)
    for v in (0, 17, 301):
        s = oracle.sphere_stroke(a.mn, a.S, m.pos[v].astype(np.float64), 0.0, 1)
        assert [s["cx"], s["cy"], s["cz"]] == q[v].tolist() and s["r2"] == 0
    rng = np.random.default_rng(3)
    for r in rng.uniform(0, 3, size=50):
        s = oracle.sphere_stroke(a.mn, a.S, [0.0, 0.0, 0.0], r, 1)
        exact = (F(float(r)) * F(a.S)) ** 2
        assert abs(s["r2"] - int(exact)) <= 1
    with pytest.raises(oracle.OracleError):
        oracle.sphere_stroke(a.mn, a.S, [1e6, 0, 0], 1.0, 1)      # centre far outside the grid
    with pytest.raises(oracle.OracleError):
        oracle.select_sphere(a, np.zeros(a.tri.shape, np.uint8),
                             np.array([(0, 0, 0, 0, 5, 256, 0)], oracle.SPHERE_DTYPE))  # label too wide


def test_camera_composition_within_one_ulp():
    m = synth.vessel_cylindrical(20, 6, seed=1)
    mn, S = oracle.quant_params(m.pos)
    cam = synth.orbit_camera(m, 64, 48, np.random.default_rng(4))
    M = oracle.camera_mq(cam.vp, mn, S)
    for i in range(4):
        for j in range(4):
            if j < 3:
                ex = F(float(cam.vp[i, j])) / F(S)
            else:
                ex = sum(F(float(cam.vp[i, k])) * F(float(mn[k])) for k in range(3)) + F(float(cam.vp[i, 3]))
            got = M[4 * i + j]
            assert abs(F(float(got)) - ex) <= F(float(np.spacing(np.float32(abs(got)))))


def project32(M, qx, qy, qz):
    """FP32 clip coordinates in the stated order, vectorised in numpy float32."""
    M = np.asarray(M, np.float32)
    x, y, z = (np.asarray(v).astype(np.float32) for v in (qx, qy, qz))
    return [((M[4 * r] * x + M[4 * r + 1] * y) + M[4 * r + 2] * z) + M[4 * r + 3] for r in range(4)]


def screen32(ndc, extent):
    return (ndc * np.float32(0.5) + np.float32(0.5)) * np.float32(extent)


def brute_depth(m, mn, S, M, Ws, Hs):
    q = oracle.quantize(m.pos, mn, S)
    best = [[None] * Ws for _ in range(Hs)]
    for t in range(m.n_tri):
        V, Z = [], []
        for k in range(3):
            c = project32(M, *q[m.tri_pos[t, k]])
            if not c[3] > 0:
                break
            zn = c[2] / c[3]
            if not (0 <= zn <= 1):
                break
            xs = screen32(c[0] / c[3], Ws) * np.float32(256)
            ys = screen32(c[1] / c[3], Hs) * np.float32(256)
            V.append((int(np.rint(xs)), int(np.rint(ys))))
            Z.append(F(float(zn)))
        if len(V) < 3:
            continue
        for j in range(Hs):
            for i in range(Ws):
                lam, grad = brute.bary((256 * i + 128, 256 * j + 128), V)
                if lam is None or not brute.covered_nudged(lam, grad):
                    continue
                z = sum(lam[k] * Z[k] for k in range(3))
                if best[j][i] is None or z < best[j][i]:
                    best[j][i] = z
    return best


@pytest.mark.parametrize("seed", [0, 1])
def test_depth_matches_exact_brute_force(seed):
    m = synth.vessel_cylindrical(10, 4, noise_amp=0.05, seed=seed)
    mn, S = oracle.quant_params(m.pos)
    Ws, Hs = 24, 16
    cam = synth.orbit_camera(m, Ws, Hs, np.random.default_rng(seed))
    M = oracle.camera_mq(cam.vp, mn, S)
    d = oracle.depth(m, mn, S, M, Ws, Hs)
    best = brute_depth(m, mn, S, M, Ws, Hs)
    drawn = 0
    for j in range(Hs):
        for i in range(Ws):
            if best[j][i] is None:
                assert d[j, i] == np.inf
            else:
                drawn += 1
                ex = float(best[j][i])
                assert abs(float(d[j, i]) - ex) <= float(np.spacing(np.float32(ex))) + 1e-300
    assert drawn > Ws * Hs // 4


def test_depth_of_facing_plane_is_constant():
    # the square patch seen straight on by an orthographic camera: every drawn pixel has the
    # plane's NDC depth exactly (interpolating equal values)
    W = H = 64
    m = synth.uv_square_patch(W, H, k=1000)
    mn, S = oracle.quant_params(m.pos)
    view = synth.look_at((32000, 32000, 5e5), (32000, 32000, 0), up=(0, 1, 0))
    proj = synth.orthographic01(40000, 40000, 1e5, 1e6)
    M = oracle.camera_mq(proj @ view, mn, S)
    d = oracle.depth(m, mn, S, M, 48, 48)
    zc = project32(M, 0, 0, 0)
    z0 = zc[2] / zc[3]
    fin = np.isfinite(d)
    assert fin.sum() > 0.3 * d.size
    assert (d[fin] == z0).all()


def _lasso_setup(seed=0, Ws=40, Hs=32):
    m = synth.vessel_cylindrical(24, 8, noise_amp=0.05, seed=seed)
    a = oracle.Atlas(m, 64, 48, tile=16)
    cam = synth.orbit_camera(m, Ws, Hs, np.random.default_rng(seed + 10))
    M = oracle.camera_mq(cam.vp, a.mn, a.S)
    dmap = oracle.depth(m, a.mn, a.S, M, Ws, Hs)
    return m, a, M, dmap


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_lasso_matches_exact_point_in_polygon(seed):
    m, a, M, dmap = _lasso_setup(seed)
    Hs, Ws = dmap.shape
    rng = np.random.default_rng(seed)
    poly = synth.star_lasso((Ws / 2, Hs / 2), 12, 0.45 * Ws, rng)
    layer = np.zeros(a.tri.shape, np.uint8)
    hits, amb = oracle.select_lasso(a, layer, M, dmap, poly, 5, BIAS)
    c = project32(M, a.px, a.py, a.pz)
    with np.errstate(all="ignore"):
        zn = c[2] / c[3]
        xs = screen32(c[0] / c[3], Ws)
        ys = screen32(c[1] / c[3], Hs)
    exp = np.zeros(a.tri.shape, bool)
    for j, i in np.argwhere(a.covered()):
        if not (c[3][j, i] > 0 and 0 <= zn[j, i] <= 1 and 0 <= xs[j, i] < Ws and 0 <= ys[j, i] < Hs):
            continue
        dref = dmap[int(ys[j, i]), int(xs[j, i])]
        vis = np.isinf(dref) or F(float(zn[j, i])) <= F(float(dref)) + F(BIAS)
        exp[j, i] = vis and brute.pip_exact(xs[j, i], ys[j, i], poly)
    got = layer == 5
    diff = got != exp
    assert not (diff & (amb == 0)).any()
    assert hits == got.sum() and 0 < hits
    assert amb.sum() <= 2


def test_lasso_invariant_under_orientation_and_start_vertex():
    m, a, M, dmap = _lasso_setup(4)
    Hs, Ws = dmap.shape
    poly = synth.star_lasso((Ws / 2, Hs / 2), 17, 0.5 * Ws, np.random.default_rng(5))
    ref = np.zeros(a.tri.shape, np.uint8)
    _, amb = oracle.select_lasso(a, ref, M, dmap, poly, 1)
    for p in (poly[::-1].copy(), np.roll(poly, 5, axis=0)):
        lay = np.zeros(a.tri.shape, np.uint8)
        _, amb2 = oracle.select_lasso(a, lay, M, dmap, p, 1)
        d = lay != ref
        assert not (d & (amb == 0) & (amb2 == 0)).any()


def test_lasso_vertical_split_is_a_disjoint_union():
    m, a, M, dmap = _lasso_setup(6)
    Hs, Ws = dmap.shape
    x0, x1, xm, y0, y1 = 2.0, Ws - 2.0, Ws / 2 + 0.25, 1.0, Hs - 1.0
    left = np.array([[x0, y0], [xm, y0], [xm, y1], [x0, y1]], np.float32)
    right = np.array([[xm, y0], [x1, y0], [x1, y1], [xm, y1]], np.float32)
    whole = np.array([[x0, y0], [x1, y0], [x1, y1], [x0, y1]], np.float32)
    L = np.zeros(a.tri.shape, np.uint8)
    R = np.zeros(a.tri.shape, np.uint8)
    U = np.zeros(a.tri.shape, np.uint8)
    hl, _ = oracle.select_lasso(a, L, M, dmap, left, 1)
    hr, _ = oracle.select_lasso(a, R, M, dmap, right, 1)
    hu, _ = oracle.select_lasso(a, U, M, dmap, whole, 1)
    assert not ((L == 1) & (R == 1)).any()
    assert np.array_equal((L == 1) | (R == 1), U == 1) and hl + hr == hu > 0


def test_lasso_depth_test_rejects_occluded_texels():
    # Two parallel squares, front (z = 1) in the left half of the texture, a smaller back one
    # (z = 0) in the right half, seen from above by an orthographic camera, so the back square lies
    # several pixels inside the front one's silhouette: a lasso over everything selects the front
    # square's texels and none of the back square's.
    pos = np.array([[0, 0, 1], [1, 0, 1], [1, 1, 1], [0, 1, 1],
                    [0.2, 0.2, 0], [0.8, 0.2, 0], [0.8, 0.8, 0], [0.2, 0.8, 0]], np.float32)
    uv = np.array([[0.01, 0.01], [0.49, 0.01], [0.49, 0.99], [0.01, 0.99],
                   [0.51, 0.01], [0.99, 0.01], [0.99, 0.99], [0.51, 0.99]], np.float32)
    tri = np.array([[0, 1, 2], [0, 2, 3], [4, 5, 6], [4, 6, 7]], np.uint32)
    m = synth.Mesh(pos, uv, tri, tri.copy()).check()
    a = oracle.Atlas(m, 64, 32, tile=16)
    view = synth.look_at((0.5, 0.5, 3.0), (0.5, 0.5, 0.0), up=(0, 1, 0))
    proj = synth.orthographic01(0.7, 0.7, 1.0, 4.0)
    M = oracle.camera_mq(proj @ view, a.mn, a.S)
    dmap = oracle.depth(m, a.mn, a.S, M, 32, 32)
    poly = np.array([[0.5, 0.5], [31.5, 0.5], [31.5, 31.5], [0.5, 31.5]], np.float32)
    lay = np.zeros(a.tri.shape, np.uint8)
    hits, _ = oracle.select_lasso(a, lay, M, dmap, poly, 2)
    front = a.covered() & (a.tri <= 1)
    back = a.covered() & (a.tri >= 2)
    assert front.sum() > 0 and back.sum() > 0
    assert (lay[front] == 2).all() and (lay[back] == 0).all() and hits == front.sum()
    # without geometry in front (depth cleared to +inf) the back square is selected as well
    lay2 = np.zeros(a.tri.shape, np.uint8)
    oracle.select_lasso(a, lay2, M, np.full_like(dmap, np.inf), poly, 2)
    assert (lay2[back] == 2).all()


def test_lasso_vertical_edges_are_half_open():
    """A vertical edge's crossing is exactly its x, so a texel whose projected x equals a
    rectangle's left edge is inside (the crossing test is a strict x < x_edge) and one on the
    right edge is outside."""
    m, a, M, dmap = _lasso_setup(7)
    Hs, Ws = dmap.shape
    c = project32(M, a.px, a.py, a.pz)
    with np.errstate(all="ignore"):
        xs = screen32(c[0] / c[3], Ws)
        ys = screen32(c[1] / c[3], Hs)
    lay0 = np.zeros(a.tri.shape, np.uint8)
    oracle.select_lasso(a, lay0, M, dmap, np.array([[0, 0], [Ws, 0], [Ws, Hs], [0, Hs]], np.float32), 1)
    j, i = np.argwhere(lay0 == 1)[7]                    # a visible texel inside the screen
    x0, y0 = float(xs[j, i]), float(ys[j, i])
    for left, want in ((True, 1), (False, 0)):
        xa, xb = (x0, x0 + 5.0) if left else (x0 - 5.0, x0)
        rect = np.array([[xa, y0 - 3.0], [xb, y0 - 3.0], [xb, y0 + 3.0], [xa, y0 + 3.0]], np.float32)
        assert float(rect[0, 0] if left else rect[1, 0]) == x0
        lay = np.zeros(a.tri.shape, np.uint8)
        oracle.select_lasso(a, lay, M, dmap, rect, 1)
        assert lay[j, i] == want


@pytest.mark.parametrize("rad,thick", [(1, 1), (2, 1), (1, 3), (3, 2), (8, 8)])
def test_texture_padding_matches_square_kernel_dilation(rad, thick):
    """Padding (Section 4.3.2) restated with morphology: after each stroke, the uncovered texels
    within `thick` of an island (square kernel) and within `rad` of a texel the stroke selected get
    its label -- computed here with scipy's maximum filter."""
    from scipy.ndimage import maximum_filter
    m = synth.vessel_charts(200, 100, 25, 10, 256, seed=5)
    a = oracle.Atlas(m, 256, 256)
    cov = a.covered()
    st = synth.sphere_strokes(m, 6, 8, 0.03, 0.25, 1, 200)
    recs = oracle.sphere_records(a.mn, a.S, st.centre, st.radius, st.label)
    recs["flags"] = oracle.pad_flags(rad, thick)
    init = np.random.default_rng(2).integers(0, 3, size=cov.shape).astype(np.uint8)
    exp = init.copy()
    q = np.stack([a.px, a.py, a.pz], -1).astype(np.int64)
    ring = ~cov & maximum_filter(cov, size=2 * thick + 1, mode="constant", cval=False)
    exp_pad = []
    for s in recs:
        hit = cov & (((q - np.array([s["cx"], s["cy"], s["cz"]])) ** 2).sum(-1) <= s["r2"])
        pad = ring & maximum_filter(hit, size=2 * rad + 1, mode="constant", cval=False)
        exp[hit] = s["label"]
        exp[pad] = s["label"]
        exp_pad.append(int(pad.sum()))
    got = init.copy()
    hits, padded = oracle.select_sphere_2d(a, got, recs)
    assert np.array_equal(got, exp)
    assert padded.tolist() == exp_pad and sum(exp_pad) > 0


def test_texture_padding_off_and_flag_checks():
    m = synth.vessel_charts(200, 100, 25, 10, 256, seed=5)
    a = oracle.Atlas(m, 256, 256)
    st = synth.sphere_strokes(m, 4, 9, 0.05, 0.2, 1, 200)
    recs = oracle.sphere_records(a.mn, a.S, st.centre, st.radius, st.label)
    l1 = np.zeros(a.tri.shape, np.uint8)
    l2 = np.zeros(a.tri.shape, np.uint8)
    oracle.select_sphere(a, l1, recs)
    _, padded = oracle.select_sphere_2d(a, l2, recs)
    assert np.array_equal(l1, l2) and padded.sum() == 0
    for bad in (9, 9 << 4, 1 << 8):
        r = recs.copy()
        r["flags"] = bad
        with pytest.raises(oracle.OracleError):
            oracle.select_sphere_2d(a, np.zeros(a.tri.shape, np.uint8), r)
    r = recs.copy()
    r["flags"] = oracle.pad_flags(1, 1)
    with pytest.raises(oracle.OracleError):       # the flat form has no texture layout for padding
        oracle.select_sphere(a, np.zeros(a.tri.shape, np.uint8), r)


@pytest.mark.parametrize("rad,thick", [(1, 1), (2, 1), (3, 4), (8, 8), (0, 5)])
def test_lasso_padding_matches_dilations(rad, thick):
    """Texture padding of a lasso edit (Section 4.3.2, read as for sphere strokes): uncovered texels
    within `thickness` of a covered texel and within `radius` of a selected texel get the label --
    square-kernel dilations with scipy; radius 0 pads nothing; the selection itself is the plain
    lasso's, and padded texels next to an ambiguous one are flagged."""
    ndimage = pytest.importorskip("scipy.ndimage")
    m = synth.vessel_charts(60, 30, 12, 6, 96, seed=2)
    a = oracle.Atlas(m, 96, 96, tile=16)
    Ws, Hs = 64, 48
    cam = synth.orbit_camera(m, Ws, Hs, np.random.default_rng(9))
    M = oracle.camera_mq(cam.vp, a.mn, a.S)
    dmap = oracle.depth(m, a.mn, a.S, M, Ws, Hs)
    poly = synth.star_lasso((Ws / 2, Hs / 2), 14, 0.45 * Ws, np.random.default_rng(4))
    plain = np.zeros(a.tri.shape, np.uint8)
    h0, amb0 = oracle.select_lasso(a, plain, M, dmap, poly, 4, BIAS)
    sel = plain == 4
    lay = np.zeros(a.tri.shape, np.uint8)
    h, npad, amb = oracle.select_lasso_2d(a, lay, M, dmap, poly, 4, BIAS, oracle.pad_flags(rad, thick))
    cov = a.covered()
    if rad == 0:
        exp_pad = np.zeros_like(cov)
    else:
        outline = ~cov & ndimage.maximum_filter(cov, size=2 * thick + 1, mode="constant")
        exp_pad = outline & ndimage.maximum_filter(sel, size=2 * rad + 1, mode="constant")
        near_amb = outline & ndimage.maximum_filter(amb0.astype(bool), size=2 * rad + 1, mode="constant")
        assert np.array_equal(amb.astype(bool)[~cov], near_amb[~cov])
    assert h == h0 and np.array_equal(amb[cov], amb0[cov])
    assert np.array_equal(lay == 4, sel | exp_pad) and npad == exp_pad.sum()
    assert h0 > 50 and (rad == 0 or npad > 0)


def test_lasso_padding_rejects_bad_flags():
    m, a, M, dmap = _lasso_setup(0)
    layer = np.zeros(a.tri.shape, np.uint8)
    poly = np.float32([[1, 1], [20, 2], [10, 20]])
    for f in (9, 9 << 4, 1 << 8):
        with pytest.raises(oracle.OracleError):
            oracle.select_lasso_2d(a, layer, M, dmap, poly, 1, BIAS, f)
