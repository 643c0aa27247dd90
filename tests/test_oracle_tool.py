"""Pins of the oracle's editing tool (Section 4.3.1: depth test, projection into the tool window,
shape mask), against exact rationals at the projected point and against the independently pinned
lasso oracle on polygons that bound or equal the tool's shape.  CPU only."""
from fractions import Fraction as F

import numpy as np
import pytest

import oracle
import synth
from test_oracle_edits import _lasso_setup, project32, screen32

BIAS = 2.0 ** -10


def _projected(a, M, Ws, Hs):
    c = project32(M, a.px, a.py, a.pz)
    with np.errstate(all="ignore"):
        zn = c[2] / c[3]
        xs = screen32(c[0] / c[3], Ws)
        ys = screen32(c[1] / c[3], Hs)
    return c[3], zn, xs, ys


def _visible(dmap, zn, x, y):
    dref = dmap[int(y), int(x)]
    return bool(np.isinf(dref) or F(float(zn)) <= F(float(dref)) + F(BIAS))


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_tool_circle_matches_exact_ellipse_test(seed):
    """An off-centre tool with tw != th: the inscribed ellipse, tested in exact rationals at the
    FP32 screen point, must agree with the oracle except on texels it flags as ambiguous."""
    m, a, M, dmap = _lasso_setup(seed)
    Hs, Ws = dmap.shape
    rng = np.random.default_rng(seed)
    px, py = np.float32(Ws * rng.uniform(0.35, 0.6)), np.float32(Hs * rng.uniform(0.35, 0.6))
    tw, th = np.float32(Ws * 0.55), np.float32(Hs * 0.35)
    layer = np.zeros(a.tri.shape, np.uint8)
    hits, amb = oracle.select_tool(a, layer, M, dmap, (px, py), (tw, th), None, 7, BIAS)
    w, zn, xs, ys = _projected(a, M, Ws, Hs)
    exp = np.zeros(a.tri.shape, bool)
    for j, i in np.argwhere(a.covered()):
        if not (w[j, i] > 0 and 0 <= zn[j, i] <= 1 and 0 <= xs[j, i] < Ws and 0 <= ys[j, i] < Hs):
            continue
        ex = (F(float(xs[j, i])) - F(float(px))) * 2 / F(float(tw))
        ey = (F(float(ys[j, i])) - F(float(py))) * 2 / F(float(th))
        exp[j, i] = ex * ex + ey * ey <= 1 and _visible(dmap, zn[j, i], xs[j, i], ys[j, i])
    got = layer == 7
    assert not ((got != exp) & (amb == 0)).any()
    assert hits == got.sum() and hits > 20
    # the ellipse is not symmetric in its axes: swapping tw and th changes the selection
    swapped = np.zeros(a.tri.shape, np.uint8)
    oracle.select_tool(a, swapped, M, dmap, (px, py), (th, tw), None, 7, BIAS)
    assert (swapped != layer).sum() > 5


def _ngon(cx, cy, r, n=64):
    t = 2 * np.pi * (np.arange(n) + 0.5) / n
    return np.stack([cx + r * np.cos(t), cy + r * np.sin(t)], -1).astype(np.float32)


@pytest.mark.parametrize("seed", [3, 4])
def test_tool_circle_lies_between_inscribed_and_circumscribed_polygons(seed):
    m, a, M, dmap = _lasso_setup(seed)
    Hs, Ws = dmap.shape
    cx, cy, r = np.float32(Ws * 0.47), np.float32(Hs * 0.52), 0.3 * Ws
    tool = np.zeros(a.tri.shape, np.uint8)
    _, amb_t = oracle.select_tool(a, tool, M, dmap, (cx, cy), (np.float32(2 * r), np.float32(2 * r)), None, 1, BIAS)
    inner = np.zeros(a.tri.shape, np.uint8)
    outer = np.zeros(a.tri.shape, np.uint8)
    _, amb_i = oracle.select_lasso(a, inner, M, dmap, _ngon(cx, cy, r * 0.999), 1, BIAS)
    _, amb_o = oracle.select_lasso(a, outer, M, dmap, _ngon(cx, cy, r / np.cos(np.pi / 64) * 1.001), 1, BIAS)
    sure = (amb_t == 0) & (amb_i == 0) & (amb_o == 0)
    assert not ((inner == 1) & (tool == 0) & sure).any()
    assert not ((tool == 1) & (outer == 0) & sure).any()
    assert (tool == 1).sum() >= (inner == 1).sum() > 20


def _rect(x0, y0, x1, y1):
    return np.array([[x0, y0], [x1, y0], [x1, y1], [x0, y1]], np.float32)


@pytest.mark.parametrize("seed", [5, 6])
def test_tool_masks_select_the_matching_window_parts(seed):
    """A full mask selects the whole window, a mask whose bottom rows are set the bottom part of
    the window (row 0 at the bottom), one whose left columns are set the left part: each equal to
    the lasso over that rectangle (half-open like the window), except on flagged texels."""
    m, a, M, dmap = _lasso_setup(seed)
    Hs, Ws = dmap.shape
    px, py, tw, th = np.float32(Ws * 0.51 + 0.13), np.float32(Hs * 0.48 + 0.29), np.float32(24.5), np.float32(17.5)
    x0, y0 = float(px) - float(tw) / 2, float(py) - float(th) / 2
    x1, y1 = x0 + float(tw), y0 + float(th)
    H_m, W_m = 8, 10
    cases = {
        "full": (np.ones((H_m, W_m), np.uint8), _rect(x0, y0, x1, y1)),
        "bottom": (np.vstack([np.ones((3, W_m)), np.zeros((H_m - 3, W_m))]).astype(np.uint8),
                   _rect(x0, y0, x1, y0 + float(th) * 3 / H_m)),
        "left": (np.hstack([np.ones((H_m, 4)), np.zeros((H_m, W_m - 4))]).astype(np.uint8),
                 _rect(x0, y0, x0 + float(tw) * 4 / W_m, y1)),
    }
    sel = {}
    for name, (shape, poly) in cases.items():
        t = np.zeros(a.tri.shape, np.uint8)
        _, amb_t = oracle.select_tool(a, t, M, dmap, (px, py), (tw, th), shape, 3, BIAS)
        l = np.zeros(a.tri.shape, np.uint8)
        _, amb_l = oracle.select_lasso(a, l, M, dmap, poly, 3, BIAS)
        assert not ((t != l) & (amb_t == 0) & (amb_l == 0)).any(), name
        sel[name] = t == 3
    assert sel["full"].sum() > sel["bottom"].sum() > 0 and sel["full"].sum() > sel["left"].sum() > 0
    assert not (sel["bottom"] & ~sel["full"]).any() and not (sel["left"] & ~sel["full"]).any()


def test_tool_depth_test_rejects_occluded_texels():
    """The two-squares scene of the lasso pin: a tool over the whole screen selects the front
    square's texels and none of the back square's."""
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
    full = np.ones((2, 2), np.uint8)
    layer = np.zeros(a.tri.shape, np.uint8)
    hits, _ = oracle.select_tool(a, layer, M, dmap, (16.0, 16.0), (31.0, 31.0), full, 9, BIAS)
    front = a.covered() & (a.tri <= 1)
    back = a.covered() & (a.tri >= 2)
    assert front.sum() > 0 and back.sum() > 0
    assert (layer[front] == 9).all() and (layer[back] == 0).all() and hits == front.sum()
    # without geometry in front (depth cleared to +inf) the back square is selected as well
    lay2 = np.zeros(a.tri.shape, np.uint8)
    oracle.select_tool(a, lay2, M, np.full_like(dmap, np.inf), (16.0, 16.0), (31.0, 31.0), full, 9, BIAS)
    assert (lay2[back] == 9).all()


def test_tool_rejects_bad_arguments():
    m, a, M, dmap = _lasso_setup(0)
    layer = np.zeros(a.tri.shape, np.uint8)
    for size in ((0.0, 5.0), (5.0, -1.0)):
        with pytest.raises(oracle.OracleError):
            oracle.select_tool(a, layer, M, dmap, (3.0, 3.0), size)
    with pytest.raises(oracle.OracleError):
        oracle.select_tool(a, layer, M, dmap, (3.0, 3.0), (5.0, 5.0), None, 256)


@pytest.mark.parametrize("rad,thick", [(1, 1), (2, 1), (3, 4), (8, 8), (0, 5)])
def test_tool_padding_matches_dilations(rad, thick):
    """Texture padding of a tool edit: uncovered texels within `thickness` of a covered texel
    (square kernel) and within `radius` of a selected texel get the label -- square-kernel
    dilations with scipy; radius 0 pads nothing."""
    ndimage = pytest.importorskip("scipy.ndimage")
    m = synth.vessel_charts(60, 30, 12, 6, 96, seed=2)
    a = oracle.Atlas(m, 96, 96, tile=16)
    Ws, Hs = 64, 48
    cam = synth.orbit_camera(m, Ws, Hs, np.random.default_rng(9))
    M = oracle.camera_mq(cam.vp, a.mn, a.S)
    dmap = oracle.depth(m, a.mn, a.S, M, Ws, Hs)
    centre, size = (Ws * 0.5, Hs * 0.5), (Ws * 0.8, Hs * 0.9)
    plain = np.zeros(a.tri.shape, np.uint8)
    h0, amb0 = oracle.select_tool(a, plain, M, dmap, centre, size, None, 4, BIAS)
    sel = plain == 4
    lay = np.zeros(a.tri.shape, np.uint8)
    h, npad, amb = oracle.select_tool_2d(a, lay, M, dmap, centre, size, None, 4, BIAS, oracle.pad_flags(rad, thick))
    cov = a.covered()
    if rad == 0:
        exp_pad = np.zeros_like(cov)
    else:
        outline = ~cov & ndimage.maximum_filter(cov, size=2 * thick + 1, mode="constant")
        exp_pad = outline & ndimage.maximum_filter(sel, size=2 * rad + 1, mode="constant")
    assert h == h0 and np.array_equal(amb[cov], amb0[cov])
    assert np.array_equal(lay == 4, sel | exp_pad) and npad == exp_pad.sum()
    assert h0 > 50 and (rad == 0 or npad > 0)


def test_tool_padding_rejects_bad_flags():
    m, a, M, dmap = _lasso_setup(0)
    layer = np.zeros(a.tri.shape, np.uint8)
    for f in (9, 9 << 4, 1 << 8):
        with pytest.raises(oracle.OracleError):
            oracle.select_tool_2d(a, layer, M, dmap, (3.0, 3.0), (5.0, 5.0), None, 1, BIAS, f)
