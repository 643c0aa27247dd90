"""Pins of the oracle's atlas (quantisation, UV rasterisation, interpolation, area
weights, tile boxes, coverage bits) against brute force in exact rationals, closed
forms and library routines.  CPU only."""
import math
import os

import numpy as np
import pytest

import brute
import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def cube_mesh(lo, hi):
    c = np.array([[x, y, z] for x in (lo[0], hi[0]) for y in (lo[1], hi[1]) for z in (lo[2], hi[2])], np.float32)
    uv = np.array([[0.1, 0.1], [0.9, 0.1], [0.5, 0.9]], np.float32)
    tri = np.array([[0, 1, 2], [3, 5, 7], [4, 6, 2]], np.uint32)
    tuv = np.array([[0, 1, 2]] * 3, np.uint32)
    return synth.Mesh(c, uv, tri, tuv).check()


def test_quantize_cube_corners_map_to_grid_ends():
    m = cube_mesh((-1.5, 2.0, 0.25), (0.5, 4.0, 2.25))   # extent 2 on every axis
    mn, S = oracle.quant_params(m.pos)
    assert list(mn) == [-1.5, 2.0, 0.25]
    assert S == ((1 << 21) - 1) / 2.0
    q = oracle.quantize(m.pos, mn, S)
    assert set(np.unique(q).tolist()) == {0, (1 << 21) - 1}


def test_quantize_is_uniform_over_axes():
    m = cube_mesh((0, 0, 0), (4.0, 1.0, 2.0))
    mn, S = oracle.quant_params(m.pos)
    q = oracle.quantize(m.pos, mn, S)
    assert q[:, 0].max() == (1 << 21) - 1
    # one scale for every axis: the y and z extents map to 1/4 and 1/2 of the grid (rounded half up)
    assert q[:, 1].max() == math.floor(((1 << 21) - 1) / 4 + 0.5)
    assert q[:, 2].max() == math.floor(((1 << 21) - 1) / 2 + 0.5)


def test_quantize_rejects_flat_or_nonfinite():
    with pytest.raises(oracle.OracleError):
        oracle.quant_params(np.zeros((3, 3), np.float32))
    p = np.random.default_rng(0).normal(size=(5, 3)).astype(np.float32)
    p[2, 1] = np.nan
    with pytest.raises(oracle.OracleError):
        oracle.quant_params(p)


@pytest.mark.parametrize("seed,W,H", [(1, 16, 12), (2, 12, 16), (3, 20, 8), (4, 9, 7)])
def test_atlas_matches_exact_brute_force_on_triangle_soup(seed, W, H):
    m = synth.random_soup(14, seed)
    a = oracle.Atlas(m, W, H, tile=8)
    tri, pos = brute.atlas(m, W, H, a.mn, a.S)
    assert np.array_equal(a.tri, tri)
    assert np.array_equal(a.px, pos[0]) and np.array_equal(a.py, pos[1]) and np.array_equal(a.pz, pos[2])


def test_atlas_matches_brute_force_on_jittered_grid():
    m = synth.grid_patch(5, 4, 24, 16, seed=7, jitter=0.35)
    a = oracle.Atlas(m, 24, 16, tile=8)
    tri, pos = brute.atlas(m, 24, 16, a.mn, a.S)
    assert np.array_equal(a.tri, tri)
    assert np.array_equal(np.stack([a.px, a.py, a.pz]), pos)


def _right_triangle(n, W, H, upper, ox=0, oy=0):
    """Right triangle with legs of n texels on texel corners (ox, oy); the lower-left half of the
    n x n square, or its upper-right half."""
    if upper:
        c = [(ox + n, oy + n), (ox, oy + n), (ox + n, oy)]
    else:
        c = [(ox, oy), (ox + n, oy), (ox, oy + n)]
    uv = np.array([[x / W, y / H] for x, y in c], np.float32)
    pos = np.array([[x, y, 0.0] for x, y in c] + [[0, 0, 100.0]], np.float32)
    return synth.Mesh(pos, uv, np.array([[0, 1, 2]], np.uint32), np.array([[0, 1, 2]], np.uint32)).check()


@pytest.mark.parametrize("n", list(range(1, 13)))
def test_right_triangle_covered_count_closed_form(n):
    # Texel centres strictly inside the lower triangle: n(n-1)/2.  Its hypotenuse runs up and to
    # the left (d.y > 0), so it is not an owned edge and the n centres on it are excluded; the
    # upper-right half owns that edge (d.y < 0) and gets them: n(n+1)/2.  Together: n^2, each once.
    W, H = 32, 32
    lo = oracle.Atlas(_right_triangle(n, W, H, False, 3, 5), W, H)
    up = oracle.Atlas(_right_triangle(n, W, H, True, 3, 5), W, H)
    assert int(lo.covered().sum()) == n * (n - 1) // 2
    assert int(up.covered().sum()) == n * (n + 1) // 2
    both = lo.covered().astype(int) + up.covered().astype(int)
    assert both.max() == 1 and both.sum() == n * n
    assert both[5:5 + n, 3:3 + n].sum() == n * n


@pytest.mark.parametrize("W,H,k", [(64, 48, 1), (32, 32, 3), (40, 12, 7)])
def test_planar_uv_square_closed_forms(W, H, k):
    """Two triangles map UV [0,1]^2 onto a kW x kH rectangle; with the bbox extent at exactly
    2^21-1 the grid scale is 1, so every texel centre (i+1/2, j+1/2) has the exact position
    (k(i+1/2), k(j+1/2), 0), rounded half up, and every texel stands for k^2 grid^2."""
    m = synth.uv_square_patch(W, H, k)
    a = oracle.Atlas(m, W, H, tile=8)
    assert a.S == 1.0 and list(a.mn) == [0.0, 0.0, 0.0]
    assert a.covered().all()
    i = np.arange(W)
    j = np.arange(H)
    ex = np.floor(k * (i + 0.5) + 0.5).astype(np.int64)
    ey = np.floor(k * (j + 0.5) + 0.5).astype(np.int64)
    assert np.array_equal(a.px, np.broadcast_to(ex, (H, W)))
    assert np.array_equal(a.py, np.broadcast_to(ey[:, None], (H, W)))
    assert (a.pz == 0).all()
    assert a.area_w.tolist() == [k * k * 256, k * k * 256]
    # each texel once: the two triangles split the texels along the diagonal
    assert set(np.unique(a.tri).tolist()) <= {0, 1}


def test_area_weights_match_exact_integer_brute_force():
    for seed in range(3):
        m = synth.random_soup(30, 100 + seed, uv_size=0.2)
        for W, H in ((64, 64), (1024, 512)):
            a = oracle.Atlas(m, W, H, tile=32, y0=0, y1=1)
            exp = [brute.area_weight(m, t, W, H, a.mn, a.S) for t in range(m.n_tri)]
            assert a.area_w.tolist() == exp


def test_area_weight_cap_and_degenerate():
    m = synth.random_soup(6, 9, uv_size=0.0005)          # tiny UV triangles: weights hit the cap
    a = oracle.Atlas(m, 16, 16)
    exp = [brute.area_weight(m, t, 16, 16, a.mn, a.S) for t in range(m.n_tri)]
    assert a.area_w.tolist() == exp
    assert int(a.area_w.max()) == (1 << 35) - 1
    assert int(a.area_w[1]) == 0                           # corners 3..5 share one UV: zero UV area


def test_tile_boxes_and_cover_bits_match_numpy_reductions():
    m = synth.vessel_cylindrical(40, 12, seed=5)
    W, H, T = 100, 70, 32                                  # ragged tiles on both axes
    a = oracle.Atlas(m, W, H, tile=T)
    box = a.tile_aabb()
    cov = a.covered()
    ntx, nty = -(-W // T), -(-H // T)
    for ty in range(nty):
        for tx in range(ntx):
            sl = (slice(ty * T, ty * T + T), slice(tx * T, tx * T + T))
            c = cov[sl]
            b = box[ty * ntx + tx]
            assert b[3] == c.sum() and b[7] == 0
            if c.any():
                for ax, plane in enumerate((a.px, a.py, a.pz)):
                    assert b[ax] == plane[sl][c].min() and b[4 + ax] == plane[sl][c].max()
            else:
                assert list(b[:3]) == [2 ** 31 - 1] * 3 and list(b[4:7]) == [-2 ** 31] * 3
    bits = a.cover_bits()
    exp = np.packbits(cov.ravel(), bitorder="little")
    exp = np.concatenate([exp, np.zeros((-len(exp)) % 4, np.uint8)]).view(np.uint32)
    assert np.array_equal(bits, exp)
    sbox = a.super_aabb(box)
    assert sbox.shape[0] == 1 and sbox[0, 3] == cov.sum()
    assert sbox[0, 0] == a.px[cov].min() and sbox[0, 6] == a.pz[cov].max()


def test_uncovered_sentinel_and_row_window():
    m = synth.vessel_cylindrical(30, 8, seed=2)
    full = oracle.Atlas(m, 48, 40, tile=16)
    win = oracle.Atlas(m, 48, 40, tile=16, y0=13, y1=29)
    assert np.array_equal(win.tri, full.tri[13:29]) and np.array_equal(win.px, full.px[13:29])
    unc = ~full.covered()
    assert (full.px[unc] == np.iinfo(np.int32).min).all() and (full.py[unc] == 0).all()


def _read_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                rows.append(line)
    return rows


def test_golden_hand_worked_triangle():
    """tests/golden/atlas_triangle_8x8.txt: coverage worked out by hand for one triangle."""
    rows = _read_golden("atlas_triangle_8x8.txt")
    # first line: the three UV corners in texel units, then 8 rows of the mask (top row = v high)
    corners = [tuple(float(v) for v in c.split(",")) for c in rows[0].split()]
    mask = np.array([[ch == "X" for ch in r] for r in rows[1:]])[::-1]
    W = H = 8
    uv = np.array([[x / W, y / H] for x, y in corners], np.float32)
    pos = np.array([[x, y, 0] for x, y in corners] + [[0, 0, 9]], np.float32)
    m = synth.Mesh(pos, uv, np.array([[0, 1, 2]], np.uint32), np.array([[0, 1, 2]], np.uint32)).check()
    a = oracle.Atlas(m, W, H, tile=8)
    assert np.array_equal(a.covered(), mask)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_atlas_brute_force_with_lattice_ties(seed):
    """Corners on the half-texel lattice, so many texel centres fall exactly on edges and
    corners: the owner rule decides them, and the brute force decides them by the nudge."""
    rng = np.random.default_rng(seed)
    W, H, n = 12, 10, 16
    c = rng.integers(-2, 2 * W + 3, size=(n, 3, 2)) / 2.0
    c[0] = [[0.5, 0.5], [6.5, 0.5], [0.5, 6.5]]
    c[1] = [[6.5, 6.5], [0.5, 6.5], [6.5, 0.5]]
    uv = (c / np.array([W, H])).reshape(-1, 2).astype(np.float32)
    pos = rng.uniform(-1, 1, size=(3 * n, 3)).astype(np.float32)
    idx = np.arange(3 * n, dtype=np.uint32).reshape(n, 3)
    m = synth.Mesh(pos, uv, idx.copy(), idx.copy()).check()
    a = oracle.Atlas(m, W, H, tile=4)
    tri, p = brute.atlas(m, W, H, a.mn, a.S)
    assert np.array_equal(a.tri, tri)
    assert np.array_equal(np.stack([a.px, a.py, a.pz]), p)
