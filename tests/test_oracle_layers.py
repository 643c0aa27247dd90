"""Pins of the oracle's layer operations: boolean overlays and per-label area, against
numpy's bitwise and scatter-add routines, De Morgan and inclusion-exclusion.  CPU only."""
import numpy as np
import pytest

import oracle
import synth


@pytest.fixture(scope="module")
def atl():
    m = synth.vessel_cylindrical(40, 12, noise_amp=0.02, seed=8)
    return oracle.Atlas(m, 100, 60, tile=32)   # uncovered gaps at the seam column are possible


def rand_layer(a, dtype, seed, hi=None):
    rng = np.random.default_rng(seed)
    hi = np.iinfo(dtype).max if hi is None else hi
    return rng.integers(0, hi + 1, size=a.tri.shape).astype(dtype)


def np_overlay(a, b, op, flags, dtype, cov):
    full = np.iinfo(dtype).max
    x = ~a & full if flags & oracle.NOT_A else a
    y = ~b & full if flags & oracle.NOT_B else b
    r = {oracle.AND: x & y, oracle.OR: x | y, oracle.XOR: x ^ y, oracle.MASK: np.where(y != 0, x, 0)}[op]
    r = ~r & full if flags & oracle.NOT_OUT else r
    return np.where(cov, r, 0).astype(dtype)


@pytest.mark.parametrize("dtype", [np.uint8, np.uint16])
@pytest.mark.parametrize("op", [oracle.AND, oracle.OR, oracle.XOR, oracle.MASK])
def test_overlay_matches_numpy_for_every_flag(atl, dtype, op):
    A = rand_layer(atl, dtype, 1)
    B = rand_layer(atl, dtype, 2)
    B[::3] = 0
    for flags in range(8):
        got = oracle.overlay(atl, A, B, op, flags)
        assert np.array_equal(got, np_overlay(A, B, op, flags, dtype, atl.covered()))


def test_overlay_identities(atl):
    A = rand_layer(atl, np.uint8, 3)
    B = rand_layer(atl, np.uint8, 4)
    cov = atl.covered()
    # De Morgan on covered texels: ~(A & B) == ~A | ~B and ~(A | B) == ~A & ~B
    assert np.array_equal(oracle.overlay(atl, A, B, "and", oracle.NOT_OUT),
                          oracle.overlay(atl, A, B, "or", oracle.NOT_A | oracle.NOT_B))
    assert np.array_equal(oracle.overlay(atl, A, B, "or", oracle.NOT_OUT),
                          oracle.overlay(atl, A, B, "and", oracle.NOT_A | oracle.NOT_B))
    assert not oracle.overlay(atl, A, A, "xor").any()
    assert np.array_equal(oracle.overlay(atl, A, A, "and"), np.where(cov, A, 0))
    assert np.array_equal(oracle.overlay(atl, A, A, "or"), np.where(cov, A, 0))
    assert (oracle.overlay(atl, A, B, "and", oracle.NOT_OUT)[~cov] == 0).all()
    with pytest.raises(oracle.OracleError):
        oracle.overlay(atl, A, B, 7)


@pytest.mark.parametrize("dtype,n_labels", [(np.uint8, 256), (np.uint8, 37), (np.uint16, 1000)])
def test_label_area_matches_scatter_add(atl, dtype, n_labels):
    L = rand_layer(atl, dtype, 5, hi=min(np.iinfo(dtype).max, n_labels + 20))
    cnt, area = oracle.label_area(atl, L, n_labels)
    cov = atl.covered()
    lab = L[cov].astype(np.int64)
    w = atl.area_w[atl.tri[cov]]
    keep = lab < n_labels
    ec = np.zeros(n_labels, np.uint64)
    ea = np.zeros(n_labels, np.uint64)
    np.add.at(ec, lab[keep], np.uint64(1))
    np.add.at(ea, lab[keep], w[keep])
    assert np.array_equal(cnt, ec) and np.array_equal(area, ea)


def test_label_area_totals_and_inclusion_exclusion(atl):
    cov = atl.covered()
    ones = np.ones(atl.tri.shape, np.uint8)
    c1, a1 = oracle.label_area(atl, ones, 2)
    assert c1[1] == cov.sum() and a1[1] == atl.area_w[atl.tri[cov]].astype(np.uint64).sum()
    rng = np.random.default_rng(9)
    A = (rng.uniform(size=cov.shape) < 0.4).astype(np.uint8)
    B = (rng.uniform(size=cov.shape) < 0.5).astype(np.uint8)
    area = lambda X: int(oracle.label_area(atl, X, 2)[1][1])
    a_or = area(oracle.overlay(atl, A, B, "or"))
    a_and = area(oracle.overlay(atl, A, B, "and"))
    assert a_or == area(A) + area(B) - a_and
    # labels partition the covered area
    L = rand_layer(atl, np.uint8, 6, hi=9)
    c, a = oracle.label_area(atl, L, 10)
    assert c.sum() == cov.sum() and a.sum() == a1[1]


def test_label_area_closed_form_square_patch():
    W, H, k = 48, 40, 5
    a = oracle.Atlas(synth.uv_square_patch(W, H, k), W, H, tile=16)
    L = np.ones((H, W), np.uint8)
    L[:, : W // 2] = 2
    c, ar = oracle.label_area(a, L, 3)
    assert c.tolist() == [0, W * H - H * (W // 2), H * (W // 2)]
    # every texel of the planar kW x kH rectangle stands for k^2 grid^2 (8 fractional bits)
    assert ar.tolist() == [0, c[1] * k * k * 256, c[2] * k * k * 256]
    assert int(ar.sum()) == (k * W) * (k * H) * 256


@pytest.mark.parametrize("side", [512, 1024])
def test_label_area_sums_to_the_surface_area_of_a_curved_mesh(side):
    """Per-texel area (the owning triangle's 3D area over its UV area, §5's area per texel): summed
    over every covered texel it must give the mesh's surface area, computed here from the triangles
    in double, up to the sampling of triangle edges by texel centres (under 1% on this chart atlas;
    a dropped factor, a wrong fixed-point shift or the UV area in the wrong units is far off)."""
    m = synth.vessel_charts(200, 100, 25, 10, side, seed=5)
    a = oracle.Atlas(m, side, side, tile=32)
    c, ar = oracle.label_area(a, np.zeros((side, side), np.uint8), 1)
    p = m.pos.astype(np.float64)
    t = m.tri_pos.astype(np.int64)
    surface = 0.5 * np.linalg.norm(np.cross(p[t[:, 1]] - p[t[:, 0]], p[t[:, 2]] - p[t[:, 0]]), axis=1).sum()
    assert c[0] > 0.75 * side * side
    assert abs(float(ar[0]) / 2.0 ** 8 / a.S ** 2 / surface - 1.0) < 0.01
