"""Pins of the oracle's numeric layers (Section 4.2: a data texture of 8/16/32-bit integers or
16/32-bit floats plus a boolean mask texture): binary16 conversion against numpy's own float16,
arithmetic overlays against numpy's integer (wrapping) and IEEE float arithmetic and, for
float16, against exact rationals rounded by brute force; selection by value against numpy
comparisons; zonal statistics against scatter-adds, math.fsum and a closed form; numeric edits
against per-texel brute force.  CPU only."""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth

INT_TYPES = ["u8", "i8", "u16", "i16", "u32", "i32"]
FLOAT_TYPES = ["f16", "f32"]
RAW = {1: np.uint8, 2: np.uint16, 4: np.uint32}


@pytest.fixture(scope="module")
def atl():
    # charts with gutters: about 40% of the texels are uncovered
    m = synth.vessel_charts(40, 20, 10, 5, 128, seed=8)
    a = oracle.Atlas(m, 128, 96, tile=32)
    a.mesh = m
    return a


def rand_values(ntype, shape, seed):
    """Random values of a numeric type with the type's special values sprinkled in."""
    rng = np.random.default_rng(seed)
    dt = oracle.NUM_NP[ntype]
    n = int(np.prod(shape))
    if ntype in INT_TYPES:
        info = np.iinfo(dt)
        v = rng.integers(info.min, info.max, size=n, endpoint=True, dtype=np.int64)
        special = [0, 1, -1 if info.min < 0 else 2, info.min, info.max, info.max - 1]
    else:
        if ntype == "f16":
            v = rng.integers(0, 1 << 16, size=n).astype(np.uint16).view(np.float16)
        else:
            v = np.concatenate([rng.standard_normal(n // 2).astype(np.float32) * 1e3,
                                rng.integers(0, 1 << 32, size=n - n // 2, dtype=np.uint64).astype(np.uint32)
                                .view(np.float32)])
        fi = np.finfo(dt)
        special = [0.0, -0.0, 1.0, -1.0, np.inf, -np.inf, np.nan, fi.max, -fi.max, fi.tiny, fi.tiny / 4]
    v = np.asarray(v).astype(dt)
    idx = rng.choice(n, size=min(n, 4 * len(special)), replace=False)
    with np.errstate(over="ignore", invalid="ignore"):
        v[idx] = np.array(special * 4, dtype=np.float64 if ntype in FLOAT_TYPES else np.int64)[: len(idx)].astype(dt)
    return v.reshape(shape)


def rand_mask(shape, seed, p=0.7):
    return (np.random.default_rng(seed).uniform(size=shape) < p).astype(np.uint8)


# ---- binary16 conversion --------------------------------------------------------------------

def test_half_decode_matches_numpy_on_every_pattern():
    h = np.arange(1 << 16, dtype=np.uint32).astype(np.uint16)
    got = oracle.half_to_float(h)
    ref = h.view(np.float16).astype(np.float32)
    same = (got.view(np.uint32) == ref.view(np.uint32)) | (np.isnan(got) & np.isnan(ref))
    assert same.all()


def test_half_encode_matches_numpy_on_random_patterns_ties_and_edges():
    rng = np.random.default_rng(1)
    x = rng.integers(0, 1 << 32, size=400_000, dtype=np.uint64).astype(np.uint32).view(np.float32)
    # every half value, the midpoints between neighbours (exact in float32: ties), and the
    # float32 neighbours of those midpoints
    hv = np.arange(0, 0x7C00, dtype=np.uint16).view(np.float16).astype(np.float64)
    mids = ((hv[:-1] + hv[1:]) / 2).astype(np.float32)
    x = np.concatenate([x, hv.astype(np.float32), mids, np.nextafter(mids, np.float32(np.inf)),
                        np.nextafter(mids, np.float32(0)), -mids, np.float32([65504, 65519.99, 65520, 1e-8, 2 ** -25,
                                                                               2 ** -24, 3 * 2 ** -26])])
    got = oracle.float_to_half(x)
    with np.errstate(over="ignore"):
        ref = x.astype(np.float16).view(np.uint16)
    nan = np.isnan(x)
    assert np.array_equal(got[~nan], ref[~nan])
    assert (got[nan] & 0x7C00 == 0x7C00).all() and (got[nan] & 0x3FF != 0).all()


# ---- arithmetic overlays --------------------------------------------------------------------

def np_arith(ntype, a, b, op):
    dt = oracle.NUM_NP[ntype]
    with np.errstate(all="ignore"):
        if op == "min":
            return np.where(a < b, a, b).astype(dt)
        if op == "max":
            return np.where(a > b, a, b).astype(dt)
        f = {"add": np.add, "sub": np.subtract, "mul": np.multiply, "div": np.divide}[op]
        return f(a, b).astype(dt)


def same_values(x, y):
    """Equal bit patterns, or both NaN (NaN payloads are not part of the result)."""
    rx, ry = x.view(RAW[x.itemsize]), y.view(RAW[y.itemsize])
    if x.dtype.kind == "f":
        return (rx == ry) | (np.isnan(x) & np.isnan(y))
    return rx == ry


@pytest.mark.parametrize("ntype", INT_TYPES + FLOAT_TYPES)
@pytest.mark.parametrize("op", ["add", "sub", "mul", "div", "min", "max"])
def test_arith_matches_numpy(atl, ntype, op):
    if op == "div" and ntype in INT_TYPES:
        with pytest.raises(oracle.OracleError):
            oracle.num_arith(atl, ntype, rand_values(ntype, atl.tri.shape, 1), rand_mask(atl.tri.shape, 2),
                             rand_values(ntype, atl.tri.shape, 3), rand_mask(atl.tri.shape, 4), op)
        return
    A = rand_values(ntype, atl.tri.shape, 11)
    B = rand_values(ntype, atl.tri.shape, 12)
    ma, mb = rand_mask(atl.tri.shape, 13), rand_mask(atl.tri.shape, 14)
    out, mout = oracle.num_arith(atl, ntype, A, ma, B, mb, op)
    valid = (ma == 1) & (mb == 1) & atl.covered()
    assert np.array_equal(mout, valid.astype(np.uint8))
    assert (out.view(RAW[out.itemsize])[~valid] == 0).all()
    assert same_values(out[valid], np_arith(ntype, A, B, op)[valid]).all()
    # scalar form: b is the same value everywhere and always valid
    s = B.flat[7]
    out2, mout2 = oracle.num_arith(atl, ntype, A, ma, None, None, op, oracle.value_bits(s, ntype))
    valid2 = (ma == 1) & atl.covered()
    assert np.array_equal(mout2, valid2.astype(np.uint8))
    assert same_values(out2[valid2], np_arith(ntype, A, np.full_like(A, s), op)[valid2]).all()


def exact_half(r: Fraction):
    """Nearest binary16 to the exact rational r (ties to even), by brute force over the neighbours
    of a first guess; returns the float16 value (inf on overflow)."""
    g = np.float16(float(r)) if abs(r) < 70000 else np.float16(np.inf if r > 0 else -np.inf)
    if np.isinf(g):
        return g
    cands = {g, np.nextafter(g, np.float16(np.inf)), np.nextafter(g, np.float16(-np.inf))}
    best = None
    for c in cands:
        if np.isinf(c):
            continue
        d = abs(Fraction(float(c)) - r)
        key = (d, int(np.array(c).view(np.uint16)) & 1)   # ties: even mantissa first
        if best is None or key < best[0]:
            best = (key, c)
    bound = Fraction(65520)   # values at or beyond the halfway point above the largest half overflow
    if abs(r) >= bound:
        return np.float16(np.inf if r > 0 else -np.inf)
    return best[1]


@pytest.mark.parametrize("op", ["add", "sub", "mul", "div"])
def test_f16_arith_is_the_correctly_rounded_operation(atl, op):
    """The float16 reading (one float32 operation, then one rounding) equals rounding the exact
    rational result once, on finite operands (this is the double-rounding bound 24 >= 2*11 + 2)."""
    rng = np.random.default_rng(21)
    n = 1500
    A = rng.integers(0, 0x7C00, size=n).astype(np.uint16).view(np.float16) * rng.choice([-1, 1], n).astype(np.float16)
    B = rng.integers(1, 0x7C00, size=n).astype(np.uint16).view(np.float16)
    H, W = atl.tri.shape
    idx = np.flatnonzero(atl.covered())[:n]
    a = np.zeros(H * W, np.float16)
    b = np.ones(H * W, np.float16)
    a[idx], b[idx] = A[: len(idx)], B[: len(idx)]
    ones = np.ones((H, W), np.uint8)
    out, _ = oracle.num_arith(atl, "f16", a.reshape(H, W), ones, b.reshape(H, W), ones, op)
    f = {"add": lambda x, y: x + y, "sub": lambda x, y: x - y, "mul": lambda x, y: x * y, "div": lambda x, y: x / y}[op]
    for i in idx:
        ref = exact_half(f(Fraction(float(a[i])), Fraction(float(b[i]))))
        got = out.reshape(-1)[i]
        assert got == ref and np.signbit(got) == np.signbit(ref) or (got == 0 and ref == 0), (a[i], b[i], got, ref)


def test_arith_rejects_bad_arguments(atl):
    A = rand_values("u8", atl.tri.shape, 1)
    m = rand_mask(atl.tri.shape, 2)
    with pytest.raises(oracle.OracleError):
        oracle.num_arith(atl, "u8", A, m, None, None, "add", 256)   # scalar wider than the type


# ---- selection by value ---------------------------------------------------------------------

@pytest.mark.parametrize("ntype", INT_TYPES + FLOAT_TYPES)
@pytest.mark.parametrize("cmp", ["lt", "le", "gt", "ge", "eq", "ne"])
def test_select_by_value_matches_numpy(atl, ntype, cmp):
    V = rand_values(ntype, atl.tri.shape, 31)
    V[::2] = V.flat[5]            # ties with the threshold
    m = rand_mask(atl.tri.shape, 32)
    t = V.flat[5]
    base = np.random.default_rng(33).integers(0, 200, size=atl.tri.shape).astype(np.uint8)
    L = base.copy()
    h = oracle.num_select(atl, ntype, V, m, cmp, oracle.value_bits(t, ntype), L, 250)
    x = V.astype(np.float64) if ntype in FLOAT_TYPES else V.astype(np.int64)
    tt = np.float64(t) if ntype in FLOAT_TYPES else np.int64(t)
    with np.errstate(invalid="ignore"):
        hit = {"lt": x < tt, "le": x <= tt, "gt": x > tt, "ge": x >= tt, "eq": x == tt, "ne": x != tt}[cmp]
    sel = hit & (m == 1) & atl.covered()
    assert h == int(sel.sum())
    assert np.array_equal(L, np.where(sel, 250, base).astype(np.uint8))


# ---- zonal statistics -----------------------------------------------------------------------

@pytest.mark.parametrize("ntype", ["u8", "i16", "i32", "u32", "f16", "f32"])
def test_stats_match_scatter_adds_and_exact_sums(atl, ntype):
    V = rand_values(ntype, atl.tri.shape, 41)
    if ntype in FLOAT_TYPES:
        V[~np.isfinite(V.astype(np.float64))] = 0   # finite values: the sums have an error bound
    m = rand_mask(atl.tri.shape, 42)
    Z = np.random.default_rng(43).integers(0, 12, size=atl.tri.shape).astype(np.uint8)
    n_labels = 10
    r = oracle.num_stats(atl, ntype, V, m, Z, n_labels)
    v = V.astype(np.float64)
    keep = atl.covered() & (m == 1) & (Z < n_labels) & ~np.isnan(v)
    z = Z[keep].astype(np.int64)
    w = atl.area_w[atl.tri[keep]]
    x = v[keep]
    ec = np.zeros(n_labels, np.uint64)
    ea = np.zeros(n_labels, np.uint64)
    np.add.at(ec, z, np.uint64(1))
    np.add.at(ea, z, w)
    assert np.array_equal(r["count"], ec) and np.array_equal(r["area"], ea)
    emin = np.full(n_labels, np.inf)
    emax = np.full(n_labels, -np.inf)
    np.minimum.at(emin, z, x)
    np.maximum.at(emax, z, x)
    assert np.array_equal(r["vmin"], emin) and np.array_equal(r["vmax"], emax)
    u = 2.0 ** -53
    for k in range(n_labels):
        xs = x[z == k]
        ws = w[z == k].astype(np.float64) * xs        # each product rounded once, as in the oracle
        for got, terms in ((r["sum"][k], xs), (r["wsum"][k], ws)):
            exact = math.fsum(terms)
            bound = max(len(terms) - 1, 0) * u * math.fsum(np.abs(terms)) * 1.0001
            assert abs(got - exact) <= bound, (k, got, exact, bound)


def test_stats_closed_form_on_the_square_patch():
    """A constant value c on the planar k x k-unit-per-texel square: every texel weighs k^2 * 256,
    so count, area, min, max, mean and the area integral are closed forms (exact in double)."""
    W, H, k = 48, 40, 5
    a = oracle.Atlas(synth.uv_square_patch(W, H, k), W, H, tile=16)
    c = -3.25
    V = np.full((H, W), c, np.float32)
    m = np.ones((H, W), np.uint8)
    r = oracle.num_stats(a, "f32", V, m, None, 1)
    n = W * H
    assert r["count"][0] == n and r["area"][0] == n * k * k * 256
    assert r["vmin"][0] == c and r["vmax"][0] == c
    assert r["sum"][0] == c * n and r["wsum"][0] == c * n * k * k * 256
    # half the texels invalid: the statistics see only the other half
    m[:, : W // 2] = 0
    r = oracle.num_stats(a, "f32", V, m, None, 1)
    assert r["count"][0] == n // 2 and r["wsum"][0] == c * (n // 2) * k * k * 256


def test_stats_skip_nan_and_fold_negative_zero(atl):
    V = np.zeros(atl.tri.shape, np.float32)
    cov = atl.covered()
    idx = np.flatnonzero(cov)
    V.flat[idx[0]] = np.nan
    V.flat[idx[1]] = -0.0
    m = np.ones(atl.tri.shape, np.uint8)
    r = oracle.num_stats(atl, "f32", V, m, None, 1)
    assert r["count"][0] == cov.sum() - 1
    assert not np.signbit(r["vmin"][0]) and r["vmin"][0] == 0 and r["vmax"][0] == 0
    empty = oracle.num_stats(atl, "f32", V, np.zeros_like(m), None, 1)
    assert empty["count"][0] == 0 and empty["vmin"][0] == np.inf and empty["vmax"][0] == -np.inf


# ---- numeric edits --------------------------------------------------------------------------

def test_numeric_sphere_edit_brute_force(atl):
    """Every covered texel within a stroke gets its value bits and a set mask; erase strokes clear
    both; texels outside every stroke keep their data and mask; later strokes win."""
    rng = np.random.default_rng(51)
    st = synth.sphere_strokes(atl.mesh, 6, 52, 0.1, 0.3, 1, 5)
    vals = [1.5, -2.25, 3e-5, 7.0, 100.0, -0.5]
    recs = oracle.sphere_records(atl.mn, atl.S, st.centre, st.radius, [oracle.value_bits(v, "f32") for v in vals])
    recs["flags"][3] = oracle.ERASE
    data = rng.standard_normal(atl.tri.shape).astype(np.float32)
    mask = rand_mask(atl.tri.shape, 53)
    d0, m0 = data.copy(), mask.copy()
    hits, _ = oracle.num_select_sphere(atl, data, mask, recs)
    q = np.stack([atl.px, atl.py, atl.pz], -1).astype(np.int64)
    ed, em = d0.copy(), m0.copy()
    cov = atl.covered()
    for k, s in enumerate(recs):
        d2 = ((q - np.array([s["cx"], s["cy"], s["cz"]], np.int64)) ** 2).sum(-1)
        sel = cov & (d2 <= s["r2"])
        assert hits[k] == sel.sum()
        if s["flags"] & oracle.ERASE:
            ed[sel], em[sel] = 0, 0
        else:
            ed[sel], em[sel] = vals[k], 1
    assert np.array_equal(data.view(np.uint32), ed.view(np.uint32)) and np.array_equal(mask, em)
    assert hits.sum() > 0
