"""GPU parity of numeric layers (Section 4.2: a data texture of 8/16/32-bit integers or 16/32-bit
floats plus a mask texture), through the C ABI against the CPU oracle on the same seeded inputs:
numeric sphere edits, arithmetic overlays and selection by value bit for bit (NaN results compared
as NaN, their payload is unspecified); lasso and tool edits equal except on the texels the oracle
flags as ambiguous; zonal statistics exact in count, area, min and max, and within the stated
summation bound in the two sums."""
import math

import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import DEV, gpu_atlas, to_dev

pytestmark = pytest.mark.gpu

from paper_2501_14807_gb300 import lcl  # noqa: E402

RAW = {1: np.uint8, 2: np.uint16, 4: np.uint32}
ALL_TYPES = ["u8", "i8", "u16", "i16", "u32", "i32", "f16", "f32"]
ATLASES = [  # (name, mesh maker, W, H, tile): grouped mask writes need tile >= 32 and W % 32 == 0
    ("charts-512-t32", lambda: synth.vessel_charts(120, 60, 20, 10, 512, seed=8), 512, 512, 32),
    ("charts-384-t16", lambda: synth.vessel_charts(120, 60, 20, 10, 384, seed=9), 384, 384, 16),
    ("ragged-300x170", lambda: synth.vessel_cylindrical(60, 20, seed=4), 300, 170, 32),
]


def bits_of(mask_u8):
    """Byte mask (H x W) -> the library's bit plane (int32 words, little-endian bit order)."""
    flat = np.ascontiguousarray(mask_u8, dtype=np.uint8).reshape(-1)
    n_words = (flat.size + 31) // 32
    padded = np.zeros(n_words * 32, np.uint8)
    padded[: flat.size] = flat
    words = np.packbits(padded, bitorder="little").view(np.uint32)
    out = np.zeros(((n_words + 3) // 4) * 4, np.uint32)
    out[:n_words] = words
    return out


def gpu_layer(ntype, data, mask, W, H):
    view = {"u8": np.uint8, "i8": np.int8, "u16": np.int16, "i16": np.int16, "u32": np.int32, "i32": np.int32,
            "f16": np.float16, "f32": np.float32}[ntype]      # torch has no uint16 / uint32: same bits
    d = torch.from_numpy(np.ascontiguousarray(data).view(view)).to(DEV)
    m = torch.from_numpy(bits_of(mask).view(np.int32)).to(DEV)
    return lcl.NumericLayer(W, H, ntype, DEV, data=d, mask=m)


def host_data(layer: lcl.NumericLayer):
    return layer.data.cpu().numpy().view(oracle.NUM_NP[layer.ntype])


def same_values(x, y):
    rx, ry = x.view(RAW[x.itemsize]), y.view(RAW[y.itemsize])
    if x.dtype.kind == "f":
        return (rx == ry) | (np.isnan(x) & np.isnan(y))
    return rx == ry


def rand_values(ntype, shape, seed):
    rng = np.random.default_rng(seed)
    dt = oracle.NUM_NP[ntype]
    n = int(np.prod(shape))
    if ntype.startswith("f"):
        if ntype == "f16":
            v = rng.integers(0, 1 << 16, size=n).astype(np.uint16).view(np.float16)
        else:
            v = np.concatenate([rng.standard_normal(n // 2).astype(np.float32) * 100,
                                rng.integers(0, 1 << 32, size=n - n // 2, dtype=np.uint64).astype(np.uint32)
                                .view(np.float32)])
            rng.shuffle(v)
    else:
        info = np.iinfo(dt)
        v = rng.integers(info.min, info.max, size=n, endpoint=True, dtype=np.int64).astype(dt)
    return np.ascontiguousarray(v.astype(dt).reshape(shape))


def rand_mask(shape, seed, p=0.7):
    return (np.random.default_rng(seed).uniform(size=shape) < p).astype(np.uint8)


@pytest.fixture(scope="module", params=ATLASES, ids=[c[0] for c in ATLASES])
def setup(request):
    name, make, W, H, T = request.param
    mesh = make()
    o = oracle.Atlas(mesh, W, H, tile=T)
    m, a = gpu_atlas(mesh, W, H, T)
    return mesh, o, m, a, W, H


@pytest.mark.parametrize("ntype", ["u8", "i16", "u32", "f16", "f32"])
def test_numeric_sphere_bit_exact(setup, ntype):
    mesh, o, m, a, W, H = setup
    st = synth.sphere_strokes(mesh, 24, 101, 0.02, 0.3, 1, 2)
    vals = rand_values(ntype, (24,), 102)
    if ntype.startswith("f"):
        vals[~np.isfinite(vals.astype(np.float64))] = 1
    recs = oracle.sphere_records(o.mn, o.S, st.centre, st.radius, [oracle.value_bits(v, ntype) for v in vals])
    recs["flags"][3::5] = oracle.ERASE
    recs["flags"][4::7] |= oracle.pad_flags(2, 3)
    data = rand_values(ntype, (H, W), 103)
    mask = rand_mask((H, W), 104)
    layer = gpu_layer(ntype, data, mask, W, H)
    hits = torch.zeros(len(recs), dtype=torch.int64, device=DEV)
    lcl.lcl_numeric_sphere(a, layer, recs, hits_out=hits)
    eh, _ = oracle.num_select_sphere(o, data, mask, recs)
    got = host_data(layer)
    assert np.array_equal(got.view(RAW[got.itemsize]), data.view(RAW[data.itemsize])), "numeric data differs"
    assert np.array_equal(layer.mask_bits(), mask.astype(bool)), "numeric mask differs"
    assert np.array_equal(hits.cpu().numpy().view(np.uint64), eh)
    assert eh.sum() > 0


@pytest.mark.parametrize("ntype", ["u16", "f32"])
def test_numeric_lasso_and_tool_within_tolerance(setup, ntype):
    mesh, o, m, a, W, H = setup
    Ws, Hs = 320, 240
    rng = np.random.default_rng(111)
    cam = synth.orbit_camera(mesh, Ws, Hs, rng)
    M = oracle.camera_mq(cam.vp, o.mn, o.S)
    dm = oracle.depth(mesh, o.mn, o.S, M, Ws, Hs)
    d = torch.empty((Hs, Ws), dtype=torch.float32, device=DEV)
    lcl.lcl_depth_render(m, a, lcl.camera(M, Ws, Hs), d)
    data = rand_values(ntype, (H, W), 112)
    mask = rand_mask((H, W), 113)
    layer = gpu_layer(ntype, data, mask, W, H)
    hits = torch.zeros(1, dtype=torch.int64, device=DEV)
    amb_all = np.zeros((H, W), bool)
    touched = 0
    las = synth.lassos(mesh, [cam], 6, 114, 1, 2, 1)
    for i, L in enumerate(las):
        v = oracle.value_bits(rand_values(ntype, (1,), 200 + i)[0], ntype)
        flags = oracle.ERASE if i == 2 else (oracle.pad_flags(2, 3) if i == 4 else 0)
        if i % 2 == 0:
            h, amb = oracle.num_select_lasso(o, data, mask, M, dm, L.poly, v, flags)
            lcl.lcl_numeric_lasso(a, layer, lcl.camera(M, Ws, Hs), d, L.poly, v, flags, hits_out=hits)
        else:
            c = L.poly.mean(0)
            size = (float(rng.uniform(30, 150)), float(rng.uniform(30, 150)))
            pad = oracle.pad_flags(2, 2) if i == 3 else 0
            h, _, amb = oracle.num_select_tool(o, data, mask, M, dm, (float(c[0]), float(c[1])), size, None, v,
                                               flags | pad)
            tool = lcl.make_tool((float(c[0]), float(c[1])), size, None, pad)
            lcl.lcl_numeric_tool(a, layer, lcl.camera(M, Ws, Hs), d, tool, v, flags, hits_out=hits)
        touched += h
        amb_all |= amb.astype(bool)
        assert abs(int(hits.item()) - h) <= amb.sum()
    got = host_data(layer)
    diff = (got.view(RAW[got.itemsize]) != data.view(RAW[data.itemsize])) | (layer.mask_bits() != mask.astype(bool))
    assert touched > 100
    assert not (diff & ~amb_all).any(), "numeric lasso / tool edits differ outside the ambiguous texels"


@pytest.mark.parametrize("ntype", ALL_TYPES)
def test_numeric_arith_bit_exact(setup, ntype):
    mesh, o, m, a, W, H = setup
    A = rand_values(ntype, (H, W), 121)
    B = rand_values(ntype, (H, W), 122)
    ma, mb = rand_mask((H, W), 123), rand_mask((H, W), 124)
    ops = ["add", "sub", "mul", "min", "max"] + (["div"] if ntype.startswith("f") else [])
    for op in ops:
        la, lb = gpu_layer(ntype, A, ma, W, H), gpu_layer(ntype, B, mb, W, H)
        out = lcl.NumericLayer(W, H, ntype, DEV)
        out.mask.fill_(-1)
        lcl.lcl_numeric_arith(a, la, lb, out, op)
        eo, em = oracle.num_arith(o, ntype, A, ma, B, mb, op)
        got = host_data(out)
        assert same_values(got, eo).all(), f"{ntype} {op}: data differs"
        assert np.array_equal(out.mask_bits(), em.astype(bool)), f"{ntype} {op}: mask differs"
        # scalar form, written in place over a (out aliases a)
        s = oracle.value_bits(B.flat[5], ntype)
        lcl.lcl_numeric_arith(a, la, None, la, op, s)
        eo2, em2 = oracle.num_arith(o, ntype, A, ma, None, None, op, s)
        got2 = host_data(la)
        assert same_values(got2, eo2).all(), f"{ntype} {op} scalar: data differs"
        assert np.array_equal(la.mask_bits(), em2.astype(bool)), f"{ntype} {op} scalar: mask differs"


@pytest.mark.parametrize("ntype", ALL_TYPES)
@pytest.mark.parametrize("ldt", [np.uint8, np.uint16])
def test_numeric_select_bit_exact(setup, ntype, ldt):
    mesh, o, m, a, W, H = setup
    V = rand_values(ntype, (H, W), 131)
    V[::3] = V.flat[17]
    mask = rand_mask((H, W), 132)
    lv = gpu_layer(ntype, V, mask, W, H)
    t = oracle.value_bits(V.flat[17], ntype)
    base = np.random.default_rng(133).integers(0, 100, size=(H, W)).astype(ldt)
    for i, cmp in enumerate(["lt", "le", "gt", "ge", "eq", "ne"]):
        layer = to_dev(base)
        hits = torch.zeros(1, dtype=torch.int64, device=DEV)
        lcl.lcl_numeric_select(a, lv, cmp, t, layer, 200 + i, hits_out=hits)
        exp = base.copy()
        h = oracle.num_select(o, ntype, V, mask, cmp, t, exp, 200 + i)
        assert np.array_equal(layer.cpu().numpy().view(ldt), exp), f"{ntype} {cmp}: labels differ"
        assert int(hits.item()) == h


@pytest.mark.parametrize("ntype", ALL_TYPES)
@pytest.mark.parametrize("zdt,n_labels", [(None, 1), (np.uint8, 40), (np.uint16, 3000)])
def test_numeric_stats(setup, ntype, zdt, n_labels):
    mesh, o, m, a, W, H = setup
    V = rand_values(ntype, (H, W), 141)
    if ntype.startswith("f"):
        V[np.isinf(V.astype(np.float64))] = 0      # finite sums (NaNs stay: they are skipped)
    mask = rand_mask((H, W), 142)
    lv = gpu_layer(ntype, V, mask, W, H)
    zones = None
    zd = None
    if zdt is not None:
        # zones in runs (as strokes leave them) plus scattered labels beyond n_labels
        rng = np.random.default_rng(143)
        zones = np.repeat(rng.integers(0, n_labels + 5, size=(H, W // 4 + 1)), 4, axis=1)[:, :W].astype(zdt)
        zd = to_dev(zones)
    out = lcl.lcl_numeric_stats(a, lv, zd, n_labels)
    got = lcl.zone_stats_host(out)
    exp = oracle.num_stats(o, ntype, V, mask, zones, n_labels)
    assert np.array_equal(got["count"], exp["count"]) and np.array_equal(got["area"], exp["area"])
    assert np.array_equal(got["vmin"], exp["vmin"]) and np.array_equal(got["vmax"], exp["vmax"])
    # summation bounds: the oracle adds the n terms in texel order, (n - 1) 2^-53 sum |terms|; the
    # library adds the values in some other order, and the weighted terms per triangle stretch as
    # w x (sum of the stretch's values), 2 n 2^-53 sum |w v|; the difference is within the sum
    v = V.astype(np.float64)
    keep = o.covered() & (mask == 1) & ~np.isnan(v)
    z = np.zeros((H, W), np.int64) if zones is None else zones.astype(np.int64)
    keep &= z < n_labels
    w = o.area_w[o.tri[keep]].astype(np.float64)
    x = np.where(v[keep] == 0, 0.0, v[keep])
    abs_sum = np.zeros(n_labels)
    abs_wsum = np.zeros(n_labels)
    np.add.at(abs_sum, z[keep], np.abs(x))
    np.add.at(abs_wsum, z[keep], np.abs(w * x))
    u = 2.0 ** -53
    n = exp["count"].astype(np.float64)
    tol_s = 2 * np.maximum(n - 1, 0) * u * abs_sum * 1.001
    tol_w = 3 * n * u * abs_wsum * 1.001
    assert (np.abs(got["sum"] - exp["sum"]) <= tol_s).all()
    assert (np.abs(got["wsum"] - exp["wsum"]) <= tol_w).all()
    assert exp["count"].sum() > 0


def test_numeric_rejections():
    mesh = synth.vessel_cylindrical(30, 10, seed=2)
    m, a = gpu_atlas(mesh, 128, 64, 32)
    f = lcl.NumericLayer(128, 64, "f32", DEV)
    i = lcl.NumericLayer(128, 64, "i16", DEV)
    with pytest.raises(lcl.LclError):
        lcl.lcl_numeric_arith(a, f, i, f, "add")          # types differ
    with pytest.raises(lcl.LclError):
        lcl.lcl_numeric_arith(a, i, i, i, "div")          # integer division
    with pytest.raises(lcl.LclError):
        lcl.lcl_numeric_arith(a, i, None, i, "add", 1 << 16)   # scalar wider than the type
    st = synth.sphere_strokes(mesh, 2, 1, 0.1, 0.1, 1, 1)
    o = oracle.Atlas(mesh, 128, 64, tile=32)
    recs = oracle.sphere_records(o.mn, o.S, st.centre, st.radius, [1 << 16, 1])
    with pytest.raises(lcl.LclError):
        lcl.lcl_numeric_sphere(a, i, recs)                # value wider than int16
    recs = oracle.sphere_records(o.mn, o.S, st.centre, st.radius, [1, 1])
    recs["flags"][0] = 0x200
    with pytest.raises(lcl.LclError):
        lcl.lcl_numeric_sphere(a, i, recs)                # unknown flag bit
    with pytest.raises(lcl.LclError):
        lcl.lcl_numeric_stats(a, f, None, 2)              # no zones, n_labels != 1


@pytest.mark.parametrize("ntype", ["f16", "f32"])
def test_numeric_stats_with_infinities(ntype):
    """Infinite values make a zone's sums infinite (or NaN when both signs meet, or a zero weight
    meets one), as in the oracle; count, area, min and max stay exact."""
    mesh = synth.vessel_charts(120, 60, 20, 10, 384, seed=9)
    W = H = 384
    o = oracle.Atlas(mesh, W, H, tile=16)
    m, a = gpu_atlas(mesh, W, H, 16)
    V = rand_values(ntype, (H, W), 151)
    V[np.isnan(V.astype(np.float64))] = 1
    cov = np.flatnonzero(o.covered())
    rng = np.random.default_rng(152)
    zones = (np.arange(H * W) // 997 % 7).astype(np.uint8).reshape(H, W)
    V.flat[rng.choice(cov, 40, replace=False)] = np.inf                 # zones get +inf ...
    V.flat[rng.choice(cov[cov % 997 < 400], 5, replace=False)] = -np.inf  # ... some also -inf
    mask = np.ones((H, W), np.uint8)
    out = lcl.lcl_numeric_stats(a, gpu_layer(ntype, V, mask, W, H), to_dev(zones), 7)
    got = lcl.zone_stats_host(out)
    exp = oracle.num_stats(o, ntype, V, mask, zones, 7)
    assert np.array_equal(got["count"], exp["count"]) and np.array_equal(got["area"], exp["area"])
    assert np.array_equal(got["vmin"], exp["vmin"]) and np.array_equal(got["vmax"], exp["vmax"])
    for f in ("sum", "wsum"):
        e, g = exp[f], got[f]
        fin = np.isfinite(e)
        assert np.array_equal(np.isnan(g), np.isnan(e)) and np.array_equal(g[np.isinf(e)], e[np.isinf(e)])
        assert not fin.all()
