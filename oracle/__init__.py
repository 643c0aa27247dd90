"""CPU oracle for the UV-atlas layer-editing path -- TEST INFRASTRUCTURE ONLY.

Plain, slow, obviously correct restatements of each step (see ``lcl_oracle.c``),
wrapped for numpy.  Only the tests, the smoke check and the benchmark's CPU
baseline / reference arm use this package; the product library never does, and it
shares no code with it.

Layouts (shared data formats, each side has its own code for them):
* position planes: three int32 planes X, Y, Z of H rows x W texels, row 0 at v = 0;
  an uncovered texel holds (INT32_MIN, 0, 0);
* triangle plane: uint32, 0xFFFFFFFF = uncovered;
* coverage bits: bit (y*W + x) of a linear uint32 array;
* tile boxes: 8 int32 per tile (min xyz, count, max xyz, 0);
* sphere stroke record: int32 cx, cy, cz, pad; int64 r2; uint32 label, flags (32 bytes).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from .build import build_oracle, library_path

_lib = None
NONE = 0xFFFFFFFF
SUPER = 16          # tiles per super-tile side
AND, OR, XOR, MASK = 0, 1, 2, 3
NOT_A, NOT_B, NOT_OUT = 1, 2, 4
OPS = {"and": AND, "or": OR, "xor": XOR, "mask": MASK}

SPHERE_DTYPE = np.dtype([("cx", "<i4"), ("cy", "<i4"), ("cz", "<i4"), ("pad", "<i4"),
                         ("r2", "<i8"), ("label", "<u4"), ("flags", "<u4")])
assert SPHERE_DTYPE.itemsize == 32


class OracleError(RuntimeError):
    pass


def lib():
    global _lib
    if _lib is None:
        path = library_path()
        if not os.path.exists(path):
            build_oracle()
        _lib = C.CDLL(path)
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _chk(rc, what):
    if rc != 0:
        raise OracleError(f"{what} failed with status {rc}")


def _f3(v):
    return (C.c_float * 3)(*[float(x) for x in v])


def quant_params(pos: np.ndarray):
    """(bbox_min float32[3], scale float64) of the 21-bit grid."""
    pos = np.ascontiguousarray(pos, dtype=np.float32)
    mn = (C.c_float * 3)()
    s = C.c_double()
    _chk(lib().orc_quant_params(_p(pos), C.c_int64(pos.shape[0]), mn, C.byref(s)), "quant_params")
    return np.array(list(mn), dtype=np.float32), float(s.value)


def quantize(pos, mn, S):
    pos = np.ascontiguousarray(pos, dtype=np.float32)
    q = np.empty((pos.shape[0], 3), dtype=np.int32)
    _chk(lib().orc_quantize(_p(pos), C.c_int64(pos.shape[0]), _f3(mn), C.c_double(S), _p(q)), "quantize")
    return q


class Atlas:
    """Oracle atlas for rows [y0, y1) of a W x H texture (full texture by default)."""

    def __init__(self, mesh, W, H, tile=32, y0=0, y1=None, quant=None):
        y1 = H if y1 is None else y1
        self.W, self.H, self.T, self.y0, self.y1 = W, H, tile, y0, y1
        self.mn, self.S = quant_params(mesh.pos) if quant is None else quant
        rows = y1 - y0
        self.px = np.empty((rows, W), np.int32)
        self.py = np.empty((rows, W), np.int32)
        self.pz = np.empty((rows, W), np.int32)
        self.tri = np.empty((rows, W), np.uint32)
        _chk(lib().orc_atlas(_p(mesh.pos), C.c_int64(mesh.pos.shape[0]), _p(mesh.uv), C.c_int64(mesh.uv.shape[0]),
                             _p(mesh.tri_pos), _p(mesh.tri_uv), C.c_int64(mesh.n_tri), _f3(self.mn),
                             C.c_double(self.S), C.c_int32(W), C.c_int32(H), C.c_int32(y0), C.c_int32(y1),
                             _p(self.px), _p(self.py), _p(self.pz), _p(self.tri)), "atlas")
        self.area_w = np.empty(mesh.n_tri, np.uint64)
        _chk(lib().orc_area_weights(_p(mesh.pos), _p(mesh.uv), _p(mesh.tri_pos), _p(mesh.tri_uv),
                                    C.c_int64(mesh.n_tri), _f3(self.mn), C.c_double(self.S), C.c_int32(W),
                                    C.c_int32(H), _p(self.area_w)), "area_weights")

    @property
    def n_texels(self):
        return (self.y1 - self.y0) * self.W

    def covered(self):
        return self.tri != NONE

    def cover_bits(self):
        rows = self.y1 - self.y0
        bits = np.empty((rows * self.W + 31) // 32, np.uint32)
        _chk(lib().orc_cover_bits(C.c_int32(self.W), C.c_int32(rows), _p(self.tri), _p(bits)), "cover_bits")
        return bits

    def tile_aabb(self):
        """Tile boxes of the rows this atlas holds, tiles counted from its first row y0."""
        rows = self.y1 - self.y0
        ntx, nty = -(-self.W // self.T), -(-rows // self.T)
        box = np.empty((nty * ntx, 8), np.int32)
        _chk(lib().orc_tile_aabb(C.c_int32(self.W), C.c_int32(rows), C.c_int32(self.T), _p(self.px),
                                 _p(self.py), _p(self.pz), _p(self.tri), _p(box)), "tile_aabb")
        return box

    def super_aabb(self, box=None):
        box = self.tile_aabb() if box is None else box
        ntx, nty = -(-self.W // self.T), -(-(self.y1 - self.y0) // self.T)
        nsx, nsy = -(-ntx // SUPER), -(-nty // SUPER)
        sbox = np.empty((nsy * nsx, 8), np.int32)
        _chk(lib().orc_super_aabb(C.c_int32(ntx), C.c_int32(nty), C.c_int32(SUPER), _p(box), _p(sbox)),
             "super_aabb")
        return sbox


def sphere_stroke(mn, S, centre, radius, label):
    out = np.zeros(1, SPHERE_DTYPE)
    c = (C.c_double * 3)(*[float(x) for x in centre])
    _chk(lib().orc_sphere_stroke(_f3(mn), C.c_double(S), c, C.c_double(float(radius)), C.c_uint32(int(label)),
                                 _p(out)), "sphere_stroke")
    return out[0]


def sphere_records(mn, S, centres, radii, labels):
    recs = np.zeros(len(radii), SPHERE_DTYPE)
    for k in range(len(radii)):
        recs[k] = sphere_stroke(mn, S, centres[k], radii[k], labels[k])
    return recs


def select_sphere(atlas: Atlas, layer: np.ndarray, strokes: np.ndarray):
    """Applies strokes in order to ``layer`` (in place, rows of the atlas window); returns hits."""
    assert layer.shape == atlas.tri.shape and layer.flags["C_CONTIGUOUS"]
    strokes = np.ascontiguousarray(strokes, dtype=SPHERE_DTYPE)
    hits = np.zeros(len(strokes), np.uint64)
    _chk(lib().orc_select_sphere(C.c_int64(atlas.n_texels), _p(atlas.px), _p(atlas.py), _p(atlas.pz),
                                 _p(atlas.tri), _p(layer), C.c_int(layer.itemsize), _p(strokes),
                                 C.c_int32(len(strokes)), _p(hits)), "select_sphere")
    return hits


def select_sphere_2d(atlas: Atlas, layer: np.ndarray, strokes: np.ndarray):
    """Like select_sphere, on the whole texture, with texture padding for strokes whose flags ask
    for it (radius = flags & 15, thickness = (flags >> 4) & 15).  Returns (hits, padded)."""
    assert atlas.y0 == 0 and atlas.y1 == atlas.H and layer.shape == atlas.tri.shape
    strokes = np.ascontiguousarray(strokes, dtype=SPHERE_DTYPE)
    hits = np.zeros(len(strokes), np.uint64)
    padded = np.zeros(len(strokes), np.uint64)
    _chk(lib().orc_select_sphere_2d(C.c_int32(atlas.W), C.c_int32(atlas.H), _p(atlas.px), _p(atlas.py), _p(atlas.pz),
                                    _p(atlas.tri), _p(layer), C.c_int(layer.itemsize), _p(strokes),
                                    C.c_int32(len(strokes)), _p(hits), _p(padded)), "select_sphere_2d")
    return hits, padded


def pad_flags(radius, thickness):
    return int(radius) | (int(thickness) << 4)


def camera_mq(vp, mn, S):
    vp = np.ascontiguousarray(vp, dtype=np.float64).reshape(16)
    m = np.empty(16, np.float32)
    _chk(lib().orc_camera_mq(_p(vp), _f3(mn), C.c_double(S), _p(m)), "camera_mq")
    return m


def depth(mesh, mn, S, m, Ws, Hs):
    m = np.ascontiguousarray(m, dtype=np.float32)
    d = np.empty((Hs, Ws), np.float32)
    _chk(lib().orc_depth(_p(mesh.pos), _p(mesh.tri_pos), C.c_int64(mesh.n_tri), _f3(mn), C.c_double(S), _p(m),
                         C.c_int32(Ws), C.c_int32(Hs), _p(d)), "depth")
    return d


def select_lasso(atlas: Atlas, layer, m, dmap, poly, label, bias=2.0 ** -10, want_ambiguous=True):
    """One lasso (screen-pixel polygon) on ``layer`` in place; returns (hits, ambiguous mask)."""
    assert layer.shape == atlas.tri.shape
    m = np.ascontiguousarray(m, dtype=np.float32)
    poly = np.ascontiguousarray(poly, dtype=np.float32)
    Hs, Ws = dmap.shape
    hits = np.zeros(1, np.uint64)
    amb = np.zeros(atlas.tri.shape, np.uint8) if want_ambiguous else None
    _chk(lib().orc_select_lasso(C.c_int64(atlas.n_texels), _p(atlas.px), _p(atlas.py), _p(atlas.pz),
                                _p(atlas.tri), _p(layer), C.c_int(layer.itemsize), _p(m), C.c_int32(Ws),
                                C.c_int32(Hs), _p(np.ascontiguousarray(dmap, np.float32)), _p(poly),
                                C.c_int32(poly.shape[0]), C.c_uint32(int(label)), C.c_float(bias), _p(hits),
                                _p(amb)), "select_lasso")
    return int(hits[0]), amb


def select_tool(atlas: Atlas, layer, m, dmap, centre, size, shape=None, label=1, bias=2.0 ** -10,
                want_ambiguous=True):
    """The paper's editing tool: a window of size = (tw, th) pixels centred at centre = (px, py) on the
    screen, masked by `shape` (uint8 [H_m, W_m], row 0 at the bottom) or, if None, by the inscribed
    circle.  Applies it to ``layer`` in place; returns (hits, ambiguous mask)."""
    assert layer.shape == atlas.tri.shape
    m = np.ascontiguousarray(m, dtype=np.float32)
    Hs, Ws = dmap.shape
    hits = np.zeros(1, np.uint64)
    amb = np.zeros(atlas.tri.shape, np.uint8) if want_ambiguous else None
    sh = None if shape is None else np.ascontiguousarray(shape, dtype=np.uint8)
    sw, shh = (0, 0) if sh is None else (sh.shape[1], sh.shape[0])
    _chk(lib().orc_select_tool(C.c_int64(atlas.n_texels), _p(atlas.px), _p(atlas.py), _p(atlas.pz), _p(atlas.tri),
                               _p(layer), C.c_int(layer.itemsize), _p(m), C.c_int32(Ws), C.c_int32(Hs),
                               _p(np.ascontiguousarray(dmap, np.float32)), C.c_float(centre[0]), C.c_float(centre[1]),
                               C.c_float(size[0]), C.c_float(size[1]), _p(sh), C.c_int32(sw), C.c_int32(shh),
                               C.c_uint32(int(label)), C.c_float(bias), _p(hits), _p(amb)), "select_tool")
    return int(hits[0]), amb


def select_tool_2d(atlas: Atlas, layer, m, dmap, centre, size, shape=None, label=1, bias=2.0 ** -10, flags=0):
    """select_tool on the whole texture with texture padding (flags = radius | thickness << 4).
    Returns (hits, padded, ambiguous mask)."""
    assert atlas.y0 == 0 and atlas.y1 == atlas.H and layer.shape == atlas.tri.shape
    m = np.ascontiguousarray(m, dtype=np.float32)
    Hs, Ws = dmap.shape
    hits = np.zeros(1, np.uint64)
    padded = np.zeros(1, np.uint64)
    amb = np.zeros(atlas.tri.shape, np.uint8)
    sh = None if shape is None else np.ascontiguousarray(shape, dtype=np.uint8)
    sw, shh = (0, 0) if sh is None else (sh.shape[1], sh.shape[0])
    _chk(lib().orc_select_tool_2d(C.c_int32(atlas.W), C.c_int32(atlas.H), _p(atlas.px), _p(atlas.py), _p(atlas.pz),
                                  _p(atlas.tri), _p(layer), C.c_int(layer.itemsize), _p(m), C.c_int32(Ws),
                                  C.c_int32(Hs), _p(np.ascontiguousarray(dmap, np.float32)), C.c_float(centre[0]),
                                  C.c_float(centre[1]), C.c_float(size[0]), C.c_float(size[1]), _p(sh), C.c_int32(sw),
                                  C.c_int32(shh), C.c_uint32(int(label)), C.c_float(bias), C.c_uint32(int(flags)),
                                  _p(hits), _p(padded), _p(amb)), "select_tool_2d")
    return int(hits[0]), int(padded[0]), amb


def overlay(atlas: Atlas, a, b, op, flags=0):
    out = np.empty_like(a)
    op = OPS[op] if isinstance(op, str) else int(op)
    _chk(lib().orc_overlay(C.c_int64(atlas.n_texels), _p(atlas.tri), _p(np.ascontiguousarray(a)),
                           _p(np.ascontiguousarray(b)), _p(out), C.c_int(a.itemsize), C.c_int(op),
                           C.c_uint32(flags)), "overlay")
    return out


def label_area(atlas: Atlas, layer, n_labels):
    count = np.empty(n_labels, np.uint64)
    area = np.empty(n_labels, np.uint64)
    _chk(lib().orc_label_area(C.c_int64(atlas.n_texels), _p(np.ascontiguousarray(layer)), C.c_int(layer.itemsize),
                              _p(atlas.tri), _p(atlas.area_w), C.c_uint32(n_labels), _p(count), _p(area)),
         "label_area")
    return count, area


# ---------------------------------------------------------------------------------------
# Numeric layers (Section 4.2): data texture + mask texture.  Masks here are uint8 arrays
# (one byte per texel, 0 or 1) of the layer's shape.
# ---------------------------------------------------------------------------------------

NUM_TYPES = {"u8": 0x11, "u16": 0x12, "u32": 0x14, "i8": 0x21, "i16": 0x22, "i32": 0x24, "f16": 0x32, "f32": 0x34}
NUM_NP = {"u8": np.uint8, "u16": np.uint16, "u32": np.uint32, "i8": np.int8, "i16": np.int16, "i32": np.int32,
          "f16": np.float16, "f32": np.float32}
ARITH = {"add": 0, "sub": 1, "mul": 2, "div": 3, "min": 4, "max": 5}
CMP = {"lt": 0, "le": 1, "gt": 2, "ge": 3, "eq": 4, "ne": 5}
ERASE = 0x100   # numeric stroke flag: clear the mask (and write 0) instead of storing the value


def value_bits(value, ntype):
    """Bits of `value` in numeric type `ntype` (numpy's own conversion: the caller-side encoding)."""
    a = np.array([value], dtype=NUM_NP[ntype])
    return int(a.view({1: np.uint8, 2: np.uint16, 4: np.uint32}[a.itemsize])[0])


def half_to_float(bits):
    """binary16 bits -> float32 values (the oracle's own decoder)."""
    bits = np.ascontiguousarray(bits, dtype=np.uint16)
    out = np.empty(bits.shape, np.float32)
    lib().orc_half_to_float_n(_p(bits), C.c_int64(bits.size), _p(out))
    return out


def float_to_half(x):
    """float32 values -> binary16 bits, round to nearest even (the oracle's own encoder)."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    out = np.empty(x.shape, np.uint16)
    lib().orc_float_to_half_n(_p(x), C.c_int64(x.size), _p(out))
    return out


def _num_edit(data, mask, sel, value_bits_, flags):
    """Stores one edit's selection into a numeric layer: the selected value into the data texture and
    true into the mask texture (Section 4.3.1, last step); with ERASE, 0 and false."""
    raw = data.view({1: np.uint8, 2: np.uint16, 4: np.uint32}[data.itemsize])
    if flags & ERASE:
        raw[sel] = 0
        mask[sel] = 0
    else:
        raw[sel] = value_bits_
        mask[sel] = 1


def num_select_sphere(atlas: Atlas, data, mask, strokes):
    """Sphere strokes on a numeric layer, in order: each stroke selects what select_sphere_2d
    selects for it (padding included) and stores its value bits (the record's `label` field) and a
    set mask there, or 0 and a clear mask with ERASE.  Returns (hits, padded) per stroke."""
    strokes = np.ascontiguousarray(strokes, dtype=SPHERE_DTYPE)
    hits = np.zeros(len(strokes), np.uint64)
    padded = np.zeros(len(strokes), np.uint64)
    for k, s in enumerate(strokes):
        one = s.copy()
        one["label"] = 1
        one["flags"] = int(s["flags"]) & 0xFF
        sel = np.zeros(atlas.tri.shape, np.uint8)
        h, p = select_sphere_2d(atlas, sel, np.array([one], SPHERE_DTYPE))
        hits[k], padded[k] = h[0], p[0]
        _num_edit(data, mask, sel == 1, int(s["label"]), int(s["flags"]))
    return hits, padded


def num_select_lasso(atlas: Atlas, data, mask, m, dmap, poly, value_bits_, flags=0, bias=2.0 ** -10):
    """A lasso on a numeric layer: the texels select_lasso_2d selects or pads (flags & 0xFF) get the
    value (or are erased with ERASE).  Returns (hits, ambiguous mask)."""
    sel = np.zeros(atlas.tri.shape, np.uint8)
    h, _, amb = select_lasso_2d(atlas, sel, m, dmap, poly, 1, bias, flags & 0xFF)
    _num_edit(data, mask, sel == 1, value_bits_, flags)
    return h, amb


def num_select_tool(atlas: Atlas, data, mask, m, dmap, centre, size, shape=None, value_bits_=0, flags=0,
                    bias=2.0 ** -10):
    """The paper's tool on a numeric layer (padding as in select_tool_2d from flags & 0xFF).
    Returns (hits, padded, ambiguous mask)."""
    sel = np.zeros(atlas.tri.shape, np.uint8)
    h, p, amb = select_tool_2d(atlas, sel, m, dmap, centre, size, shape, 1, bias, flags & 0xFF)
    _num_edit(data, mask, sel == 1, value_bits_, flags)
    return h, p, amb


def num_arith(atlas: Atlas, ntype, a, ma, b, mb, op, scalar_bits=0):
    """Arithmetic overlay (b None: the scalar); returns (out data, out mask)."""
    out = np.empty_like(a)
    mout = np.empty(a.shape, np.uint8)
    _chk(lib().orc_num_arith(C.c_int64(atlas.n_texels), _p(atlas.tri), C.c_int(NUM_TYPES[ntype]),
                             _p(np.ascontiguousarray(a)), _p(np.ascontiguousarray(ma, np.uint8)),
                             _p(None if b is None else np.ascontiguousarray(b)),
                             _p(None if mb is None else np.ascontiguousarray(mb, np.uint8)),
                             C.c_uint32(int(scalar_bits)), _p(out), _p(mout), C.c_int(ARITH[op])), "num_arith")
    return out, mout


def num_select(atlas: Atlas, ntype, data, mask, cmp, threshold_bits, layer, label):
    """Selection by value into a label layer (in place); returns hits."""
    hits = np.zeros(1, np.uint64)
    _chk(lib().orc_num_select(C.c_int64(atlas.n_texels), _p(atlas.tri), C.c_int(NUM_TYPES[ntype]),
                              _p(np.ascontiguousarray(data)), _p(np.ascontiguousarray(mask, np.uint8)),
                              C.c_int(CMP[cmp]), C.c_uint32(int(threshold_bits)), _p(layer), C.c_int(layer.itemsize),
                              C.c_uint32(int(label)), _p(hits)), "num_select")
    return int(hits[0])


def num_stats(atlas: Atlas, ntype, data, mask, zones, n_labels):
    """Zonal statistics; returns a dict of arrays count, area (uint64), vmin, vmax, sum, wsum (float64)."""
    r = {k: np.empty(n_labels, np.uint64) for k in ("count", "area")}
    r.update({k: np.empty(n_labels, np.float64) for k in ("vmin", "vmax", "sum", "wsum")})
    zb = 0 if zones is None else zones.itemsize
    _chk(lib().orc_num_stats(C.c_int64(atlas.n_texels), _p(atlas.tri), _p(atlas.area_w), C.c_int(NUM_TYPES[ntype]),
                             _p(np.ascontiguousarray(data)), _p(np.ascontiguousarray(mask, np.uint8)),
                             _p(None if zones is None else np.ascontiguousarray(zones)), C.c_int(zb),
                             C.c_uint32(n_labels), _p(r["count"]), _p(r["area"]), _p(r["vmin"]), _p(r["vmax"]),
                             _p(r["sum"]), _p(r["wsum"])), "num_stats")
    return r


def select_lasso_2d(atlas: Atlas, layer, m, dmap, poly, label, bias=2.0 ** -10, flags=0):
    """select_lasso on the whole texture with texture padding (flags = radius | thickness << 4).
    Returns (hits, padded, ambiguous mask)."""
    assert atlas.y0 == 0 and atlas.y1 == atlas.H and layer.shape == atlas.tri.shape
    m = np.ascontiguousarray(m, dtype=np.float32)
    poly = np.ascontiguousarray(poly, dtype=np.float32)
    Hs, Ws = dmap.shape
    hits = np.zeros(1, np.uint64)
    padded = np.zeros(1, np.uint64)
    amb = np.zeros(atlas.tri.shape, np.uint8)
    _chk(lib().orc_select_lasso_2d(C.c_int32(atlas.W), C.c_int32(atlas.H), _p(atlas.px), _p(atlas.py), _p(atlas.pz),
                                   _p(atlas.tri), _p(layer), C.c_int(layer.itemsize), _p(m), C.c_int32(Ws),
                                   C.c_int32(Hs), _p(np.ascontiguousarray(dmap, np.float32)), _p(poly),
                                   C.c_int32(poly.shape[0]), C.c_uint32(int(label)), C.c_float(bias),
                                   C.c_uint32(int(flags)), _p(hits), _p(padded), _p(amb)), "select_lasso_2d")
    return int(hits[0]), int(padded[0]), amb
