"""Thin Python binding of the C ABI in include/lcl.h (ctypes).

The functions keep the C names (``lcl_atlas_build`` ...) and only marshal arguments:
every step of the path runs in the CUDA library ``liblcl.so``.  PyTorch provides device
memory and streams.  If the library has not been built, loading fails loudly: there is
no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liblcl.so")
# The same library built with bounds checks in every kernel (LCL_DEBUG_BOUNDS); loaded instead of
# liblcl.so when the environment variable LCL_DEBUG_BOUNDS is 1.
DEBUG_LIB_PATH = os.path.join(HERE, "liblcl_debug.so")

LCL_OK = 0
STATUS = {0: "LCL_OK", 1: "LCL_ERR_INVALID_ARG", 2: "LCL_ERR_OUT_OF_MEMORY", 3: "LCL_ERR_CUDA",
          4: "LCL_ERR_UNSUPPORTED", 5: "LCL_ERR_TIMEOUT", 6: "LCL_ERR_INTERNAL"}
LCL_U8, LCL_U16 = 1, 2
LCL_AND, LCL_OR, LCL_XOR, LCL_MASK = 0, 1, 2, 3
LCL_NOT_A, LCL_NOT_B, LCL_NOT_OUT = 1, 2, 4
OPS = {"and": LCL_AND, "or": LCL_OR, "xor": LCL_XOR, "mask": LCL_MASK}
NO_TRIANGLE = 0xFFFFFFFF
SUPER = 16
DEFAULT_BIAS = 2.0 ** -10

EXPORTS = ["lcl_atlas_bytes", "lcl_atlas_bind", "lcl_atlas_bind_band", "lcl_atlas_rows", "lcl_atlas_workspace_bytes", "lcl_atlas_build",
           "lcl_quantize_sphere", "lcl_quantize_spheres", "lcl_camera_from_vp", "lcl_select_workspace_bytes", "lcl_select_sphere",
           "lcl_select_sphere_static", "lcl_depth_workspace_bytes", "lcl_depth_render", "lcl_select_lasso", "lcl_select_tool",
           "lcl_batch_limits_of", "lcl_batch_workspace_bytes", "lcl_batch_staging_bytes", "lcl_batch_upload",
           "lcl_batch_launch", "lcl_batch_edit", "lcl_batch_tune",
           "lcl_overlay", "lcl_label_area", "lcl_numeric_sphere", "lcl_numeric_lasso", "lcl_numeric_tool",
           "lcl_numeric_arith", "lcl_numeric_select", "lcl_numeric_stats",
           "lcl_pool_create", "lcl_pool_acquire", "lcl_pool_release", "lcl_pool_stats_get", "lcl_pool_destroy",
           "lcl_status_str", "lcl_last_error", "lcl_kernel_launches", "lcl_last_device_status", "lcl_build_flags",
           "lcl_describe_site", "lcl_check_division",
           "lcl_serve_clock", "lcl_serve_create", "lcl_serve_add_model", "lcl_serve_work_bytes",
           "lcl_serve_host_work_bytes", "lcl_serve_start", "lcl_serve_submit", "lcl_serve_poll", "lcl_serve_stats_get",
           "lcl_serve_read_layer", "lcl_serve_destroy"]
LCL_BUILD_BOUNDS_CHECKS = 1


class lcl_mesh(C.Structure):
    _fields_ = [("pos", C.c_void_p), ("n_pos", C.c_int64), ("uv", C.c_void_p), ("n_uv", C.c_int64),
                ("tri_pos", C.c_void_p), ("tri_uv", C.c_void_p), ("n_tri", C.c_int64)]


class lcl_atlas(C.Structure):
    _fields_ = [("width", C.c_int32), ("height", C.c_int32), ("tile", C.c_int32),
                ("tiles_x", C.c_int32), ("tiles_y", C.c_int32), ("supers_x", C.c_int32), ("supers_y", C.c_int32),
                ("row0", C.c_int32), ("n_tri", C.c_int64),
                ("pos_x", C.c_void_p), ("pos_y", C.c_void_p), ("pos_z", C.c_void_p), ("tri", C.c_void_p),
                ("cover", C.c_void_p), ("tile_box", C.c_void_p), ("super_box", C.c_void_p), ("area_w", C.c_void_p),
                ("bbox_min", C.c_float * 3), ("tex_height", C.c_int32), ("scale", C.c_double)]


class lcl_sphere(C.Structure):
    _fields_ = [("cx", C.c_int32), ("cy", C.c_int32), ("cz", C.c_int32), ("_pad", C.c_int32),
                ("r2", C.c_int64), ("label", C.c_uint32), ("flags", C.c_uint32)]


class lcl_camera(C.Structure):
    _fields_ = [("m", C.c_float * 16), ("width", C.c_int32), ("height", C.c_int32)]


class lcl_tool(C.Structure):
    _fields_ = [("px", C.c_float), ("py", C.c_float), ("tw", C.c_float), ("th", C.c_float),
                ("shape", C.c_void_p), ("shape_w", C.c_int32), ("shape_h", C.c_int32), ("flags", C.c_uint32),
                ("_pad", C.c_int32)]


class lcl_numeric_layer(C.Structure):
    _fields_ = [("data", C.c_void_p), ("mask", C.c_void_p), ("type", C.c_int), ("_pad", C.c_int32)]


class lcl_zone_stats(C.Structure):
    _fields_ = [("count", C.c_uint64), ("area", C.c_uint64), ("vmin", C.c_double), ("vmax", C.c_double),
                ("sum", C.c_double), ("wsum", C.c_double)]


class lcl_pool_layer(C.Structure):
    _fields_ = [("data", C.c_void_p), ("mask", C.c_void_p), ("handle", C.c_uint64), ("width", C.c_int32),
                ("height", C.c_int32), ("type", C.c_int32), ("_pad", C.c_int32)]


class lcl_pool_stats(C.Structure):
    _fields_ = [("reserved_bytes", C.c_uint64), ("committed_bytes", C.c_uint64), ("layers", C.c_int64),
                ("arrays", C.c_int32), ("_pad", C.c_int32), ("granularity", C.c_uint64)]


class lcl_batch_model(C.Structure):
    _fields_ = [("atlas", C.POINTER(lcl_atlas)), ("layer", C.c_void_p), ("dtype", C.c_int),
                ("first_stroke", C.c_int32), ("n_strokes", C.c_int32), ("_pad", C.c_int32)]


class lcl_batch_stroke(C.Structure):
    _fields_ = [("kind", C.c_int32), ("lasso", C.c_int32), ("sphere", lcl_sphere)]


class lcl_batch_lasso(C.Structure):
    _fields_ = [("camera", lcl_camera), ("depth", C.c_void_p), ("poly_xy", C.c_void_p), ("n_vertices", C.c_int32),
                ("label", C.c_uint32), ("bias", C.c_float), ("flags", C.c_uint32)]


class lcl_serve_config(C.Structure):
    _fields_ = [("arena_bytes", C.c_size_t), ("max_in_flight", C.c_int32), ("max_edits", C.c_int32),
                ("max_queries", C.c_int32), ("max_labels", C.c_int32), ("max_admitting", C.c_int32),
                ("_pad", C.c_int32)]


class lcl_serve_model(C.Structure):
    _fields_ = [("side", C.c_int32), ("tile", C.c_int32), ("n_tri", C.c_int64), ("bbox_min", C.c_float * 3),
                ("n_layers", C.c_int32), ("scale", C.c_double), ("cams", C.c_void_p), ("depth_offsets", C.c_void_p),
                ("n_cams", C.c_int32), ("_pad", C.c_int32), ("host_image", C.c_void_p), ("image_bytes", C.c_size_t),
                ("layer_offset", C.c_size_t), ("layer_stride", C.c_size_t)]


class lcl_serve_done(C.Structure):
    _fields_ = [("tag", C.c_uint64), ("t_done", C.c_double), ("t_launch", C.c_double), ("t_gpu", C.c_double)]


class lcl_serve_stats(C.Structure):
    _fields_ = [("submitted", C.c_uint64), ("done", C.c_uint64), ("epochs", C.c_uint64), ("admissions", C.c_uint64),
                ("spills", C.c_uint64), ("resident_bytes", C.c_uint64), ("resident_models", C.c_uint64),
                ("host_busy_s", C.c_double), ("admitted_bytes", C.c_uint64), ("deferred", C.c_uint64)]


# lcl_serve_request as a numpy record (608 bytes), so a whole trace is one array
SERVE_REQUEST_DTYPE = np.dtype([("t_arrive", "<f8"), ("tag", "<u8"), ("model", "<i4"), ("kind", "<i4"),
                                ("layer", "<i4"), ("label", "<i4"), ("centre", "<f8", (3,)), ("radius", "<f8"),
                                ("cam", "<i4"), ("n_vertices", "<i4"), ("op", "<i4"), ("layer_b", "<i4"),
                                ("n_labels", "<i4"), ("_pad", "<i4"), ("result", "<u8"), ("poly", "<f4", (128,))])
LCL_REQ_SPHERE, LCL_REQ_LASSO, LCL_REQ_QUERY = 0, 1, 2


class lcl_batch_limits(C.Structure):
    _fields_ = [("models", C.c_int32), ("strokes", C.c_int32), ("lassos", C.c_int32), ("_pad", C.c_int32),
                ("supers", C.c_int64), ("tiles", C.c_int64)]


class lcl_batch_config(C.Structure):
    _fields_ = [("threads", C.c_int32), ("ctas_per_sm", C.c_int32), ("split", C.c_int32), ("_pad", C.c_int32)]

    def as_dict(self):
        return {"threads": self.threads, "ctas_per_sm": self.ctas_per_sm, "split": self.split}


LCL_STROKE_SPHERE, LCL_STROKE_LASSO = 0, 1
BATCH_MAX_STROKES = 64

assert C.sizeof(lcl_sphere) == 32 and C.sizeof(lcl_camera) == 72 and C.sizeof(lcl_atlas) == 128
assert C.sizeof(lcl_batch_model) == 32 and C.sizeof(lcl_batch_stroke) == 40 and C.sizeof(lcl_batch_lasso) == 104
assert C.sizeof(lcl_batch_limits) == 32 and C.sizeof(lcl_batch_config) == 16 and C.sizeof(lcl_tool) == 40
assert C.sizeof(lcl_numeric_layer) == 24 and C.sizeof(lcl_zone_stats) == 48
assert C.sizeof(lcl_pool_layer) == 40 and C.sizeof(lcl_pool_stats) == 40
assert C.sizeof(lcl_serve_config) == 32 and C.sizeof(lcl_serve_model) == 96 and C.sizeof(lcl_serve_done) == 32
assert C.sizeof(lcl_serve_stats) == 80 and SERVE_REQUEST_DTYPE.itemsize == 608

SPHERE_DTYPE = np.dtype([("cx", "<i4"), ("cy", "<i4"), ("cz", "<i4"), ("pad", "<i4"),
                         ("r2", "<i8"), ("label", "<u4"), ("flags", "<u4")])


class LclError(RuntimeError):
    def __init__(self, fn, status, msg):
        super().__init__(f"{fn}: {STATUS.get(status, status)}: {msg}")
        self.status = status


_lib = None


def library():
    """Loads liblcl.so (built by __graft_entry__.build() or paper_2501_14807_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    path = DEBUG_LIB_PATH if os.environ.get("LCL_DEBUG_BOUNDS") == "1" else LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build the CUDA library first (python -c 'import "
                           "__graft_entry__ as g; g.build()'); there is no CPU fallback")
    lib = C.CDLL(path)
    P, I32, I64, U32, SZ, F, D = C.c_void_p, C.c_int32, C.c_int64, C.c_uint32, C.c_size_t, C.c_float, C.c_double
    st = C.c_int
    sig = {
        "lcl_atlas_bytes": (SZ, [I32, I32, I32, I64]),
        "lcl_atlas_bind": (st, [P, SZ, I32, I32, I32, I64, C.POINTER(lcl_atlas)]),
        "lcl_atlas_rows": (st, [C.POINTER(lcl_atlas), I32, I32, C.POINTER(lcl_atlas)]),
        "lcl_atlas_bind_band": (st, [P, SZ, I32, I32, I32, I32, I32, I64, C.POINTER(lcl_atlas)]),
        "lcl_atlas_workspace_bytes": (SZ, [C.POINTER(lcl_mesh), I32, I32]),
        "lcl_atlas_build": (st, [C.POINTER(lcl_mesh), C.POINTER(lcl_atlas), P, SZ, P]),
        "lcl_quantize_sphere": (st, [C.POINTER(lcl_atlas), C.POINTER(D), D, U32, C.POINTER(lcl_sphere)]),
        "lcl_quantize_spheres": (st, [C.POINTER(lcl_atlas), I32, P, P, P, P]),
        "lcl_camera_from_vp": (st, [C.POINTER(lcl_atlas), C.POINTER(D), I32, I32, C.POINTER(lcl_camera)]),
        "lcl_select_workspace_bytes": (SZ, [C.POINTER(lcl_atlas), I32]),
        "lcl_select_sphere": (st, [C.POINTER(lcl_atlas), P, C.c_int, P, I32, P, P, SZ, P]),
        "lcl_select_sphere_static": (st, [C.POINTER(lcl_atlas), P, C.c_int, P, I32, P, P]),
        "lcl_depth_workspace_bytes": (SZ, [C.POINTER(lcl_mesh), I32, I32]),
        "lcl_depth_render": (st, [C.POINTER(lcl_mesh), C.POINTER(lcl_atlas), C.POINTER(lcl_camera), P, P, SZ, P]),
        "lcl_select_lasso": (st, [C.POINTER(lcl_atlas), P, C.c_int, C.POINTER(lcl_camera), P, P, I32, U32, U32, F, P,
                                  P, SZ, P]),
        "lcl_select_tool": (st, [C.POINTER(lcl_atlas), P, C.c_int, C.POINTER(lcl_camera), P, C.POINTER(lcl_tool), U32, F,
                                 P, P, SZ, P]),
        "lcl_batch_limits_of": (st, [C.POINTER(lcl_batch_model), I32, I32, I32, C.POINTER(lcl_batch_limits)]),
        "lcl_batch_workspace_bytes": (SZ, [C.POINTER(lcl_batch_limits)]),
        "lcl_batch_staging_bytes": (SZ, [C.POINTER(lcl_batch_limits)]),
        "lcl_batch_upload": (st, [C.POINTER(lcl_batch_limits), C.POINTER(lcl_batch_model), I32,
                                  C.POINTER(lcl_batch_stroke), I32, C.POINTER(lcl_batch_lasso), I32, P, SZ, P, SZ, P]),
        "lcl_batch_launch": (st, [C.POINTER(lcl_batch_limits), C.POINTER(lcl_batch_config), P, SZ, P]),
        "lcl_batch_edit": (st, [C.POINTER(lcl_batch_limits), C.POINTER(lcl_batch_config), C.POINTER(lcl_batch_model),
                                I32, C.POINTER(lcl_batch_stroke), I32, C.POINTER(lcl_batch_lasso), I32, P, SZ, P, SZ,
                                P]),
        "lcl_batch_tune": (st, [C.POINTER(lcl_batch_limits), P, SZ, I32, P, C.POINTER(lcl_batch_config),
                                C.POINTER(C.c_float)]),
        "lcl_overlay": (st, [C.POINTER(lcl_atlas), P, P, P, C.c_int, C.c_int, U32, P]),
        "lcl_label_area": (st, [C.POINTER(lcl_atlas), P, C.c_int, U32, P, P, P]),
        "lcl_numeric_sphere": (st, [C.POINTER(lcl_atlas), C.POINTER(lcl_numeric_layer), P, I32, P, P, SZ, P]),
        "lcl_numeric_lasso": (st, [C.POINTER(lcl_atlas), C.POINTER(lcl_numeric_layer), C.POINTER(lcl_camera), P, P,
                                   I32, U32, U32, F, P, P, SZ, P]),
        "lcl_numeric_tool": (st, [C.POINTER(lcl_atlas), C.POINTER(lcl_numeric_layer), C.POINTER(lcl_camera), P,
                                  C.POINTER(lcl_tool), U32, U32, F, P, P, SZ, P]),
        "lcl_numeric_arith": (st, [C.POINTER(lcl_atlas), C.POINTER(lcl_numeric_layer), C.POINTER(lcl_numeric_layer),
                                   U32, C.POINTER(lcl_numeric_layer), C.c_int, P]),
        "lcl_numeric_select": (st, [C.POINTER(lcl_atlas), C.POINTER(lcl_numeric_layer), C.c_int, U32, P, C.c_int, U32,
                                    P, P]),
        "lcl_numeric_stats": (st, [C.POINTER(lcl_atlas), C.POINTER(lcl_numeric_layer), P, C.c_int, U32, P, P]),
        "lcl_pool_create": (st, [I32, C.POINTER(P)]),
        "lcl_pool_acquire": (st, [P, I32, I32, I32, P, C.POINTER(lcl_pool_layer)]),
        "lcl_pool_release": (st, [P, C.c_uint64, P]),
        "lcl_pool_stats_get": (st, [P, C.POINTER(lcl_pool_stats)]),
        "lcl_pool_destroy": (st, [P]),
        "lcl_status_str": (C.c_char_p, [C.c_int]),
        "lcl_last_error": (C.c_char_p, []),
        "lcl_kernel_launches": (C.c_uint64, []),
        "lcl_last_device_status": (st, [P]),
        "lcl_build_flags": (U32, []),
        "lcl_describe_site": (SZ, [U32, P, SZ]),
        "lcl_check_division": (st, [C.c_uint64, U32, P, P]),
        "lcl_serve_clock": (D, []),
        "lcl_serve_create": (st, [C.POINTER(lcl_serve_config), C.POINTER(P)]),
        "lcl_serve_add_model": (st, [P, C.POINTER(lcl_serve_model), C.POINTER(I32)]),
        "lcl_serve_work_bytes": (SZ, [P]),
        "lcl_serve_host_work_bytes": (SZ, [P]),
        "lcl_serve_start": (st, [P, P, P, SZ, P, SZ]),
        "lcl_serve_submit": (st, [P, P, I32]),
        "lcl_serve_poll": (st, [P, P, I32, C.POINTER(I32)]),
        "lcl_serve_stats_get": (st, [P, C.POINTER(lcl_serve_stats)]),
        "lcl_serve_read_layer": (st, [P, I32, I32, P]),
        "lcl_serve_destroy": (st, [P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _check(fn, status):
    if status != LCL_OK:
        raise LclError(fn, status, library().lcl_last_error().decode())


def _stream(stream):
    if stream is None:
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, torch.cuda.Stream):
        return C.c_void_p(stream.cuda_stream)
    return C.c_void_p(int(stream))


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _addr(a: np.ndarray) -> int:
    """Address of a contiguous numpy array's data."""
    return a.__array_interface__["data"][0]


def _dtype_code(layer: torch.Tensor) -> int:
    if layer.element_size() == 1:
        return LCL_U8
    if layer.element_size() == 2:
        return LCL_U16
    raise ValueError("layers hold uint8 or 16-bit labels")


def _workspace(nbytes, device):
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)


class Mesh:
    """Mesh arrays resident on the device plus their lcl_mesh descriptor."""

    def __init__(self, pos: torch.Tensor, uv: torch.Tensor, tri_pos: torch.Tensor, tri_uv: torch.Tensor):
        for t in (pos, uv, tri_pos, tri_uv):
            assert t.is_cuda and t.is_contiguous()
        self.pos, self.uv, self.tri_pos, self.tri_uv = pos, uv, tri_pos, tri_uv
        self.c = lcl_mesh(pos.data_ptr(), pos.shape[0], uv.data_ptr(), uv.shape[0], tri_pos.data_ptr(),
                          tri_uv.data_ptr(), tri_pos.shape[0])

    @property
    def n_tri(self):
        return int(self.c.n_tri)

    @staticmethod
    def from_host(mesh, device="cuda", non_blocking=False):
        """Copies a host mesh (numpy arrays: pos float32 [n,3], uv float32 [n,2], tri_pos/tri_uv uint32 [n,3])."""
        def up(a, dt):
            t = torch.from_numpy(np.ascontiguousarray(a).view(dt))
            if non_blocking:
                t = t.pin_memory()
            return t.to(device, non_blocking=non_blocking)
        return Mesh(up(mesh.pos, np.float32), up(mesh.uv, np.float32), up(mesh.tri_pos, np.int32),
                    up(mesh.tri_uv, np.int32))


class Atlas:
    """One atlas buffer (device) bound with lcl_atlas_bind, or with band=(y0, y1) a band atlas of
    rows [y0, y1) of a width x height texture (lcl_atlas_bind_band)."""

    def __init__(self, width, height, tile, n_tri, device="cuda", buffer=None, band=None):
        lib = library()
        y0, y1 = (0, height) if band is None else (int(band[0]), int(band[1]))
        nbytes = lib.lcl_atlas_bytes(width, y1 - y0, tile, n_tri) if y1 > y0 else 0
        if nbytes == 0:
            raise LclError("lcl_atlas_bytes", 1, "invalid atlas sizes")
        self.buf = torch.empty(nbytes, dtype=torch.uint8, device=device) if buffer is None else buffer
        self.c = lcl_atlas()
        if band is None:
            _check("lcl_atlas_bind", lib.lcl_atlas_bind(C.c_void_p(self.buf.data_ptr()), nbytes, width, height, tile,
                                                       n_tri, C.byref(self.c)))
        else:
            _check("lcl_atlas_bind_band", lib.lcl_atlas_bind_band(C.c_void_p(self.buf.data_ptr()), nbytes, width,
                                                                 height, y0, y1, tile, n_tri, C.byref(self.c)))

    width = property(lambda s: int(s.c.width))
    height = property(lambda s: int(s.c.height))       # rows this atlas holds
    tile = property(lambda s: int(s.c.tile))
    row0 = property(lambda s: int(s.c.row0))           # first texture row it holds
    tex_height = property(lambda s: int(s.c.tex_height))

    def _view(self, ptr, count, dtype, shape):
        off = ptr - self.buf.data_ptr()
        esz = torch.empty((), dtype=dtype).element_size()
        return self.buf[off:off + count * esz].view(dtype).view(shape)

    def plane(self, name):
        """Device view of pos_x / pos_y / pos_z (int32) or tri (int32 bits of uint32) as [H, W]."""
        return self._view(getattr(self.c, name), self.width * self.height, torch.int32, (self.height, self.width))

    def cover(self):
        n = (self.width * self.height + 31) // 32
        return self._view(self.c.cover, n, torch.int32, (n,))

    def tile_box(self):
        n = self.c.tiles_x * self.c.tiles_y
        return self._view(self.c.tile_box, n * 8, torch.int32, (n, 8))

    def super_box(self):
        n = self.c.supers_x * self.c.supers_y
        return self._view(self.c.super_box, n * 8, torch.int32, (n, 8))

    def area_w(self):
        return self._view(self.c.area_w, int(self.c.n_tri), torch.int64, (int(self.c.n_tri),))

    @property
    def bbox_min(self):
        return np.array(list(self.c.bbox_min), np.float32)

    @property
    def scale(self):
        return float(self.c.scale)


# ---- entry points (same names as the C ABI) ----------------------------------------

def lcl_atlas_bytes(width, height, tile, n_tri):
    return int(library().lcl_atlas_bytes(width, height, tile, n_tri))


def lcl_atlas_workspace_bytes(mesh: Mesh, width, height):
    return int(library().lcl_atlas_workspace_bytes(C.byref(mesh.c), width, height))


def lcl_atlas_build(mesh: Mesh, atlas: Atlas, workspace=None, stream=None):
    ws = workspace if workspace is not None else _workspace(lcl_atlas_workspace_bytes(mesh, atlas.width,
                                                                                      atlas.height), mesh.pos.device)
    _check("lcl_atlas_build", library().lcl_atlas_build(C.byref(mesh.c), C.byref(atlas.c), _ptr(ws), ws.numel(),
                                                        _stream(stream)))
    return atlas


def lcl_atlas_rows(atlas: Atlas, y0, y1):
    out = lcl_atlas()
    _check("lcl_atlas_rows", library().lcl_atlas_rows(C.byref(atlas.c), y0, y1, C.byref(out)))
    view = Atlas.__new__(Atlas)
    view.buf, view.c = atlas.buf, out
    return view


def lcl_quantize_sphere(atlas: Atlas, centre, radius, label):
    out = lcl_sphere()
    c = (C.c_double * 3)(*[float(v) for v in centre])
    _check("lcl_quantize_sphere", library().lcl_quantize_sphere(C.byref(atlas.c), c, float(radius), int(label),
                                                                C.byref(out)))
    rec = np.zeros(1, SPHERE_DTYPE)
    rec[0] = (out.cx, out.cy, out.cz, 0, out.r2, out.label, out.flags)
    return rec[0]


def lcl_quantize_spheres(atlas: Atlas, centres, radii, labels):
    """Stroke records (SPHERE_DTYPE) for n world-space spheres."""
    c = np.ascontiguousarray(centres, dtype=np.float64)
    r = np.ascontiguousarray(radii, dtype=np.float64)
    lab = np.ascontiguousarray(labels, dtype=np.uint32)
    n = r.size
    if c.size != 3 * n or lab.size != n:
        raise ValueError("centres must be n x 3, radii and labels n")
    out = np.zeros(n, SPHERE_DTYPE)
    _check("lcl_quantize_spheres", library().lcl_quantize_spheres(
        C.byref(atlas.c), n, _addr(c), _addr(r), _addr(lab), _addr(out)))
    return out


def lcl_camera_from_vp(atlas: Atlas, vp, width, height):
    out = lcl_camera()
    v = (C.c_double * 16)(*[float(x) for x in np.asarray(vp, np.float64).reshape(16)])
    _check("lcl_camera_from_vp", library().lcl_camera_from_vp(C.byref(atlas.c), v, width, height, C.byref(out)))
    return out


def camera(m, width, height):
    """lcl_camera from a float32[16] matrix already in grid space."""
    cam = lcl_camera()
    for i, x in enumerate(np.asarray(m, np.float32).reshape(16)):
        cam.m[i] = float(x)
    cam.width, cam.height = int(width), int(height)
    return cam


def lcl_select_workspace_bytes(atlas: Atlas, n_strokes):
    return int(library().lcl_select_workspace_bytes(C.byref(atlas.c), int(n_strokes)))


def lcl_select_sphere(atlas: Atlas, layer: torch.Tensor, strokes, hits_out=None, workspace=None, stream=None):
    """Applies sphere strokes (numpy records of SPHERE_DTYPE, in order) to ``layer`` on the device."""
    recs = np.ascontiguousarray(strokes, dtype=SPHERE_DTYPE)
    n = len(recs)
    ws = workspace if workspace is not None else _workspace(lcl_select_workspace_bytes(atlas, n), layer.device)
    _check("lcl_select_sphere", library().lcl_select_sphere(
        C.byref(atlas.c), _ptr(layer), _dtype_code(layer), recs.ctypes.data_as(C.c_void_p), n, _ptr(hits_out),
        _ptr(ws), ws.numel(), _stream(stream)))
    return hits_out


def lcl_select_sphere_static(atlas: Atlas, layer: torch.Tensor, strokes, hits_out=None, stream=None):
    """lcl_select_sphere with the library's built-in scratch array instead of a workspace (allocates
    nothing; see include/lcl.h for its limits and its one-stream rule)."""
    recs = np.ascontiguousarray(strokes, dtype=SPHERE_DTYPE)
    _check("lcl_select_sphere_static", library().lcl_select_sphere_static(
        C.byref(atlas.c), _ptr(layer), _dtype_code(layer), recs.ctypes.data_as(C.c_void_p), len(recs),
        _ptr(hits_out), _stream(stream)))
    return hits_out


def lcl_depth_workspace_bytes(mesh: Mesh, width, height):
    return int(library().lcl_depth_workspace_bytes(C.byref(mesh.c), width, height))


def lcl_depth_render(mesh: Mesh, atlas: Atlas, cam: lcl_camera, depth: torch.Tensor, workspace=None, stream=None):
    ws = workspace if workspace is not None else _workspace(lcl_depth_workspace_bytes(mesh, cam.width, cam.height),
                                                            depth.device)
    _check("lcl_depth_render", library().lcl_depth_render(C.byref(mesh.c), C.byref(atlas.c), C.byref(cam),
                                                          _ptr(depth), _ptr(ws), ws.numel(), _stream(stream)))
    return depth


def lcl_select_lasso(atlas: Atlas, layer: torch.Tensor, cam: lcl_camera, depth: torch.Tensor, poly, label,
                     bias=DEFAULT_BIAS, hits_out=None, workspace=None, stream=None, flags=0):
    """A lasso (screen polygon) on ``layer``; flags: texture padding (pad_flags)."""
    poly = np.ascontiguousarray(poly, dtype=np.float32)
    ws = workspace if workspace is not None else _workspace(lcl_select_workspace_bytes(atlas, 1), layer.device)
    _check("lcl_select_lasso", library().lcl_select_lasso(
        C.byref(atlas.c), _ptr(layer), _dtype_code(layer), C.byref(cam), _ptr(depth),
        poly.ctypes.data_as(C.c_void_p), poly.shape[0], int(label), int(flags), float(bias), _ptr(hits_out),
        _ptr(ws), ws.numel(), _stream(stream)))
    return hits_out


def pad_flags(radius, thickness):
    """Texture padding flags of a sphere stroke or a tool: kernel radius and outline thickness (<= 8)."""
    return int(radius) | (int(thickness) << 4)


def make_tool(centre, size, shape=None, flags=0):
    """lcl_tool for a window of size = (tw, th) pixels centred at centre = (px, py); shape: None (the
    inscribed circle) or a device uint8 tensor [shape_h, shape_w], row 0 at the bottom; flags:
    texture padding (pad_flags)."""
    t = lcl_tool()
    t.flags = int(flags)
    t.px, t.py = float(centre[0]), float(centre[1])
    t.tw, t.th = float(size[0]), float(size[1])
    if shape is not None:
        assert shape.dtype == torch.uint8 and shape.is_cuda and shape.is_contiguous() and shape.dim() == 2
        t.shape = shape.data_ptr()
        t.shape_h, t.shape_w = int(shape.shape[0]), int(shape.shape[1])
    return t


def lcl_select_tool(atlas: Atlas, layer: torch.Tensor, cam: lcl_camera, depth: torch.Tensor, tool: lcl_tool, label,
                    bias=DEFAULT_BIAS, hits_out=None, workspace=None, stream=None):
    """The paper's editing tool (window + shape or inscribed circle, depth test) on ``layer``."""
    ws = workspace if workspace is not None else _workspace(lcl_select_workspace_bytes(atlas, 1), layer.device)
    _check("lcl_select_tool", library().lcl_select_tool(
        C.byref(atlas.c), _ptr(layer), _dtype_code(layer), C.byref(cam), _ptr(depth), C.byref(tool), int(label),
        float(bias), _ptr(hits_out), _ptr(ws), ws.numel(), _stream(stream)))
    return hits_out


BATCH_STROKE_DTYPE = np.dtype([("kind", "<i4"), ("lasso", "<i4"), ("cx", "<i4"), ("cy", "<i4"), ("cz", "<i4"),
                               ("pad", "<i4"), ("r2", "<i8"), ("label", "<u4"), ("flags", "<u4")])
assert BATCH_STROKE_DTYPE.itemsize == C.sizeof(lcl_batch_stroke)


def batch_limits(models=0, strokes=0, lassos=0, supers=0, tiles=0):
    """Capacity of a batch workspace (see lcl_batch_limits)."""
    return lcl_batch_limits(int(models), int(strokes), int(lassos), 0, int(supers), int(tiles))


def limits_max(a: lcl_batch_limits, b: lcl_batch_limits):
    """Field-wise maximum of two limits."""
    return batch_limits(max(a.models, b.models), max(a.strokes, b.strokes), max(a.lassos, b.lassos),
                        max(a.supers, b.supers), max(a.tiles, b.tiles))


def limits_fit(inner: lcl_batch_limits, outer: lcl_batch_limits):
    return (inner.models <= outer.models and inner.strokes <= outer.strokes and inner.lassos <= outer.lassos and
            inner.supers <= outer.supers and inner.tiles <= outer.tiles)


def batch_workspace(limits: lcl_batch_limits, device):
    """A device workspace for batches within `limits`."""
    n = int(library().lcl_batch_workspace_bytes(C.byref(limits)))
    if n == 0:
        raise ValueError("invalid batch limits")
    return torch.empty(n, dtype=torch.uint8, device=device)


def batch_config(threads=256, ctas_per_sm=0, split=1):
    return lcl_batch_config(int(threads), int(ctas_per_sm), int(split), 0)


class Batch:
    """Arguments of one batched edit, kept alive for lcl_batch_upload / lcl_batch_edit.

    models: list of (Atlas, layer tensor); queues: per model, a list of ("sphere", record) or
    ("lasso", (camera, depth tensor, polygon float32 [n, 2], label, bias[, flags])) in queue order
    (flags, and a sphere record's flags: texture padding, pad_flags).
    limits: capacity of the workspace (lcl_batch_limits); by default exactly this batch's.  A
    workspace with larger limits can take many different batches under one launch shape (and one
    captured graph, see BatchGraph).  config: launch shape (lcl_batch_config) or None (default);
    lcl_batch_tune sets it.  workspace / staging: optional reusable buffers (device uint8 / pinned
    host uint8); new ones are allocated if they are missing or too small.  A pinned staging is read
    by the copy that lcl_batch_upload enqueues, so it is not rewritten before that copy has run."""

    def __init__(self, models, queues, workspace=None, staging=None, limits=None, config=None):
        assert len(models) == len(queues)
        self._keep = []
        n_total = sum(len(q) for q in queues)
        rows = []
        lassos = []
        self.models = (lcl_batch_model * max(len(models), 1))()
        k = 0
        for i, ((atlas, layer), queue) in enumerate(zip(models, queues)):
            if len(queue) > BATCH_MAX_STROKES:
                raise ValueError("at most 64 queued strokes per model per batch")
            bm = self.models[i]
            bm.atlas = C.pointer(atlas.c)
            bm.layer = layer.data_ptr()
            bm.dtype = _dtype_code(layer)
            bm.first_stroke = k
            bm.n_strokes = len(queue)
            self._keep.append((atlas, layer))
            for kind, payload in queue:
                if kind == "sphere":
                    r = payload
                    rows.append((LCL_STROKE_SPHERE, 0, r["cx"], r["cy"], r["cz"], 0, r["r2"], r["label"], r["flags"]))
                else:
                    cam, depth, poly, label, bias = payload[:5]
                    flags = payload[5] if len(payload) > 5 else 0
                    poly = np.ascontiguousarray(poly, dtype=np.float32)
                    bl = lcl_batch_lasso(cam, depth.data_ptr(), _addr(poly), poly.shape[0], int(label),
                                         float(bias), int(flags))
                    self._keep.append((depth, poly))
                    rows.append((LCL_STROKE_LASSO, len(lassos), 0, 0, 0, 0, 0, 0, 0))
                    lassos.append(bl)
                k += 1
        strokes = np.array(rows, dtype=BATCH_STROKE_DTYPE) if rows else np.zeros(1, BATCH_STROKE_DTYPE)
        self.n_models, self.n_strokes, self.n_lassos = len(models), n_total, len(lassos)
        self._strokes_np = strokes
        self.strokes = C.cast(_addr(strokes), C.POINTER(lcl_batch_stroke))
        self.lassos = (lcl_batch_lasso * max(len(lassos), 1))(*lassos)
        lib = library()
        own = lcl_batch_limits()
        _check("lcl_batch_limits_of", lib.lcl_batch_limits_of(self.models, self.n_models, self.n_strokes,
                                                               self.n_lassos, C.byref(own)))
        self.own_limits = own
        self.limits = own if limits is None else limits
        if not limits_fit(own, self.limits):
            raise ValueError("batch exceeds the given limits")
        self.config = config
        self.ws_bytes = int(lib.lcl_batch_workspace_bytes(C.byref(self.limits)))
        self.staging_bytes = int(lib.lcl_batch_staging_bytes(C.byref(self.limits)))
        dev = models[0][1].device if models else torch.device("cuda")
        if workspace is None or workspace.numel() < self.ws_bytes:
            workspace = torch.empty(max(self.ws_bytes, 256), dtype=torch.uint8, device=dev)
        if staging is None or staging.numel() < self.staging_bytes:
            staging = torch.empty(max(self.staging_bytes, 256), dtype=torch.uint8).pin_memory()
        self.workspace, self.staging = workspace, staging


def _torch_stream(stream):
    if stream is None:
        return torch.cuda.current_stream()
    if isinstance(stream, torch.cuda.Stream):
        return stream
    return torch.cuda.ExternalStream(int(stream))


def _cfg(config):
    return None if config is None else C.byref(config)


def _staging_wait(batch):
    """The staging is rewritten on the host by every upload, and the upload of the previous call that
    used it may still be queued on the device: wait (on the host) until that call has passed."""
    busy = getattr(batch.staging, "_lcl_busy", None)
    if busy is not None:
        busy.synchronize()


def _staging_mark(batch, stream):
    done = torch.cuda.Event()
    done.record(_torch_stream(stream))
    batch.staging._lcl_busy = done


def lcl_batch_upload(batch: Batch, stream=None):
    """Packs the batch's descriptors into its pinned staging and copies them to its workspace."""
    _staging_wait(batch)
    _check("lcl_batch_upload", library().lcl_batch_upload(
        C.byref(batch.limits), batch.models, batch.n_models, batch.strokes, batch.n_strokes, batch.lassos,
        batch.n_lassos, _ptr(batch.workspace), batch.workspace.numel(), C.c_void_p(batch.staging.data_ptr()),
        batch.staging.numel(), _stream(stream)))
    _staging_mark(batch, stream)
    return batch


def lcl_batch_launch(batch: Batch, stream=None, config=None):
    """Launches the batch last uploaded to the batch's workspace (config: this shape, else batch.config)."""
    cfg = config if config is not None else batch.config
    _check("lcl_batch_launch", library().lcl_batch_launch(C.byref(batch.limits), _cfg(cfg), _ptr(batch.workspace),
                                                          batch.workspace.numel(), _stream(stream)))
    return batch


def lcl_batch_edit(batch: Batch, stream=None):
    """Upload + launch (batch.config)."""
    _staging_wait(batch)
    _check("lcl_batch_edit", library().lcl_batch_edit(
        C.byref(batch.limits), _cfg(batch.config), batch.models, batch.n_models, batch.strokes, batch.n_strokes,
        batch.lassos, batch.n_lassos, _ptr(batch.workspace), batch.workspace.numel(),
        C.c_void_p(batch.staging.data_ptr()), batch.staging.numel(), _stream(stream)))
    _staging_mark(batch, stream)
    return batch


def lcl_batch_tune(batch: Batch, stream=None, reps=2):
    """Autotunes the launch shape on the batch last uploaded to the batch's workspace (its strokes are
    re-applied, which leaves the labels as they are); sets batch.config.  Returns (config, ms)."""
    best = lcl_batch_config()
    ms = C.c_float()
    _check("lcl_batch_tune", library().lcl_batch_tune(C.byref(batch.limits), _ptr(batch.workspace),
                                                      batch.workspace.numel(), int(reps), _stream(stream),
                                                      C.byref(best), C.byref(ms)))
    batch.config = best
    return best, float(ms.value)


class BatchGraph:
    """A CUDA graph holding one batched launch (lcl_batch_launch) on a workspace of given limits and
    launch shape.  The launch reads everything from the workspace, so after any batch within the
    limits has been uploaded there (lcl_batch_upload), replay() edits it."""

    def __init__(self, limits: lcl_batch_limits, config, workspace: torch.Tensor):
        self.limits, self.config, self.workspace = limits, config, workspace
        self.graph = torch.cuda.CUDAGraph()
        cur = torch.cuda.current_stream(workspace.device)
        side = torch.cuda.Stream(workspace.device)
        side.wait_stream(cur)
        with torch.cuda.stream(side):
            with torch.cuda.graph(self.graph, stream=side):
                _check("lcl_batch_launch", library().lcl_batch_launch(
                    C.byref(limits), _cfg(config), _ptr(workspace), workspace.numel(), _stream(side)))
        cur.wait_stream(side)

    def replay(self):
        self.graph.replay()


def lcl_overlay(atlas: Atlas, a: torch.Tensor, b: torch.Tensor, out: torch.Tensor, op, flags=0, stream=None):
    op = OPS[op] if isinstance(op, str) else int(op)
    _check("lcl_overlay", library().lcl_overlay(C.byref(atlas.c), _ptr(a), _ptr(b), _ptr(out), _dtype_code(a), op,
                                                int(flags), _stream(stream)))
    return out


def lcl_label_area(atlas: Atlas, layer: torch.Tensor, n_labels, count_out=None, area_out=None, stream=None):
    dev = layer.device
    count_out = torch.empty(n_labels, dtype=torch.int64, device=dev) if count_out is None else count_out
    area_out = torch.empty(n_labels, dtype=torch.int64, device=dev) if area_out is None else area_out
    _check("lcl_label_area", library().lcl_label_area(C.byref(atlas.c), _ptr(layer), _dtype_code(layer),
                                                      int(n_labels), _ptr(count_out), _ptr(area_out),
                                                      _stream(stream)))
    return count_out, area_out


# ---- numeric layers ------------------------------------------------------------------------

NUM_TYPES = {"u8": 0x11, "u16": 0x12, "u32": 0x14, "i8": 0x21, "i16": 0x22, "i32": 0x24, "f16": 0x32, "f32": 0x34}
NUM_TORCH = {"u8": torch.uint8, "u16": torch.int16, "u32": torch.int32, "i8": torch.int8, "i16": torch.int16,
             "i32": torch.int32, "f16": torch.float16, "f32": torch.float32}
ARITH = {"add": 0, "sub": 1, "mul": 2, "div": 3, "min": 4, "max": 5}
CMP = {"lt": 0, "le": 1, "gt": 2, "ge": 3, "eq": 4, "ne": 5}
LCL_ERASE = 0x100
ZONE_DTYPE = np.dtype([("count", "<u8"), ("area", "<u8"), ("vmin", "<f8"), ("vmax", "<f8"), ("sum", "<f8"),
                       ("wsum", "<f8")])


class NumericLayer:
    """A numeric layer on the device (Section 4.2): ``data`` (height x width values; u16 / u32 held in
    int16 / int32 tensors, bit for bit) and ``mask`` (one bit per texel, ceil(W*H/32) int32 words)."""

    def __init__(self, width, height, ntype, device="cuda", data=None, mask=None):
        self.width, self.height, self.ntype = int(width), int(height), ntype
        self.data = torch.zeros((height, width), dtype=NUM_TORCH[ntype], device=device) if data is None else data
        n_words = (width * height + 31) // 32
        self.mask = torch.zeros(((n_words + 3) // 4) * 4, dtype=torch.int32, device=device) if mask is None else mask
        self.c = lcl_numeric_layer(self.data.data_ptr(), self.mask.data_ptr(), NUM_TYPES[ntype], 0)

    def mask_bits(self):
        """The mask as a host bool array of the layer's shape."""
        w = self.mask.cpu().numpy().view(np.uint32)
        bits = np.unpackbits(w.view(np.uint8), bitorder="little")[: self.width * self.height]
        return bits.reshape(self.height, self.width).astype(bool)


def lcl_numeric_sphere(atlas: Atlas, layer: NumericLayer, strokes, hits_out=None, workspace=None, stream=None):
    """Sphere strokes on a numeric layer (the record's ``label`` field holds the value's bits; flags
    may add LCL_ERASE)."""
    recs = np.ascontiguousarray(strokes, dtype=SPHERE_DTYPE)
    n = len(recs)
    ws = workspace if workspace is not None else _workspace(lcl_select_workspace_bytes(atlas, n), layer.data.device)
    _check("lcl_numeric_sphere", library().lcl_numeric_sphere(
        C.byref(atlas.c), C.byref(layer.c), recs.ctypes.data_as(C.c_void_p), n, _ptr(hits_out), _ptr(ws), ws.numel(),
        _stream(stream)))
    return hits_out


def lcl_numeric_lasso(atlas: Atlas, layer: NumericLayer, cam: lcl_camera, depth: torch.Tensor, poly, value_bits,
                      flags=0, bias=DEFAULT_BIAS, hits_out=None, workspace=None, stream=None):
    poly = np.ascontiguousarray(poly, dtype=np.float32)
    ws = workspace if workspace is not None else _workspace(lcl_select_workspace_bytes(atlas, 1), layer.data.device)
    _check("lcl_numeric_lasso", library().lcl_numeric_lasso(
        C.byref(atlas.c), C.byref(layer.c), C.byref(cam), _ptr(depth), poly.ctypes.data_as(C.c_void_p), poly.shape[0],
        int(value_bits), int(flags), float(bias), _ptr(hits_out), _ptr(ws), ws.numel(), _stream(stream)))
    return hits_out


def lcl_numeric_tool(atlas: Atlas, layer: NumericLayer, cam: lcl_camera, depth: torch.Tensor, tool: lcl_tool,
                     value_bits, flags=0, bias=DEFAULT_BIAS, hits_out=None, workspace=None, stream=None):
    ws = workspace if workspace is not None else _workspace(lcl_select_workspace_bytes(atlas, 1), layer.data.device)
    _check("lcl_numeric_tool", library().lcl_numeric_tool(
        C.byref(atlas.c), C.byref(layer.c), C.byref(cam), _ptr(depth), C.byref(tool), int(value_bits), int(flags),
        float(bias), _ptr(hits_out), _ptr(ws), ws.numel(), _stream(stream)))
    return hits_out


def lcl_numeric_arith(atlas: Atlas, a: NumericLayer, b, out: NumericLayer, op, b_value_bits=0, stream=None):
    """out = a <op> b (b a NumericLayer, or None for the scalar b_value_bits)."""
    op = ARITH[op] if isinstance(op, str) else int(op)
    _check("lcl_numeric_arith", library().lcl_numeric_arith(
        C.byref(atlas.c), C.byref(a.c), None if b is None else C.byref(b.c), int(b_value_bits), C.byref(out.c), op,
        _stream(stream)))
    return out


def lcl_numeric_select(atlas: Atlas, values: NumericLayer, cmp, threshold_bits, layer: torch.Tensor, label,
                       hits_out=None, stream=None):
    cmp = CMP[cmp] if isinstance(cmp, str) else int(cmp)
    _check("lcl_numeric_select", library().lcl_numeric_select(
        C.byref(atlas.c), C.byref(values.c), cmp, int(threshold_bits), _ptr(layer), _dtype_code(layer), int(label),
        _ptr(hits_out), _stream(stream)))
    return hits_out


def lcl_numeric_stats(atlas: Atlas, values: NumericLayer, zones, n_labels, out=None, stream=None):
    """Zonal statistics; ``out``: device uint8 tensor of n_labels * 48 bytes (allocated if None)."""
    dev = values.data.device
    out = torch.empty(n_labels * 48, dtype=torch.uint8, device=dev) if out is None else out
    zcode = 0 if zones is None else _dtype_code(zones)
    _check("lcl_numeric_stats", library().lcl_numeric_stats(
        C.byref(atlas.c), C.byref(values.c), _ptr(zones), zcode, int(n_labels), _ptr(out), _stream(stream)))
    return out


def zone_stats_host(out: torch.Tensor):
    """Device zone records -> numpy structured array (count, area, vmin, vmax, sum, wsum)."""
    return out.cpu().numpy().view(ZONE_DTYPE)


# ---- sparse layer pool -------------------------------------------------------------------

_POOL_TYPES = {"u8": (LCL_U8, torch.uint8), "u16": (LCL_U16, torch.int16)}


class _DeviceArray:
    """__cuda_array_interface__ of a pool layer's memory, so torch can view it without copying."""

    def __init__(self, ptr, shape, typestr):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr, "data": (int(ptr), False),
                                         "version": 3, "strides": None}


_TYPESTR = {torch.uint8: "|u1", torch.int8: "|i1", torch.int16: "<i2", torch.int32: "<i4", torch.float16: "<f2",
            torch.float32: "<f4"}


class PoolLayer:
    """A layer committed by a Pool: ``data`` (and, for numeric types, ``mask``) are torch views of the
    pool's memory; ``numeric`` is the NumericLayer over them (numeric types only)."""

    def __init__(self, pool, rec: lcl_pool_layer, kind, device):
        self.pool, self.rec, self.kind = pool, rec, kind
        self.handle = int(rec.handle)
        W, H = rec.width, rec.height
        dt = _POOL_TYPES[kind][1] if kind in _POOL_TYPES else NUM_TORCH[kind]
        self.data = torch.as_tensor(_DeviceArray(rec.data, (H, W), _TYPESTR[dt]), device=device)
        self.mask = None
        self.numeric = None
        if rec.mask:
            n_words = (W * H + 31) // 32
            self.mask = torch.as_tensor(_DeviceArray(rec.mask, (n_words,), "<i4"), device=device)
            self.numeric = NumericLayer(W, H, kind, device, data=self.data, mask=self.mask)


class Pool:
    """The sparse layer pool (lcl_pool_*): layers of one (width, height, type) share one reserved
    address range; memory is committed per acquired layer and returned on release."""

    def __init__(self, max_layers_per_array=256, device=None):
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        self.ptr = C.c_void_p()
        with torch.cuda.device(self.device):
            _check("lcl_pool_create", library().lcl_pool_create(int(max_layers_per_array), C.byref(self.ptr)))

    def acquire(self, width, height, kind="u8", stream=None) -> PoolLayer:
        code = _POOL_TYPES[kind][0] if kind in _POOL_TYPES else NUM_TYPES[kind]
        rec = lcl_pool_layer()
        _check("lcl_pool_acquire", library().lcl_pool_acquire(self.ptr, int(width), int(height), code,
                                                              _stream(stream), C.byref(rec)))
        return PoolLayer(self, rec, kind, self.device)

    def release(self, layer: PoolLayer, stream=None):
        _check("lcl_pool_release", library().lcl_pool_release(self.ptr, layer.handle, _stream(stream)))
        layer.data = layer.mask = layer.numeric = None

    def stats(self):
        st = lcl_pool_stats()
        _check("lcl_pool_stats_get", library().lcl_pool_stats_get(self.ptr, C.byref(st)))
        return {"reserved_bytes": st.reserved_bytes, "committed_bytes": st.committed_bytes, "layers": st.layers,
                "arrays": st.arrays, "granularity": st.granularity}

    def destroy(self):
        if self.ptr:
            _check("lcl_pool_destroy", library().lcl_pool_destroy(self.ptr))
            self.ptr = C.c_void_p()


def lcl_status_str(status):
    return library().lcl_status_str(int(status)).decode()


def lcl_last_error():
    return library().lcl_last_error().decode()


def lcl_kernel_launches():
    return int(library().lcl_kernel_launches())


def lcl_last_device_status(stream=None):
    """Synchronises `stream` (default: the current torch stream) and returns the library's device
    status (an lcl_status code; lcl_last_error() explains a non-zero one).  Raises nothing."""
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    elif isinstance(stream, torch.cuda.Stream):
        stream = stream.cuda_stream
    return int(library().lcl_last_device_status(C.c_void_p(stream)))


def lcl_build_flags():
    return int(library().lcl_build_flags())


def lcl_describe_site(site):
    buf = C.create_string_buffer(64)
    library().lcl_describe_site(C.c_uint32(site), buf, 64)
    return buf.value.decode()


def lcl_check_division(n, seed=1, stream=None, device="cuda"):
    """Runs the library's division self-check on n operand pairs; returns (compared, mismatches)."""
    counts = torch.zeros(2, dtype=torch.int64, device=device)
    _check("lcl_check_division", library().lcl_check_division(C.c_uint64(int(n)), C.c_uint32(int(seed)),
                                                              _ptr(counts), _stream(stream)))
    c = counts.cpu().numpy().view(np.uint64)
    return int(c[0]), int(c[1])
