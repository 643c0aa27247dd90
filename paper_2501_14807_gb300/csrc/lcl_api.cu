// lcl_api.cu -- the extern "C" entry points declared in include/lcl.h: argument checks on
// the host, buffer layout, host-side helpers (stroke quantisation, camera composition),
// and dispatch to the launchers of the other translation units.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "lcl_impl.cuh"

namespace lcl {

namespace {
thread_local std::string g_last_error;
std::atomic<uint64_t> g_launches{0};
int g_sm_count[64] = {0};
}  // namespace

lcl_status fail(lcl_status s, const std::string &why) {
    g_last_error = why;
    return s;
}

lcl_status cuda_fail(cudaError_t e, const char *where) {
    g_last_error = std::string(where) + ": " + cudaGetErrorString(e);
    return LCL_ERR_CUDA;
}

int sm_count() {
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    if (g_sm_count[dev] == 0) {
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 1;
        g_sm_count[dev] = n;
    }
    return g_sm_count[dev];
}

void count_launches(int n) { g_launches.fetch_add((uint64_t)n, std::memory_order_relaxed); }

// Readers of the bounds-check records, one per module of the debug build (empty otherwise).
namespace {
std::vector<BoundsReader> &bounds_readers() {
    static std::vector<BoundsReader> r;
    return r;
}
std::mutex &bounds_mu() {
    static std::mutex m;
    return m;
}

// Source files whose checks can report, for decoding a site's file hash.
const char *const kSourceNames[] = {"atlas.cu", "batch.cu", "depth.cu", "layers.cu", "numeric.cu", "select.cu",
                                    "noalloc.cu", "lcl_api.cu", "pool.cu", "select_common.cuh", "lcl_impl.cuh"};
}  // namespace

void register_bounds_reader(BoundsReader reader) {
    std::lock_guard<std::mutex> lock(bounds_mu());
    bounds_readers().push_back(reader);
}


namespace {

bool tile_ok(int32_t t) { return t == 8 || t == 16 || t == 32 || t == 64 || t == 128; }

bool dims_ok(int32_t w, int32_t h, int32_t tile) {
    return w >= 4 && w <= 16384 && (w % 4) == 0 && h >= 1 && h <= 16384 && tile_ok(tile);
}

struct Layout {
    size_t px, py, pz, tri, cover, tile_box, super_box, area_w, total;
    int32_t tiles_x, tiles_y, supers_x, supers_y;
};

Layout layout(int32_t w, int32_t h, int32_t tile, int64_t n_tri) {
    Layout L;
    const size_t plane = align256((size_t)w * h * 4);
    L.tiles_x = (w + tile - 1) / tile;
    L.tiles_y = (h + tile - 1) / tile;
    L.supers_x = (L.tiles_x + LCL_SUPER - 1) / LCL_SUPER;
    L.supers_y = (L.tiles_y + LCL_SUPER - 1) / LCL_SUPER;
    L.px = 0;
    L.py = L.px + plane;
    L.pz = L.py + plane;
    L.tri = L.pz + plane;
    L.cover = L.tri + plane;
    L.tile_box = L.cover + align256((((size_t)w * h + 31) / 32) * 4);
    L.super_box = L.tile_box + align256((size_t)L.tiles_x * L.tiles_y * 32);
    L.area_w = L.super_box + align256((size_t)L.supers_x * L.supers_y * 32);
    L.total = L.area_w + align256((size_t)std::max<int64_t>(n_tri, 1) * 8);
    return L;
}

bool aligned(const void *p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

// A band (or a view) holds only some rows of its texture: texture padding, which reads texels up
// to 8 rows away, is not available on it.
bool partial_rows(const lcl_atlas *a) { return a->tex_height > 0 && a->height != a->tex_height; }

lcl_status check_padding_rows(const lcl_atlas *a, uint32_t pad_flags) {
    if ((pad_flags & 15u) && partial_rows(a))
        return fail(LCL_ERR_UNSUPPORTED, "texture padding needs the whole texture, not a band of its rows");
    return LCL_OK;
}

lcl_status check_atlas(const lcl_atlas *a, bool need_boxes) {
    if (!a) return fail(LCL_ERR_INVALID_ARG, "atlas is NULL");
    if (!dims_ok(a->width, a->height, a->tile)) return fail(LCL_ERR_INVALID_ARG, "atlas sizes out of range");
    const int32_t th = a->tex_height > 0 ? a->tex_height : a->height;
    if (a->row0 < 0 || th > 16384 || (int64_t)a->row0 + a->height > th)
        return fail(LCL_ERR_INVALID_ARG, "atlas rows lie outside its texture");
    if (!a->pos_x || !a->pos_y || !a->pos_z || !a->tri || !a->cover || !a->area_w)
        return fail(LCL_ERR_INVALID_ARG, "atlas is not bound");
    if (need_boxes && (!a->tile_box || !a->super_box))
        return fail(LCL_ERR_INVALID_ARG, "selections need a whole atlas, not a row view");
    return LCL_OK;
}

lcl_status check_mesh(const lcl_mesh *m) {
    if (!m) return fail(LCL_ERR_INVALID_ARG, "mesh is NULL");
    if (m->n_pos < 1 || m->n_uv < 1 || m->n_tri < 0 || m->n_tri > (int64_t)0xFFFFFFFEu)
        return fail(LCL_ERR_INVALID_ARG, "mesh sizes out of range");
    if (!m->pos || !m->uv || (m->n_tri > 0 && (!m->tri_pos || !m->tri_uv)))
        return fail(LCL_ERR_INVALID_ARG, "mesh pointer is NULL");
    if (!aligned(m->pos, 4) || !aligned(m->uv, 4) || !aligned(m->tri_pos, 4) || !aligned(m->tri_uv, 4))
        return fail(LCL_ERR_INVALID_ARG, "mesh arrays must be 4-byte aligned");
    return LCL_OK;
}

int dtype_bytes(lcl_dtype d) { return d == LCL_U8 ? 1 : d == LCL_U16 ? 2 : 0; }

bool num_type_ok(int t) {
    switch (t) {
    case LCL_NUM_U8: case LCL_NUM_U16: case LCL_NUM_U32: case LCL_NUM_I8: case LCL_NUM_I16: case LCL_NUM_I32:
    case LCL_NUM_F16: case LCL_NUM_F32: return true;
    default: return false;
    }
}

uint32_t value_mask(int t) { return (t & 15) == 4 ? 0xFFFFFFFFu : ((1u << (8 * (t & 15))) - 1u); }

lcl_status check_numeric(const lcl_numeric_layer *l, const char *what) {
    if (!l) return fail(LCL_ERR_INVALID_ARG, std::string(what) + " is NULL");
    if (!num_type_ok((int)l->type)) return fail(LCL_ERR_INVALID_ARG, std::string(what) + ": unknown numeric type");
    if (!l->data || !aligned(l->data, 16) || !l->mask || !aligned(l->mask, 16))
        return fail(LCL_ERR_INVALID_ARG, std::string(what) + ": data and mask must be 16-byte aligned device pointers");
    return LCL_OK;
}

lcl_status check_tool(const lcl_tool *tool) {
    if (!tool) return fail(LCL_ERR_INVALID_ARG, "tool is NULL");
    if (!std::isfinite(tool->px) || !std::isfinite(tool->py) || !std::isfinite(tool->tw) || !std::isfinite(tool->th) ||
        !(tool->tw > 0.0f) || !(tool->th > 0.0f) || std::fabs(tool->px) > 1e7f || std::fabs(tool->py) > 1e7f ||
        tool->tw > 1e7f || tool->th > 1e7f)
        return fail(LCL_ERR_INVALID_ARG, "tool window must be finite, positive and below 1e7 px");
    if (tool->shape && (tool->shape_w < 1 || tool->shape_w > 4096 || tool->shape_h < 1 || tool->shape_h > 4096))
        return fail(LCL_ERR_INVALID_ARG, "tool shape sizes must be 1..4096");
    if ((tool->flags & ~0xFFu) || (tool->flags & 15u) > 8 || ((tool->flags >> 4) & 15u) > 8)
        return fail(LCL_ERR_INVALID_ARG, "tool padding radius and thickness must be <= 8, other flag bits 0");
    return LCL_OK;
}

lcl_status check_camera(const lcl_camera *c) {
    if (!c) return fail(LCL_ERR_INVALID_ARG, "camera is NULL");
    if (c->width < 1 || c->width > 16384 || c->height < 1 || c->height > 16384)
        return fail(LCL_ERR_INVALID_ARG, "camera size out of range");
    for (int i = 0; i < 16; ++i)
        if (!std::isfinite(c->m[i])) return fail(LCL_ERR_INVALID_ARG, "camera matrix is not finite");
    return LCL_OK;
}

}  // namespace
}  // namespace lcl

using namespace lcl;

extern "C" {

size_t lcl_atlas_bytes(int32_t width, int32_t height, int32_t tile, int64_t n_tri) {
    if (!dims_ok(width, height, tile) || n_tri < 0) return 0;
    return layout(width, height, tile, n_tri).total;
}

lcl_status lcl_atlas_bind(void *base, size_t bytes, int32_t width, int32_t height, int32_t tile, int64_t n_tri,
                          lcl_atlas *out) {
    if (!out || !base) return fail(LCL_ERR_INVALID_ARG, "NULL argument");
    if (!dims_ok(width, height, tile) || n_tri < 0 || n_tri > (int64_t)0xFFFFFFFEu)
        return fail(LCL_ERR_INVALID_ARG, "atlas sizes out of range");
    if (!aligned(base, 256)) return fail(LCL_ERR_INVALID_ARG, "atlas buffer must be 256-byte aligned");
    const Layout L = layout(width, height, tile, n_tri);
    if (bytes < L.total) return fail(LCL_ERR_OUT_OF_MEMORY, "atlas buffer smaller than lcl_atlas_bytes");
    char *b = static_cast<char *>(base);
    std::memset(out, 0, sizeof(*out));
    out->width = width;
    out->height = height;
    out->tile = tile;
    out->tiles_x = L.tiles_x;
    out->tiles_y = L.tiles_y;
    out->supers_x = L.supers_x;
    out->supers_y = L.supers_y;
    out->row0 = 0;
    out->tex_height = height;
    out->n_tri = n_tri;
    out->pos_x = reinterpret_cast<int32_t *>(b + L.px);
    out->pos_y = reinterpret_cast<int32_t *>(b + L.py);
    out->pos_z = reinterpret_cast<int32_t *>(b + L.pz);
    out->tri = reinterpret_cast<uint32_t *>(b + L.tri);
    out->cover = reinterpret_cast<uint32_t *>(b + L.cover);
    out->tile_box = reinterpret_cast<int32_t *>(b + L.tile_box);
    out->super_box = reinterpret_cast<int32_t *>(b + L.super_box);
    out->area_w = reinterpret_cast<uint64_t *>(b + L.area_w);
    out->scale = 0.0;
    return LCL_OK;
}

lcl_status lcl_atlas_bind_band(void *base, size_t bytes, int32_t width, int32_t tex_height, int32_t y0, int32_t y1,
                               int32_t tile, int64_t n_tri, lcl_atlas *out) {
    if (tex_height < 1 || tex_height > 16384 || y0 < 0 || y1 > tex_height || y0 >= y1)
        return fail(LCL_ERR_INVALID_ARG, "band rows out of range");
    const lcl_status s = lcl_atlas_bind(base, bytes, width, y1 - y0, tile, n_tri, out);
    if (s != LCL_OK) return s;
    out->row0 = y0;
    out->tex_height = tex_height;
    return LCL_OK;
}

lcl_status lcl_atlas_rows(const lcl_atlas *atlas, int32_t y0, int32_t y1, lcl_atlas *out) {
    lcl_status s = check_atlas(atlas, false);
    if (s != LCL_OK) return s;
    if (!out) return fail(LCL_ERR_INVALID_ARG, "out is NULL");
    if (y0 < 0 || y1 > atlas->height || y0 >= y1) return fail(LCL_ERR_INVALID_ARG, "row range out of bounds");
    if (((int64_t)y0 * atlas->width) % 32 != 0) return fail(LCL_ERR_INVALID_ARG, "y0 * width must be a multiple of 32");
    lcl_atlas v = *atlas;
    const int64_t off = (int64_t)y0 * atlas->width;
    v.height = y1 - y0;
    v.row0 = atlas->row0 + y0;
    v.tiles_y = (v.height + v.tile - 1) / v.tile;
    v.supers_y = (v.tiles_y + LCL_SUPER - 1) / LCL_SUPER;
    v.pos_x += off;
    v.pos_y += off;
    v.pos_z += off;
    v.tri += off;
    v.cover += off / 32;
    v.tile_box = nullptr;
    v.super_box = nullptr;
    *out = v;
    return LCL_OK;
}

size_t lcl_atlas_workspace_bytes(const lcl_mesh *mesh, int32_t width, int32_t height) {
    if (!mesh || mesh->n_pos < 0 || mesh->n_uv < 0 || mesh->n_tri < 0) return 0;
    return atlas_ws_bytes(mesh->n_pos, mesh->n_uv, mesh->n_tri, width, height);
}

lcl_status lcl_atlas_build(const lcl_mesh *mesh, lcl_atlas *atlas, void *workspace, size_t ws_bytes,
                           lcl_stream stream) {
    lcl_status s = check_mesh(mesh);
    if (s != LCL_OK) return s;
    s = check_atlas(atlas, true);
    if (s != LCL_OK) return s;
    if (mesh->n_tri != atlas->n_tri) return fail(LCL_ERR_INVALID_ARG, "atlas was bound for another triangle count");
    if (!workspace || !aligned(workspace, 256)) return fail(LCL_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
    return atlas_build_impl(mesh, atlas, workspace, ws_bytes, reinterpret_cast<cudaStream_t>(stream));
}

lcl_status lcl_quantize_sphere(const lcl_atlas *atlas, const double centre[3], double radius, uint32_t label,
                               lcl_sphere *out) {
    if (!atlas || !centre || !out) return fail(LCL_ERR_INVALID_ARG, "NULL argument");
    if (!(atlas->scale > 0.0)) return fail(LCL_ERR_INVALID_ARG, "atlas has not been built");
    if (!(radius >= 0.0) || !std::isfinite(radius)) return fail(LCL_ERR_INVALID_ARG, "radius must be finite and >= 0");
    int32_t q[3];
    for (int a = 0; a < 3; ++a) {
        if (!std::isfinite(centre[a])) return fail(LCL_ERR_INVALID_ARG, "centre is not finite");
        volatile double d = centre[a] - (double)atlas->bbox_min[a];
        volatile double t = d * atlas->scale;
        volatile double u = t + 0.5;
        const double f = std::floor(u);
        if (f < -(double)(1 << 22) || f > (double)((1 << 22) + (1 << 21)))
            return fail(LCL_ERR_INVALID_ARG, "centre lies too far outside the model's grid");
        q[a] = (int32_t)f;
    }
    volatile double rs = radius * atlas->scale;
    volatile double rs2 = rs * rs;
    const double fl = std::floor(rs2);
    out->cx = q[0];
    out->cy = q[1];
    out->cz = q[2];
    out->_pad = 0;
    out->r2 = fl >= (double)kR2Cap ? kR2Cap : (int64_t)fl;
    out->label = label;
    out->flags = 0;
    return LCL_OK;
}

lcl_status lcl_quantize_spheres(const lcl_atlas *atlas, int32_t n, const double *centres, const double *radii,
                                const uint32_t *labels, lcl_sphere *out) {
    if (n < 0 || (n > 0 && (!centres || !radii || !labels || !out))) return fail(LCL_ERR_INVALID_ARG, "NULL argument");
    for (int32_t k = 0; k < n; ++k) {
        const lcl_status s = lcl_quantize_sphere(atlas, centres + 3 * (int64_t)k, radii[k], labels[k], out + k);
        if (s != LCL_OK) return s;
    }
    return LCL_OK;
}

lcl_status lcl_camera_from_vp(const lcl_atlas *atlas, const double vp[16], int32_t width, int32_t height,
                              lcl_camera *out) {
    if (!atlas || !vp || !out) return fail(LCL_ERR_INVALID_ARG, "NULL argument");
    if (!(atlas->scale > 0.0)) return fail(LCL_ERR_INVALID_ARG, "atlas has not been built");
    if (width < 1 || width > 16384 || height < 1 || height > 16384)
        return fail(LCL_ERR_INVALID_ARG, "camera size out of range");
    for (int i = 0; i < 4; ++i) {
        for (int j = 0; j < 3; ++j) {
            volatile double v = vp[4 * i + j] / atlas->scale;
            out->m[4 * i + j] = (float)v;
        }
        volatile double p0 = vp[4 * i + 0] * (double)atlas->bbox_min[0];
        volatile double p1 = vp[4 * i + 1] * (double)atlas->bbox_min[1];
        volatile double p2 = vp[4 * i + 2] * (double)atlas->bbox_min[2];
        volatile double s01 = p0 + p1;
        volatile double s012 = s01 + p2;
        volatile double t = s012 + vp[4 * i + 3];
        out->m[4 * i + 3] = (float)t;
    }
    out->width = width;
    out->height = height;
    for (int i = 0; i < 16; ++i)
        if (!std::isfinite(out->m[i])) return fail(LCL_ERR_INVALID_ARG, "camera matrix is not finite");
    return LCL_OK;
}

size_t lcl_select_workspace_bytes(const lcl_atlas *atlas, int32_t n_strokes) {
    if (!atlas || n_strokes < 0 || atlas->tiles_x <= 0 || atlas->tiles_y <= 0) return 0;
    return select_ws_bytes(atlas, std::max(n_strokes, 1));
}

}  // extern "C"

namespace lcl {

// Every check of lcl_select_sphere except those of the workspace (shared with the entry point
// that brings its own scratch).  *proceed is false when there is nothing to do (n == 0).
lcl_status check_sphere_call(const lcl_atlas *atlas, const void *layer, lcl_dtype dtype, const lcl_sphere *strokes,
                             int32_t n, const uint64_t *hits_out, bool *proceed) {
    *proceed = false;
    lcl_status s = check_atlas(atlas, true);
    if (s != LCL_OK) return s;
    const int db = dtype_bytes(dtype);
    if (!db) return fail(LCL_ERR_INVALID_ARG, "dtype must be LCL_U8 or LCL_U16");
    if (!layer || !aligned(layer, 16)) return fail(LCL_ERR_INVALID_ARG, "layer must be a 16-byte aligned device pointer");
    if (n < 0 || n > (1 << 24)) return fail(LCL_ERR_INVALID_ARG, "stroke count out of range");
    if (n == 0) return LCL_OK;
    if (!strokes) return fail(LCL_ERR_INVALID_ARG, "strokes is NULL");
    if (hits_out && !aligned(hits_out, 8)) return fail(LCL_ERR_INVALID_ARG, "hits_out must be 8-byte aligned");
    const uint32_t lab_max = db == 1 ? 0xFFu : 0xFFFFu;
    for (int32_t k = 0; k < n; ++k) {
        const lcl_sphere &st = strokes[k];
        if (st.r2 < 0) return fail(LCL_ERR_INVALID_ARG, "stroke r2 < 0");
        if (st.label > lab_max) return fail(LCL_ERR_INVALID_ARG, "stroke label does not fit the layer dtype");
        if ((st.flags & ~0xFFu) || (st.flags & 15u) > 8 || ((st.flags >> 4) & 15u) > 8)
            return fail(LCL_ERR_INVALID_ARG, "stroke flags: padding radius and thickness at most 8, other bits 0");
        const int32_t lo = -(1 << 22), hi = (1 << 22) + (1 << 21);
        if (st.cx < lo || st.cx > hi || st.cy < lo || st.cy > hi || st.cz < lo || st.cz > hi)
            return fail(LCL_ERR_INVALID_ARG, "stroke centre outside [-2^22, 2^22 + 2^21]");
        if ((s = check_padding_rows(atlas, st.flags)) != LCL_OK) return s;
    }
    *proceed = true;
    return LCL_OK;
}

}  // namespace lcl

extern "C" {

lcl_status lcl_select_sphere(const lcl_atlas *atlas, void *layer, lcl_dtype dtype, const lcl_sphere *strokes,
                             int32_t n, uint64_t *hits_out, void *workspace, size_t ws_bytes, lcl_stream stream) {
    bool proceed = false;
    lcl_status s = check_sphere_call(atlas, layer, dtype, strokes, n, hits_out, &proceed);
    if (s != LCL_OK || !proceed) return s;
    if (!workspace || !aligned(workspace, 256)) return fail(LCL_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
    if (ws_bytes < select_ws_bytes(atlas, n)) return fail(LCL_ERR_OUT_OF_MEMORY, "workspace smaller than lcl_select_workspace_bytes");
    return select_sphere_impl(atlas, layer, dtype_bytes(dtype), strokes, n, hits_out, workspace,
                              reinterpret_cast<cudaStream_t>(stream));
}

size_t lcl_depth_workspace_bytes(const lcl_mesh *mesh, int32_t width, int32_t height) {
    if (!mesh || mesh->n_tri < 0 || mesh->n_pos < 0) return 0;
    return depth_ws_bytes(mesh->n_pos, mesh->n_tri, width, height);
}

lcl_status lcl_depth_render(const lcl_mesh *mesh, const lcl_atlas *atlas, const lcl_camera *camera, float *depth,
                            void *workspace, size_t ws_bytes, lcl_stream stream) {
    lcl_status s = check_mesh(mesh);
    if (s != LCL_OK) return s;
    if (!atlas || !(atlas->scale > 0.0)) return fail(LCL_ERR_INVALID_ARG, "atlas has not been built");
    s = check_camera(camera);
    if (s != LCL_OK) return s;
    if (!depth || !aligned(depth, 4)) return fail(LCL_ERR_INVALID_ARG, "depth must be a 4-byte aligned device pointer");
    if (!workspace || !aligned(workspace, 256)) return fail(LCL_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
    return depth_render_impl(mesh, atlas, camera, depth, workspace, ws_bytes, reinterpret_cast<cudaStream_t>(stream));
}

lcl_status lcl_select_lasso(const lcl_atlas *atlas, void *layer, lcl_dtype dtype, const lcl_camera *camera,
                            const float *depth, const float *poly_xy, int32_t n_vertices, uint32_t label,
                            uint32_t flags, float bias, uint64_t *hits_out, void *workspace, size_t ws_bytes,
                            lcl_stream stream) {
    lcl_status s = check_atlas(atlas, true);
    if (s != LCL_OK) return s;
    const int db = dtype_bytes(dtype);
    if (!db) return fail(LCL_ERR_INVALID_ARG, "dtype must be LCL_U8 or LCL_U16");
    if (!layer || !aligned(layer, 16)) return fail(LCL_ERR_INVALID_ARG, "layer must be a 16-byte aligned device pointer");
    s = check_camera(camera);
    if (s != LCL_OK) return s;
    if (!depth || !aligned(depth, 4)) return fail(LCL_ERR_INVALID_ARG, "depth must be a 4-byte aligned device pointer");
    if (!poly_xy) return fail(LCL_ERR_INVALID_ARG, "polygon is NULL");
    if (n_vertices < 3 || n_vertices > LCL_MAX_LASSO_VERTICES)
        return fail(LCL_ERR_UNSUPPORTED, "lasso polygons need 3..64 vertices");
    for (int i = 0; i < 2 * n_vertices; ++i)
        if (!std::isfinite(poly_xy[i])) return fail(LCL_ERR_INVALID_ARG, "polygon vertex is not finite");
    if (label > (db == 1 ? 0xFFu : 0xFFFFu)) return fail(LCL_ERR_INVALID_ARG, "label does not fit the layer dtype");
    if ((flags & ~0xFFu) || (flags & 15u) > 8 || ((flags >> 4) & 15u) > 8)
        return fail(LCL_ERR_INVALID_ARG, "lasso flags: padding radius and thickness at most 8, other bits 0");
    if ((s = check_padding_rows(atlas, flags)) != LCL_OK) return s;
    if (!std::isfinite(bias)) return fail(LCL_ERR_INVALID_ARG, "bias is not finite");
    if (hits_out && !aligned(hits_out, 8)) return fail(LCL_ERR_INVALID_ARG, "hits_out must be 8-byte aligned");
    if (!workspace || !aligned(workspace, 256)) return fail(LCL_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
    if (ws_bytes < select_ws_bytes(atlas, 1)) return fail(LCL_ERR_OUT_OF_MEMORY, "workspace smaller than lcl_select_workspace_bytes");
    return select_lasso_impl(atlas, layer, db, camera, depth, poly_xy, n_vertices, label, flags, bias, hits_out,
                             workspace, reinterpret_cast<cudaStream_t>(stream));
}

lcl_status lcl_select_tool(const lcl_atlas *atlas, void *layer, lcl_dtype dtype, const lcl_camera *camera,
                           const float *depth, const lcl_tool *tool, uint32_t label, float bias, uint64_t *hits_out,
                           void *workspace, size_t ws_bytes, lcl_stream stream) {
    lcl_status s = check_atlas(atlas, true);
    if (s != LCL_OK) return s;
    const int db = dtype_bytes(dtype);
    if (!db) return fail(LCL_ERR_INVALID_ARG, "dtype must be LCL_U8 or LCL_U16");
    if (!layer || !aligned(layer, 16)) return fail(LCL_ERR_INVALID_ARG, "layer must be a 16-byte aligned device pointer");
    s = check_camera(camera);
    if (s != LCL_OK) return s;
    if (!depth || !aligned(depth, 4)) return fail(LCL_ERR_INVALID_ARG, "depth must be a 4-byte aligned device pointer");
    s = check_tool(tool);
    if (s != LCL_OK) return s;
    if ((s = check_padding_rows(atlas, tool->flags)) != LCL_OK) return s;
    if (label > (db == 1 ? 0xFFu : 0xFFFFu)) return fail(LCL_ERR_INVALID_ARG, "label does not fit the layer dtype");
    if (!std::isfinite(bias)) return fail(LCL_ERR_INVALID_ARG, "bias is not finite");
    if (hits_out && !aligned(hits_out, 8)) return fail(LCL_ERR_INVALID_ARG, "hits_out must be 8-byte aligned");
    if (!workspace || !aligned(workspace, 256)) return fail(LCL_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
    if (ws_bytes < select_ws_bytes(atlas, 1)) return fail(LCL_ERR_OUT_OF_MEMORY, "workspace smaller than lcl_select_workspace_bytes");
    return select_tool_impl(atlas, layer, db, camera, depth, tool, label, bias, hits_out, workspace,
                            reinterpret_cast<cudaStream_t>(stream));
}

lcl_status lcl_batch_limits_of(const lcl_batch_model *models, int32_t n_models, int32_t n_strokes, int32_t n_lassos,
                               lcl_batch_limits *out) {
    return batch_limits_of(models, n_models, n_strokes, n_lassos, out);
}

size_t lcl_batch_workspace_bytes(const lcl_batch_limits *limits) { return batch_ws_bytes(limits); }

size_t lcl_batch_staging_bytes(const lcl_batch_limits *limits) { return batch_host_bytes(limits); }

lcl_status lcl_batch_upload(const lcl_batch_limits *limits, const lcl_batch_model *models, int32_t n_models,
                            const lcl_batch_stroke *strokes, int32_t n_strokes, const lcl_batch_lasso *lassos,
                            int32_t n_lassos, void *workspace, size_t ws_bytes, void *host_staging,
                            size_t staging_bytes, lcl_stream stream) {
    if (!workspace || !aligned(workspace, 256)) return fail(LCL_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
    if (!host_staging || !aligned(host_staging, 16)) return fail(LCL_ERR_INVALID_ARG, "host staging must be 16-byte aligned");
    return batch_upload_impl(limits, models, n_models, strokes, n_strokes, lassos, n_lassos, workspace, ws_bytes,
                             host_staging, staging_bytes, reinterpret_cast<cudaStream_t>(stream));
}

lcl_status lcl_batch_launch(const lcl_batch_limits *limits, const lcl_batch_config *config, void *workspace,
                            size_t ws_bytes, lcl_stream stream) {
    if (!workspace || !aligned(workspace, 256)) return fail(LCL_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
    return batch_launch_impl(limits, config, workspace, ws_bytes, reinterpret_cast<cudaStream_t>(stream));
}

lcl_status lcl_batch_edit(const lcl_batch_limits *limits, const lcl_batch_config *config,
                          const lcl_batch_model *models, int32_t n_models, const lcl_batch_stroke *strokes,
                          int32_t n_strokes, const lcl_batch_lasso *lassos, int32_t n_lassos, void *workspace,
                          size_t ws_bytes, void *host_staging, size_t staging_bytes, lcl_stream stream) {
    lcl_status s = lcl_batch_upload(limits, models, n_models, strokes, n_strokes, lassos, n_lassos, workspace,
                                    ws_bytes, host_staging, staging_bytes, stream);
    if (s != LCL_OK) return s;
    return lcl_batch_launch(limits, config, workspace, ws_bytes, stream);
}

lcl_status lcl_batch_tune(const lcl_batch_limits *limits, void *workspace, size_t ws_bytes, int32_t reps,
                          lcl_stream stream, lcl_batch_config *best, float *best_ms) {
    if (!workspace || !aligned(workspace, 256)) return fail(LCL_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
    return batch_tune_impl(limits, workspace, ws_bytes, reps, reinterpret_cast<cudaStream_t>(stream), best, best_ms);
}

lcl_status lcl_overlay(const lcl_atlas *atlas, const void *a, const void *b, void *out, lcl_dtype dtype, lcl_op op,
                       uint32_t flags, lcl_stream stream) {
    lcl_status s = check_atlas(atlas, false);
    if (s != LCL_OK) return s;
    const int db = dtype_bytes(dtype);
    if (!db) return fail(LCL_ERR_INVALID_ARG, "dtype must be LCL_U8 or LCL_U16");
    if ((int)op < 0 || (int)op > 3) return fail(LCL_ERR_INVALID_ARG, "unknown overlay op");
    if (flags & ~7u) return fail(LCL_ERR_INVALID_ARG, "unknown overlay flags");
    if (!a || !b || !out || !aligned(a, 16) || !aligned(b, 16) || !aligned(out, 16))
        return fail(LCL_ERR_INVALID_ARG, "layers must be 16-byte aligned device pointers");
    return overlay_impl(atlas, a, b, out, db, (int)op, flags, reinterpret_cast<cudaStream_t>(stream));
}

lcl_status lcl_label_area(const lcl_atlas *atlas, const void *layer, lcl_dtype dtype, uint32_t n_labels,
                          uint64_t *count_out, uint64_t *area_out, lcl_stream stream) {
    lcl_status s = check_atlas(atlas, false);
    if (s != LCL_OK) return s;
    const int db = dtype_bytes(dtype);
    if (!db) return fail(LCL_ERR_INVALID_ARG, "dtype must be LCL_U8 or LCL_U16");
    if (n_labels < 1 || n_labels > 65536) return fail(LCL_ERR_INVALID_ARG, "n_labels must be in [1, 65536]");
    if (!layer || !aligned(layer, 16)) return fail(LCL_ERR_INVALID_ARG, "layer must be a 16-byte aligned device pointer");
    if (!count_out || !area_out || !aligned(count_out, 8) || !aligned(area_out, 8))
        return fail(LCL_ERR_INVALID_ARG, "outputs must be 8-byte aligned device pointers");
    return label_area_impl(atlas, layer, db, n_labels, count_out, area_out, reinterpret_cast<cudaStream_t>(stream));
}

// ---- numeric layers ----------------------------------------------------------------

lcl_status lcl_numeric_sphere(const lcl_atlas *atlas, const lcl_numeric_layer *layer, const lcl_sphere *strokes,
                              int32_t n, uint64_t *hits_out, void *workspace, size_t ws_bytes, lcl_stream stream) {
    lcl_status s = check_atlas(atlas, true);
    if (s != LCL_OK) return s;
    s = check_numeric(layer, "layer");
    if (s != LCL_OK) return s;
    if (n < 0 || n > (1 << 24)) return fail(LCL_ERR_INVALID_ARG, "stroke count out of range");
    if (n == 0) return LCL_OK;
    if (!strokes) return fail(LCL_ERR_INVALID_ARG, "strokes is NULL");
    if (hits_out && !aligned(hits_out, 8)) return fail(LCL_ERR_INVALID_ARG, "hits_out must be 8-byte aligned");
    if (!workspace || !aligned(workspace, 256)) return fail(LCL_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
    if (ws_bytes < select_ws_bytes(atlas, n)) return fail(LCL_ERR_OUT_OF_MEMORY, "workspace smaller than lcl_select_workspace_bytes");
    const uint32_t vmax = value_mask(layer->type);
    for (int32_t k = 0; k < n; ++k) {
        const lcl_sphere &st = strokes[k];
        if (st.r2 < 0) return fail(LCL_ERR_INVALID_ARG, "stroke r2 < 0");
        if (st.label & ~vmax) return fail(LCL_ERR_INVALID_ARG, "stroke value is wider than the layer type");
        if ((st.flags & ~0x1FFu) || (st.flags & 15u) > 8 || ((st.flags >> 4) & 15u) > 8)
            return fail(LCL_ERR_INVALID_ARG, "stroke flags: padding radius and thickness at most 8, LCL_ERASE, other bits 0");
        if ((s = check_padding_rows(atlas, st.flags)) != LCL_OK) return s;
        const int32_t lo = -(1 << 22), hi = (1 << 22) + (1 << 21);
        if (st.cx < lo || st.cx > hi || st.cy < lo || st.cy > hi || st.cz < lo || st.cz > hi)
            return fail(LCL_ERR_INVALID_ARG, "stroke centre outside [-2^22, 2^22 + 2^21]");
    }
    return numeric_sphere_impl(atlas, layer->data, layer->type & 15, layer->mask, strokes, n, hits_out, workspace,
                               reinterpret_cast<cudaStream_t>(stream));
}

lcl_status lcl_numeric_lasso(const lcl_atlas *atlas, const lcl_numeric_layer *layer, const lcl_camera *camera,
                             const float *depth, const float *poly_xy, int32_t n_vertices, uint32_t value,
                             uint32_t flags, float bias, uint64_t *hits_out, void *workspace, size_t ws_bytes,
                             lcl_stream stream) {
    lcl_status s = check_atlas(atlas, true);
    if (s != LCL_OK) return s;
    s = check_numeric(layer, "layer");
    if (s != LCL_OK) return s;
    s = check_camera(camera);
    if (s != LCL_OK) return s;
    if (!depth || !aligned(depth, 4)) return fail(LCL_ERR_INVALID_ARG, "depth must be a 4-byte aligned device pointer");
    if (!poly_xy) return fail(LCL_ERR_INVALID_ARG, "polygon is NULL");
    if (n_vertices < 3 || n_vertices > LCL_MAX_LASSO_VERTICES)
        return fail(LCL_ERR_UNSUPPORTED, "lasso polygons need 3..64 vertices");
    for (int i = 0; i < 2 * n_vertices; ++i)
        if (!std::isfinite(poly_xy[i])) return fail(LCL_ERR_INVALID_ARG, "polygon vertex is not finite");
    if (value & ~value_mask(layer->type)) return fail(LCL_ERR_INVALID_ARG, "value is wider than the layer type");
    if ((flags & ~(0xFFu | LCL_ERASE)) || (flags & 15u) > 8 || ((flags >> 4) & 15u) > 8)
        return fail(LCL_ERR_INVALID_ARG, "flags: padding radius and thickness at most 8, LCL_ERASE, other bits 0");
    if ((s = check_padding_rows(atlas, flags)) != LCL_OK) return s;
    if (!std::isfinite(bias)) return fail(LCL_ERR_INVALID_ARG, "bias is not finite");
    if (hits_out && !aligned(hits_out, 8)) return fail(LCL_ERR_INVALID_ARG, "hits_out must be 8-byte aligned");
    if (!workspace || !aligned(workspace, 256)) return fail(LCL_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
    if (ws_bytes < select_ws_bytes(atlas, 1)) return fail(LCL_ERR_OUT_OF_MEMORY, "workspace smaller than lcl_select_workspace_bytes");
    return numeric_lasso_impl(atlas, layer->data, layer->type & 15, layer->mask, value, flags, camera, depth, poly_xy,
                              n_vertices, bias, hits_out, workspace, reinterpret_cast<cudaStream_t>(stream));
}

lcl_status lcl_numeric_tool(const lcl_atlas *atlas, const lcl_numeric_layer *layer, const lcl_camera *camera,
                            const float *depth, const lcl_tool *tool, uint32_t value, uint32_t flags, float bias,
                            uint64_t *hits_out, void *workspace, size_t ws_bytes, lcl_stream stream) {
    lcl_status s = check_atlas(atlas, true);
    if (s != LCL_OK) return s;
    s = check_numeric(layer, "layer");
    if (s != LCL_OK) return s;
    s = check_camera(camera);
    if (s != LCL_OK) return s;
    if (!depth || !aligned(depth, 4)) return fail(LCL_ERR_INVALID_ARG, "depth must be a 4-byte aligned device pointer");
    s = check_tool(tool);
    if (s != LCL_OK) return s;
    if ((s = check_padding_rows(atlas, tool->flags)) != LCL_OK) return s;
    if (value & ~value_mask(layer->type)) return fail(LCL_ERR_INVALID_ARG, "value is wider than the layer type");
    if (flags & ~LCL_ERASE) return fail(LCL_ERR_INVALID_ARG, "flags must be 0 or LCL_ERASE");
    if (!std::isfinite(bias)) return fail(LCL_ERR_INVALID_ARG, "bias is not finite");
    if (hits_out && !aligned(hits_out, 8)) return fail(LCL_ERR_INVALID_ARG, "hits_out must be 8-byte aligned");
    if (!workspace || !aligned(workspace, 256)) return fail(LCL_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
    if (ws_bytes < select_ws_bytes(atlas, 1)) return fail(LCL_ERR_OUT_OF_MEMORY, "workspace smaller than lcl_select_workspace_bytes");
    return numeric_tool_impl(atlas, layer->data, layer->type & 15, layer->mask, value, flags, camera, depth, tool, bias,
                             hits_out, workspace, reinterpret_cast<cudaStream_t>(stream));
}

lcl_status lcl_numeric_arith(const lcl_atlas *atlas, const lcl_numeric_layer *a, const lcl_numeric_layer *b,
                             uint32_t b_value, const lcl_numeric_layer *out, lcl_arith op, lcl_stream stream) {
    lcl_status s = check_atlas(atlas, false);
    if (s != LCL_OK) return s;
    if ((s = check_numeric(a, "a")) != LCL_OK) return s;
    if (b && (s = check_numeric(b, "b")) != LCL_OK) return s;
    if ((s = check_numeric(out, "out")) != LCL_OK) return s;
    if ((b && b->type != a->type) || out->type != a->type)
        return fail(LCL_ERR_INVALID_ARG, "numeric layers of an arithmetic overlay must have one type");
    if ((int)op < LCL_ADD || (int)op > LCL_MAX) return fail(LCL_ERR_INVALID_ARG, "unknown arithmetic op");
    if (op == LCL_DIV && (a->type >> 4) != 3) return fail(LCL_ERR_UNSUPPORTED, "LCL_DIV is for float layers only");
    if (!b && (b_value & ~value_mask(a->type))) return fail(LCL_ERR_INVALID_ARG, "scalar is wider than the layer type");
    return numeric_arith_impl(atlas, a->type, a->data, a->mask, b ? b->data : nullptr, b ? b->mask : nullptr, b_value,
                              out->data, out->mask, (int)op, reinterpret_cast<cudaStream_t>(stream));
}

lcl_status lcl_numeric_select(const lcl_atlas *atlas, const lcl_numeric_layer *values, lcl_cmp cmp,
                              uint32_t threshold, void *layer, lcl_dtype dtype, uint32_t label, uint64_t *hits_out,
                              lcl_stream stream) {
    lcl_status s = check_atlas(atlas, false);
    if (s != LCL_OK) return s;
    if ((s = check_numeric(values, "values")) != LCL_OK) return s;
    const int db = dtype_bytes(dtype);
    if (!db) return fail(LCL_ERR_INVALID_ARG, "dtype must be LCL_U8 or LCL_U16");
    if (!layer || !aligned(layer, 16)) return fail(LCL_ERR_INVALID_ARG, "layer must be a 16-byte aligned device pointer");
    if ((int)cmp < LCL_LT || (int)cmp > LCL_NE) return fail(LCL_ERR_INVALID_ARG, "unknown comparison");
    if (threshold & ~value_mask(values->type)) return fail(LCL_ERR_INVALID_ARG, "threshold is wider than the layer type");
    if (label > (db == 1 ? 0xFFu : 0xFFFFu)) return fail(LCL_ERR_INVALID_ARG, "label does not fit the layer dtype");
    if (hits_out && !aligned(hits_out, 8)) return fail(LCL_ERR_INVALID_ARG, "hits_out must be 8-byte aligned");
    return numeric_select_impl(atlas, values->type, values->data, values->mask, (int)cmp, threshold, layer, db, label,
                               hits_out, reinterpret_cast<cudaStream_t>(stream));
}

lcl_status lcl_numeric_stats(const lcl_atlas *atlas, const lcl_numeric_layer *values, const void *zones,
                             lcl_dtype zone_dtype, uint32_t n_labels, lcl_zone_stats *out, lcl_stream stream) {
    lcl_status s = check_atlas(atlas, false);
    if (s != LCL_OK) return s;
    if ((s = check_numeric(values, "values")) != LCL_OK) return s;
    if (n_labels < 1 || n_labels > 65536) return fail(LCL_ERR_INVALID_ARG, "n_labels must be in [1, 65536]");
    int zb = 0;
    if (zones) {
        zb = dtype_bytes(zone_dtype);
        if (!zb) return fail(LCL_ERR_INVALID_ARG, "zone dtype must be LCL_U8 or LCL_U16");
        if (!aligned(zones, 16)) return fail(LCL_ERR_INVALID_ARG, "zones must be a 16-byte aligned device pointer");
    } else if (n_labels != 1) {
        return fail(LCL_ERR_INVALID_ARG, "without zones n_labels must be 1");
    }
    if (!out || !aligned(out, 16)) return fail(LCL_ERR_INVALID_ARG, "out must be a 16-byte aligned device pointer");
    return numeric_stats_impl(atlas, values->type, values->data, values->mask, zones, zb, n_labels, out,
                              reinterpret_cast<cudaStream_t>(stream));
}

const char *lcl_status_str(lcl_status status) {
    switch (status) {
    case LCL_OK: return "LCL_OK";
    case LCL_ERR_INVALID_ARG: return "LCL_ERR_INVALID_ARG";
    case LCL_ERR_OUT_OF_MEMORY: return "LCL_ERR_OUT_OF_MEMORY";
    case LCL_ERR_CUDA: return "LCL_ERR_CUDA";
    case LCL_ERR_UNSUPPORTED: return "LCL_ERR_UNSUPPORTED";
    case LCL_ERR_TIMEOUT: return "LCL_ERR_TIMEOUT";
    case LCL_ERR_INTERNAL: return "LCL_ERR_INTERNAL";
    }
    return "LCL_ERR_UNKNOWN";
}

const char *lcl_last_error(void) { return g_last_error.c_str(); }

lcl_status lcl_check_division(uint64_t n, uint32_t seed, uint64_t *counts, lcl_stream stream) {
    if (!counts || !aligned(counts, 8)) return fail(LCL_ERR_INVALID_ARG, "counts must be an 8-byte aligned device pointer");
    return division_check_impl(n, seed, counts, reinterpret_cast<cudaStream_t>(stream));
}

uint32_t lcl_build_flags(void) {
#ifdef LCL_DEBUG_BOUNDS
    return LCL_BUILD_BOUNDS_CHECKS;
#else
    return 0u;
#endif
}

size_t lcl_describe_site(uint32_t site, char *buf, size_t n) {
    const uint32_t h = site >> 16, line = site & 0xFFFFu;
    const char *name = nullptr;
    for (const char *cand : kSourceNames)
        if (file_hash16(cand) == h) name = cand;
    char tmp[64];
    if (name) std::snprintf(tmp, sizeof(tmp), "%s:%u", name, line);
    else std::snprintf(tmp, sizeof(tmp), "file#%04x:%u", h, line);
    const size_t len = std::strlen(tmp);
    if (buf && n) {
        std::strncpy(buf, tmp, n - 1);
        buf[n - 1] = '\0';
    }
    return len;
}

lcl_status lcl_last_device_status(lcl_stream stream) {
    const cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "lcl_last_device_status: the stream reported an error");
    std::vector<BoundsReader> readers;
    {
        std::lock_guard<std::mutex> lock(bounds_mu());
        readers = bounds_readers();
    }
    BoundsRecord first = {0, 0, 0, 0};
    unsigned long long total = 0;
    for (BoundsReader r : readers) {
        BoundsRecord rec;
        e = r(st, &rec);
        if (e != cudaSuccess) return cuda_fail(e, "lcl_last_device_status: reading a bounds record");
        if (rec.count && !total) first = rec;
        total += rec.count;
    }
    if (!total) return LCL_OK;
    char where[64];
    lcl_describe_site((uint32_t)first.site, where, sizeof(where));
    char msg[256];
    std::snprintf(msg, sizeof(msg), "bounds check at %s: index %lld outside [0, %llu); %llu out-of-range accesses skipped",
                  where, (long long)first.index, first.extent, total);
    return fail(LCL_ERR_INTERNAL, msg);
}

uint64_t lcl_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

}  // extern "C"
