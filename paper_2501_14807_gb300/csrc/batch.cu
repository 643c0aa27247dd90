// batch.cu -- batched edits: many models, each with a queue of sphere and lasso strokes, edited
// by one cull launch and one persistent apply launch (capturable in a CUDA graph).
//
// The paper edits one layer of one model per operation (Section 4.3.1).  A server holding many
// models batches their queued strokes instead: the result must equal applying each model's
// strokes one by one, in queue order, so
//   k_batch_cull   gives every tile of every model a 64-bit mask of the model's queued strokes
//                  (queue order = bit order) whose conservative box test can reach the tile; the
//                  super-tile's mask is computed first and only its strokes are tested per tile;
//                  tiles with a non-empty mask become work items (model, tile, mask);
//   k_batch_apply  walks the items; a thread loads its four texels' positions once, runs the
//                  masked strokes in ascending order (a later hit overwrites an earlier label in
//                  registers), and writes each label word once.
// Each texel belongs to one item and one thread, so no two threads write a texel and the order
// per texel is the queue order: the result is bit-identical to sequential single-stroke calls.
#include <cstring>

#include "select_common.cuh"

namespace lcl {
namespace {

struct BModel {
    AtlasDev a;
    void *layer;
    int32_t dtype_bytes;
    int32_t s0, ns;   // this model's strokes: [s0, s0 + ns) of the batch's stroke array, ns <= 64
    int32_t super0;   // first flattened super-tile of this model
};

struct BStroke {
    int32_t kind;     // LCL_STROKE_SPHERE or LCL_STROKE_LASSO
    int32_t lasso;    // index into the lasso array
    SphereArg sphere;
};

struct BLasso {
    LassoArg arg;
    const float *depth;
};

struct BItem {
    uint32_t model, tile;
    unsigned long long mask;
};

// Workspace header (first 256 bytes), uploaded with the descriptors.
struct BHdr {
    int32_t n_models, n_strokes, n_lassos, n_supers;
    int64_t n_tiles;          // capacity of the item list
    unsigned int n_items;     // written by k_batch_cull
    int32_t pad;
};

struct BLayout {
    size_t hdr, models, strokes, lassos, super_model, items, total;
};

BLayout b_layout(int32_t n_models, int32_t n_strokes, int32_t n_lassos, int64_t n_supers, int64_t n_tiles) {
    BLayout L;
    L.hdr = 0;
    L.models = align256(sizeof(BHdr));
    L.strokes = L.models + align256((size_t)n_models * sizeof(BModel));
    L.lassos = L.strokes + align256((size_t)std::max(n_strokes, 1) * sizeof(BStroke));
    L.super_model = L.lassos + align256((size_t)std::max(n_lassos, 1) * sizeof(BLasso));
    L.items = L.super_model + align256((size_t)std::max<int64_t>(n_supers, 1) * 4);
    L.total = L.items + align256((size_t)std::max<int64_t>(n_tiles, 1) * sizeof(BItem));
    return L;
}

__device__ __forceinline__ bool stroke_may_touch(const BStroke &st, const BLasso *lassos, int4 lo, int4 hi) {
    if (lo.w == 0) return false;
    if (st.kind == LCL_STROKE_SPHERE) return box_dist2(lo, hi, st.sphere) <= st.sphere.r2;
    return box_may_touch(lassos[st.lasso].arg, lo, hi, lassos[st.lasso].depth);
}

__global__ void k_batch_init(BHdr *hdr) { hdr->n_items = 0; }

__global__ void __launch_bounds__(kThreads) k_batch_cull(const BHdr *__restrict__ hdr, const BModel *__restrict__ models,
                                                         const BStroke *__restrict__ strokes,
                                                         const BLasso *__restrict__ lassos,
                                                         const uint32_t *__restrict__ super_model, BItem *items,
                                                         unsigned int *n_items) {
    pdl_wait();
    pdl_allow_next();
    __shared__ unsigned long long s_mask;
    const int32_t n_supers = hdr->n_supers;
    for (int32_t g = blockIdx.x; g < n_supers; g += gridDim.x) {
        const uint32_t mi = super_model[g];
        const BModel &M = models[mi];
        const AtlasDev &a = M.a;
        const int32_t sidx = g - M.super0;
        if (threadIdx.x == 0) s_mask = 0ull;
        __syncthreads();
        const int4 *sb = reinterpret_cast<const int4 *>(a.super_box + 8 * (int64_t)sidx);
        const int4 slo = sb[0], shi = sb[1];
        // strokes that can reach the super-tile, one thread per stroke (ns <= 64)
        if (threadIdx.x < (unsigned)M.ns && stroke_may_touch(strokes[M.s0 + threadIdx.x], lassos, slo, shi))
            atomicOr(&s_mask, 1ull << threadIdx.x);
        __syncthreads();
        const unsigned long long smask = s_mask;
        __syncthreads();
        if (smask == 0ull) continue;  // uniform over the CTA
        const int32_t tx = (sidx % a.supers_x) * LCL_SUPER + (threadIdx.x % LCL_SUPER);
        const int32_t ty = (sidx / a.supers_x) * LCL_SUPER + (threadIdx.x / LCL_SUPER);
        unsigned long long mask = 0ull;
        if (tx < a.tiles_x && ty < a.tiles_y) {
            const int4 *tb = reinterpret_cast<const int4 *>(a.tile_box + 8 * ((int64_t)ty * a.tiles_x + tx));
            const int4 lo = tb[0], hi = tb[1];
            for (unsigned long long m = smask; m; m &= m - 1) {
                const int k = __ffsll((long long)m) - 1;
                if (stroke_may_touch(strokes[M.s0 + k], lassos, lo, hi)) mask |= 1ull << k;
            }
        }
        const bool cand = mask != 0ull;
        const uint32_t bal = __ballot_sync(0xffffffffu, cand);
        if (bal) {
            const int lane = threadIdx.x & 31;
            uint32_t base = 0;
            if (lane == __ffs(bal) - 1) base = atomicAdd(n_items, (unsigned)__popc(bal));
            base = __shfl_sync(0xffffffffu, base, __ffs(bal) - 1);
            if (cand) {
                BItem it;
                it.model = mi;
                it.tile = (uint32_t)(ty * a.tiles_x + tx);
                it.mask = mask;
                items[base + __popc(bal & ((1u << lane) - 1))] = it;
            }
        }
    }
}

// Writes per-texel labels lab[k] into the texels of a quad whose bit is set in m (m != 0).
template <typename L>
__device__ __forceinline__ void store_labels(L *layer, int64_t l, uint32_t m, const uint32_t lab[4]);

template <>
__device__ __forceinline__ void store_labels<uint8_t>(uint8_t *layer, int64_t l, uint32_t m, const uint32_t lab[4]) {
    uint32_t *p = reinterpret_cast<uint32_t *>(layer + l);
    const uint32_t v = (lab[0] & 0xFFu) | ((lab[1] & 0xFFu) << 8) | ((lab[2] & 0xFFu) << 16) | ((lab[3] & 0xFFu) << 24);
    if (m == 0xFu) {
        *p = v;
        return;
    }
    const uint32_t bm = ((m * 0x00204081u) & 0x01010101u) * 0xFFu;
    *p = (*p & ~bm) | (v & bm);
}

template <>
__device__ __forceinline__ void store_labels<uint16_t>(uint16_t *layer, int64_t l, uint32_t m, const uint32_t lab[4]) {
    uint2 *p = reinterpret_cast<uint2 *>(layer + l);
    const uint32_t v0 = (lab[0] & 0xFFFFu) | (lab[1] << 16), v1 = (lab[2] & 0xFFFFu) | (lab[3] << 16);
    if (m == 0xFu) {
        *p = make_uint2(v0, v1);
        return;
    }
    const uint2 o = *p;
    const uint32_t lo = ((m & 1u) ? 0x0000FFFFu : 0u) | ((m & 2u) ? 0xFFFF0000u : 0u);
    const uint32_t hi = ((m & 4u) ? 0x0000FFFFu : 0u) | ((m & 8u) ? 0xFFFF0000u : 0u);
    *p = make_uint2((o.x & ~lo) | (v0 & lo), (o.y & ~hi) | (v1 & hi));
}

template <typename L>
__device__ __forceinline__ void apply_item(const BModel &M, const BItem &it, const BStroke *__restrict__ strokes,
                                           const BLasso *__restrict__ lassos) {
    const AtlasDev &a = M.a;
    L *layer = static_cast<L *>(M.layer);
    const int32_t tx = it.tile % a.tiles_x, ty = it.tile / a.tiles_x;
    const int32_t qpr = a.T / 4, nq = a.T * qpr;
    for (int32_t qd = threadIdx.x; qd < nq; qd += kThreads) {
        const int32_t x = tx * a.T + 4 * (qd % qpr), y = ty * a.T + qd / qpr;
        if (x >= a.w || y >= a.h) continue;
        const int64_t l = (int64_t)y * a.w + x;
        const int4 X = __ldg(reinterpret_cast<const int4 *>(a.px + l));
        const int4 Y = __ldg(reinterpret_cast<const int4 *>(a.py + l));
        const int4 Z = __ldg(reinterpret_cast<const int4 *>(a.pz + l));
        const int32_t xs[4] = {X.x, X.y, X.z, X.w}, ys[4] = {Y.x, Y.y, Y.z, Y.w}, zs[4] = {Z.x, Z.y, Z.z, Z.w};
        uint32_t lab[4] = {0u, 0u, 0u, 0u}, hit = 0u;
        for (unsigned long long m = it.mask; m; m &= m - 1) {
            const BStroke &st = strokes[M.s0 + __ffsll((long long)m) - 1];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                bool h;
                if (st.kind == LCL_STROKE_SPHERE) {
                    // uncovered texels hold x = INT32_MIN and never test as hit (see select.cu)
                    const int64_t dx = (int64_t)xs[k] - st.sphere.cx, dy = (int64_t)ys[k] - st.sphere.cy;
                    const int64_t dz = (int64_t)zs[k] - st.sphere.cz;
                    h = dx * dx + dy * dy + dz * dz <= st.sphere.r2;
                } else {
                    const BLasso &ls = lassos[st.lasso];
                    h = lasso_hit(ls.arg, ls.arg, ls.depth, xs[k], ys[k], zs[k]);
                }
                if (h) {
                    lab[k] = st.kind == LCL_STROKE_SPHERE ? st.sphere.label : lassos[st.lasso].arg.label;
                    hit |= 1u << k;
                }
            }
        }
        if (hit) store_labels<L>(layer, l, hit, lab);
    }
}

__global__ void __launch_bounds__(kThreads) k_batch_apply(const BModel *__restrict__ models,
                                                          const BStroke *__restrict__ strokes,
                                                          const BLasso *__restrict__ lassos,
                                                          const BItem *__restrict__ items,
                                                          const unsigned int *__restrict__ n_items) {
    pdl_wait();
    pdl_allow_next();
    const unsigned int n = *n_items;
    for (unsigned int i = blockIdx.x; i < n; i += gridDim.x) {
        const BItem it = items[i];
        const BModel &M = models[it.model];
        if (M.dtype_bytes == 1) apply_item<uint8_t>(M, it, strokes, lassos);
        else apply_item<uint16_t>(M, it, strokes, lassos);
    }
}

}  // namespace

// ---- host side -------------------------------------------------------------------------

namespace {

lcl_status check_batch(const lcl_batch_model *models, int32_t n_models, const lcl_batch_stroke *strokes,
                       int32_t n_strokes, const lcl_batch_lasso *lassos, int32_t n_lassos, int64_t *n_supers,
                       int64_t *n_tiles) {
    if (n_models < 0 || n_strokes < 0 || n_lassos < 0) return fail(LCL_ERR_INVALID_ARG, "negative batch count");
    if ((n_models && !models) || (n_strokes && !strokes) || (n_lassos && !lassos))
        return fail(LCL_ERR_INVALID_ARG, "batch array is NULL");
    int64_t ns = 0, nt = 0;
    for (int32_t i = 0; i < n_models; ++i) {
        const lcl_batch_model &m = models[i];
        const lcl_atlas *a = m.atlas;
        if (!a || !a->pos_x || !a->tile_box || !a->super_box || a->tiles_x <= 0 || a->tiles_y <= 0)
            return fail(LCL_ERR_INVALID_ARG, "batch model needs a bound, whole atlas");
        if (m.dtype != LCL_U8 && m.dtype != LCL_U16) return fail(LCL_ERR_INVALID_ARG, "batch model dtype");
        if (!m.layer || (reinterpret_cast<uintptr_t>(m.layer) & 15))
            return fail(LCL_ERR_INVALID_ARG, "batch layers must be 16-byte aligned device pointers");
        if (m.n_strokes < 0 || m.n_strokes > LCL_BATCH_MAX_STROKES)
            return fail(LCL_ERR_UNSUPPORTED, "at most LCL_BATCH_MAX_STROKES (64) strokes per model per batch");
        if (m.first_stroke < 0 || (int64_t)m.first_stroke + m.n_strokes > n_strokes)
            return fail(LCL_ERR_INVALID_ARG, "batch model stroke range out of bounds");
        const uint32_t lab_max = m.dtype == LCL_U8 ? 0xFFu : 0xFFFFu;
        for (int32_t k = 0; k < m.n_strokes; ++k) {
            const lcl_batch_stroke &s = strokes[m.first_stroke + k];
            if (s.kind == LCL_STROKE_SPHERE) {
                const lcl_sphere &sp = s.sphere;
                const int32_t lo = -(1 << 22), hi = (1 << 22) + (1 << 21);
                if (sp.r2 < 0 || sp.label > lab_max || sp.cx < lo || sp.cx > hi || sp.cy < lo || sp.cy > hi ||
                    sp.cz < lo || sp.cz > hi || (sp.flags & ~0xFFu))
                    return fail(LCL_ERR_INVALID_ARG, "batch sphere stroke out of range");
                if (sp.flags != 0)
                    return fail(LCL_ERR_UNSUPPORTED, "texture padding is not supported in batched edits");
            } else if (s.kind == LCL_STROKE_LASSO) {
                if (s.lasso < 0 || s.lasso >= n_lassos) return fail(LCL_ERR_INVALID_ARG, "batch lasso index");
                if (lassos[s.lasso].label > lab_max) return fail(LCL_ERR_INVALID_ARG, "batch lasso label too wide");
            } else {
                return fail(LCL_ERR_INVALID_ARG, "unknown batch stroke kind");
            }
        }
        ns += (int64_t)a->supers_x * a->supers_y;
        nt += (int64_t)a->tiles_x * a->tiles_y;
    }
    for (int32_t j = 0; j < n_lassos; ++j) {
        const lcl_batch_lasso &L = lassos[j];
        const lcl_camera &c = L.camera;
        if (c.width < 1 || c.width > 16384 || c.height < 1 || c.height > 16384 || !L.depth || !L.poly_xy)
            return fail(LCL_ERR_INVALID_ARG, "batch lasso camera or buffers");
        for (int i = 0; i < 16; ++i)
            if (!std::isfinite(c.m[i])) return fail(LCL_ERR_INVALID_ARG, "batch lasso camera is not finite");
        if (L.n_vertices < 3 || L.n_vertices > LCL_MAX_LASSO_VERTICES)
            return fail(LCL_ERR_UNSUPPORTED, "lasso polygons need 3..64 vertices");
        for (int i = 0; i < 2 * L.n_vertices; ++i)
            if (!std::isfinite(L.poly_xy[i])) return fail(LCL_ERR_INVALID_ARG, "batch lasso vertex is not finite");
        if (!std::isfinite(L.bias)) return fail(LCL_ERR_INVALID_ARG, "batch lasso bias is not finite");
    }
    if (ns > INT32_MAX || nt > UINT32_MAX) return fail(LCL_ERR_UNSUPPORTED, "batch too large");
    *n_supers = ns;
    *n_tiles = nt;
    return LCL_OK;
}

struct LaunchInfo {  // what lcl_batch_launch needs on the host, kept at the start of the staging
    int32_t n_models, n_strokes, n_lassos, n_supers;
    int64_t n_tiles;
    int64_t ws_bytes;
};

}  // namespace

size_t batch_host_bytes(int32_t n_models, int32_t n_strokes, int32_t n_lassos, int64_t n_supers, int64_t n_tiles) {
    return align256(sizeof(LaunchInfo)) + b_layout(n_models, n_strokes, n_lassos, n_supers, n_tiles).items;
}

size_t batch_ws_bytes(int32_t n_models, int32_t n_strokes, int32_t n_lassos, int64_t n_supers, int64_t n_tiles) {
    return b_layout(n_models, n_strokes, n_lassos, n_supers, n_tiles).total;
}

lcl_status batch_sizes(const lcl_batch_model *models, int32_t n_models, int64_t *n_supers, int64_t *n_tiles) {
    int64_t ns = 0, nt = 0;
    for (int32_t i = 0; i < n_models; ++i) {
        if (!models[i].atlas) return fail(LCL_ERR_INVALID_ARG, "batch model without atlas");
        ns += (int64_t)models[i].atlas->supers_x * models[i].atlas->supers_y;
        nt += (int64_t)models[i].atlas->tiles_x * models[i].atlas->tiles_y;
    }
    *n_supers = ns;
    *n_tiles = nt;
    return LCL_OK;
}

lcl_status batch_launch_impl(void *ws, const void *host_staging, cudaStream_t st) {
    const LaunchInfo &info = *static_cast<const LaunchInfo *>(host_staging);
    const BLayout L = b_layout(info.n_models, info.n_strokes, info.n_lassos, info.n_supers, info.n_tiles);
    char *base = static_cast<char *>(ws);
    BHdr *hdr = reinterpret_cast<BHdr *>(base + L.hdr);
    const BModel *models = reinterpret_cast<const BModel *>(base + L.models);
    const BStroke *strokes = reinterpret_cast<const BStroke *>(base + L.strokes);
    const BLasso *lassos = reinterpret_cast<const BLasso *>(base + L.lassos);
    const uint32_t *super_model = reinterpret_cast<const uint32_t *>(base + L.super_model);
    BItem *items = reinterpret_cast<BItem *>(base + L.items);
    k_batch_init<<<1, 1, 0, st>>>(hdr);
    cudaError_t e = cudaSuccess;
    if (info.n_supers > 0) {
        const int cg = std::min<int64_t>(info.n_supers, resident_grid(k_batch_cull));
        e = launch_pdl(k_batch_cull, dim3(cg), st, (const BHdr *)hdr, models, strokes, lassos, super_model, items,
                       &hdr->n_items);
        if (e == cudaSuccess)
            e = launch_pdl(k_batch_apply, dim3(resident_grid(k_batch_apply)), st, models, strokes, lassos,
                           (const BItem *)items, (const unsigned int *)&hdr->n_items);
    }
    count_launches(info.n_supers > 0 ? 3 : 1);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "batch launch");
    return LCL_OK;
}

lcl_status batch_edit_impl(const lcl_batch_model *models, int32_t n_models, const lcl_batch_stroke *strokes,
                           int32_t n_strokes, const lcl_batch_lasso *lassos, int32_t n_lassos, void *ws,
                           size_t ws_bytes, void *host_staging, size_t host_bytes, cudaStream_t st) {
    int64_t n_supers = 0, n_tiles = 0;
    lcl_status s = check_batch(models, n_models, strokes, n_strokes, lassos, n_lassos, &n_supers, &n_tiles);
    if (s != LCL_OK) return s;
    const BLayout L = b_layout(n_models, n_strokes, n_lassos, n_supers, n_tiles);
    if (ws_bytes < L.total) return fail(LCL_ERR_OUT_OF_MEMORY, "batch workspace smaller than lcl_batch_workspace_bytes");
    const size_t need_host = align256(sizeof(LaunchInfo)) + L.items;
    if (host_bytes < need_host) return fail(LCL_ERR_OUT_OF_MEMORY, "batch staging smaller than lcl_batch_staging_bytes");
    char *hs = static_cast<char *>(host_staging);
    LaunchInfo info;
    info.n_models = n_models;
    info.n_strokes = n_strokes;
    info.n_lassos = n_lassos;
    info.n_supers = (int32_t)n_supers;
    info.n_tiles = n_tiles;
    info.ws_bytes = (int64_t)L.total;
    std::memcpy(hs, &info, sizeof(info));
    char *img = hs + align256(sizeof(LaunchInfo));  // image of the workspace up to the item list
    std::memset(img, 0, L.items);
    BHdr hdr;
    std::memset(&hdr, 0, sizeof(hdr));
    hdr.n_models = n_models;
    hdr.n_strokes = n_strokes;
    hdr.n_lassos = n_lassos;
    hdr.n_supers = (int32_t)n_supers;
    hdr.n_tiles = n_tiles;
    std::memcpy(img + L.hdr, &hdr, sizeof(hdr));
    BModel *bm = reinterpret_cast<BModel *>(img + L.models);
    uint32_t *super_model = reinterpret_cast<uint32_t *>(img + L.super_model);
    int32_t super0 = 0;
    for (int32_t i = 0; i < n_models; ++i) {
        const lcl_batch_model &m = models[i];
        BModel d;
        std::memset(&d, 0, sizeof(d));
        d.a = dev_view(m.atlas);
        d.layer = m.layer;
        d.dtype_bytes = m.dtype == LCL_U8 ? 1 : 2;
        d.s0 = m.first_stroke;
        d.ns = m.n_strokes;
        d.super0 = super0;
        bm[i] = d;
        const int32_t nsup = m.atlas->supers_x * m.atlas->supers_y;
        for (int32_t k = 0; k < nsup; ++k) super_model[super0 + k] = (uint32_t)i;
        super0 += nsup;
    }
    BStroke *bs = reinterpret_cast<BStroke *>(img + L.strokes);
    for (int32_t k = 0; k < n_strokes; ++k) {
        BStroke d;
        std::memset(&d, 0, sizeof(d));
        d.kind = strokes[k].kind;
        d.lasso = strokes[k].lasso;
        d.sphere.cx = strokes[k].sphere.cx;
        d.sphere.cy = strokes[k].sphere.cy;
        d.sphere.cz = strokes[k].sphere.cz;
        d.sphere.r2 = strokes[k].sphere.r2 > kR2Cap ? kR2Cap : strokes[k].sphere.r2;
        d.sphere.label = strokes[k].sphere.label;
        d.sphere.pad_r = 0;
        d.sphere.pad_t = 0;
        bs[k] = d;
    }
    BLasso *bl = reinterpret_cast<BLasso *>(img + L.lassos);
    for (int32_t j = 0; j < n_lassos; ++j) {
        fill_lasso_arg(bl[j].arg, &lassos[j].camera, lassos[j].poly_xy, lassos[j].n_vertices, lassos[j].label,
                       lassos[j].bias);
        bl[j].depth = lassos[j].depth;
    }
    cudaError_t e = cudaMemcpyAsync(ws, img, L.items, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e, "batch descriptor upload");
    return batch_launch_impl(ws, host_staging, st);
}

}  // namespace lcl
