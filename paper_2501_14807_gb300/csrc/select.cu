// select.cu -- per-texel selection edits: the sphere brush and the screen-space lasso
// (arXiv 2501.14807, Section 4.3.1, Fig. 3: depth test, projection of the tool, shape mask,
// then the selected value is stored in the texels that survive).
//
// Every stroke is two launches on the caller's stream:
//   cull   one CTA per super-tile (16 x 16 tiles).  The CTA leaves at once if the
//          super-tile's box cannot touch the stroke; otherwise each thread tests one tile
//          box and the candidates are appended to a list with one atomic per warp (ballot +
//          popc).  Both tests are conservative, so culling never changes a result.
//   apply  a persistent grid (a few CTAs per SM) walks the candidate list; each thread owns
//          four consecutive texels of a tile row: three 16-byte loads of the position planes,
//          the per-texel test, and one 4-byte (uint8) or 8-byte (uint16) label word written
//          only if a texel in it was hit (read first only if some of its texels were not).
// Strokes of one call run in order (stream order), so a later stroke overwrites an earlier
// one.  The hit count is a per-warp popcount reduced per CTA into one 64-bit atomic.
#include <cmath>

#include "lcl_impl.cuh"

namespace lcl {
namespace {

struct AtlasDev {
    const int32_t *px, *py, *pz;
    const int32_t *tile_box, *super_box;
    int32_t w, h, T, tiles_x, tiles_y;
};

AtlasDev dev_view(const lcl_atlas *a) {
    AtlasDev d;
    d.px = a->pos_x;
    d.py = a->pos_y;
    d.pz = a->pos_z;
    d.tile_box = a->tile_box;
    d.super_box = a->super_box;
    d.w = a->width;
    d.h = a->height;
    d.T = a->tile;
    d.tiles_x = a->tiles_x;
    d.tiles_y = a->tiles_y;
    return d;
}

struct SphereArg {
    int64_t cx, cy, cz, r2;
    uint32_t label;
};

__global__ void k_sel_init(uint32_t *counters, int32_t n, unsigned long long *hits) {
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        counters[i] = 0;
        if (hits) hits[i] = 0;
    }
}

__device__ __forceinline__ int64_t box_dist2(int4 lo, int4 hi, const SphereArg &s) {
    int64_t ex = max(max((int64_t)lo.x - s.cx, s.cx - (int64_t)hi.x), (int64_t)0);
    int64_t ey = max(max((int64_t)lo.y - s.cy, s.cy - (int64_t)hi.y), (int64_t)0);
    int64_t ez = max(max((int64_t)lo.z - s.cz, s.cz - (int64_t)hi.z), (int64_t)0);
    return ex * ex + ey * ey + ez * ez;
}

// Appends this lane's tile to the candidate list if `cand`; one atomic per warp.
__device__ __forceinline__ void append_candidate(bool cand, uint32_t tile, uint32_t *counter, uint32_t *list) {
    uint32_t m = __ballot_sync(0xffffffffu, cand);
    if (!m) return;
    const int lane = threadIdx.x & 31;
    uint32_t base = 0;
    if (lane == __ffs(m) - 1) base = atomicAdd(counter, (uint32_t)__popc(m));
    base = __shfl_sync(0xffffffffu, base, __ffs(m) - 1);
    if (cand) list[base + __popc(m & ((1u << lane) - 1))] = tile;
}

__global__ void __launch_bounds__(kThreads) k_sphere_cull(AtlasDev a, SphereArg s, uint32_t *counter,
                                                          uint32_t *list) {
    const int4 *sb = reinterpret_cast<const int4 *>(a.super_box + 8 * ((int64_t)blockIdx.y * gridDim.x + blockIdx.x));
    int4 slo = sb[0], shi = sb[1];
    if (slo.w == 0 || box_dist2(slo, shi, s) > s.r2) return;  // uniform over the CTA
    const int32_t tx = blockIdx.x * LCL_SUPER + (threadIdx.x % LCL_SUPER);
    const int32_t ty = blockIdx.y * LCL_SUPER + (threadIdx.x / LCL_SUPER);
    bool cand = false;
    if (tx < a.tiles_x && ty < a.tiles_y) {
        const int4 *tb = reinterpret_cast<const int4 *>(a.tile_box + 8 * ((int64_t)ty * a.tiles_x + tx));
        int4 lo = tb[0], hi = tb[1];
        cand = lo.w > 0 && box_dist2(lo, hi, s) <= s.r2;
    }
    append_candidate(cand, (uint32_t)(ty * a.tiles_x + tx), counter, list);
}

// Writes `label` into the texels of one 4-texel word whose bit is set in `m` (m != 0).
template <typename L>
__device__ __forceinline__ void store_hits(L *layer, int64_t l, uint32_t m, uint32_t label);

template <>
__device__ __forceinline__ void store_hits<uint8_t>(uint8_t *layer, int64_t l, uint32_t m, uint32_t label) {
    uint32_t *p = reinterpret_cast<uint32_t *>(layer + l);
    uint32_t rep = label * 0x01010101u;
    if (m == 0xFu) {
        *p = rep;
        return;
    }
    uint32_t bm = (m * 0x00204081u) & 0x01010101u;  // bit k of m -> byte k
    bm *= 0xFFu;
    *p = (*p & ~bm) | (rep & bm);
}

template <>
__device__ __forceinline__ void store_hits<uint16_t>(uint16_t *layer, int64_t l, uint32_t m, uint32_t label) {
    uint2 *p = reinterpret_cast<uint2 *>(layer + l);
    uint32_t rep = label * 0x00010001u;
    if (m == 0xFu) {
        *p = make_uint2(rep, rep);
        return;
    }
    uint2 o = *p;
    uint32_t lo = ((m & 1u) ? 0x0000FFFFu : 0u) | ((m & 2u) ? 0xFFFF0000u : 0u);
    uint32_t hi = ((m & 4u) ? 0x0000FFFFu : 0u) | ((m & 8u) ? 0xFFFF0000u : 0u);
    *p = make_uint2((o.x & ~lo) | (rep & lo), (o.y & ~hi) | (rep & hi));
}

__device__ __forceinline__ void add_hits(unsigned long long *hits, uint32_t cnt) {
    if (!hits) return;
    __shared__ uint32_t s_cnt;
    if (threadIdx.x == 0) s_cnt = 0;
    __syncthreads();
    for (int o = 16; o; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(&s_cnt, cnt);
    __syncthreads();
    if (threadIdx.x == 0 && s_cnt) atomicAdd(hits, (unsigned long long)s_cnt);
}

template <typename L>
__global__ void __launch_bounds__(kThreads) k_sphere_apply(AtlasDev a, L *__restrict__ layer, SphereArg s,
                                                           const uint32_t *__restrict__ counter,
                                                           const uint32_t *__restrict__ list,
                                                           unsigned long long *hits) {
    const uint32_t n = *counter;
    const int32_t qpr = a.T / 4, nq = a.T * qpr;
    uint32_t cnt = 0;
    for (uint32_t i = blockIdx.x; i < n; i += gridDim.x) {
        const uint32_t tile = list[i];
        const int32_t tx = tile % a.tiles_x, ty = tile / a.tiles_x;
        for (int32_t qd = threadIdx.x; qd < nq; qd += kThreads) {
            const int32_t x = tx * a.T + 4 * (qd % qpr), y = ty * a.T + qd / qpr;
            if (x >= a.w || y >= a.h) continue;
            const int64_t l = (int64_t)y * a.w + x;
            const int4 X = __ldg(reinterpret_cast<const int4 *>(a.px + l));
            const int4 Y = __ldg(reinterpret_cast<const int4 *>(a.py + l));
            const int4 Z = __ldg(reinterpret_cast<const int4 *>(a.pz + l));
            // Uncovered texels hold x = INT32_MIN, y = z = 0: their squared distance exceeds
            // 2^61, above every accepted r2 (<= 2^50), so they never test as hit.
            const int32_t xs[4] = {X.x, X.y, X.z, X.w}, ys[4] = {Y.x, Y.y, Y.z, Y.w}, zs[4] = {Z.x, Z.y, Z.z, Z.w};
            uint32_t m = 0;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                int64_t dx = (int64_t)xs[k] - s.cx, dy = (int64_t)ys[k] - s.cy, dz = (int64_t)zs[k] - s.cz;
                m |= (dx * dx + dy * dy + dz * dz <= s.r2 ? 1u : 0u) << k;
            }
            if (m) {
                store_hits<L>(layer, l, m, s.label);
                cnt += __popc(m);
            }
        }
    }
    add_hits(hits, cnt);
}

// ---- lasso ---------------------------------------------------------------------------

struct LassoArg {
    float m[16];
    float ws, hs;           // screen size as float
    int32_t w_s, h_s;
    float bias;
    uint32_t label;
    int32_t nv;
    float bx0, by0, bx1, by1;  // polygon bbox (clipped to the screen) widened by a margin
    float vx[LCL_MAX_LASSO_VERTICES + 1], vy[LCL_MAX_LASSO_VERTICES + 1];  // vertex nv = vertex 0
};

// Conservative: false only if no point of the box can project inside the widened lasso bbox.
__device__ bool box_may_touch(const LassoArg &p, int4 lo, int4 hi) {
    float xmin = INFINITY, xmax = -INFINITY, ymin = INFINITY, ymax = -INFINITY;
#pragma unroll 1
    for (int c = 0; c < 8; ++c) {
        float x = (float)((c & 1) ? hi.x : lo.x), y = (float)((c & 2) ? hi.y : lo.y), z = (float)((c & 4) ? hi.z : lo.z);
        float cw = clip_row(p.m + 12, x, y, z);
        if (!(cw > 0.0f)) return true;
        float xs = screen_of(__fdiv_rn(clip_row(p.m, x, y, z), cw), p.ws);
        float ys = screen_of(__fdiv_rn(clip_row(p.m + 4, x, y, z), cw), p.hs);
        xmin = fminf(xmin, xs); xmax = fmaxf(xmax, xs);
        ymin = fminf(ymin, ys); ymax = fmaxf(ymax, ys);
    }
    return !(xmax < p.bx0 || xmin > p.bx1 || ymax < p.by0 || ymin > p.by1);
}

__global__ void __launch_bounds__(kThreads) k_lasso_cull(AtlasDev a, const __grid_constant__ LassoArg p,
                                                         uint32_t *counter, uint32_t *list) {
    const int4 *sb = reinterpret_cast<const int4 *>(a.super_box + 8 * ((int64_t)blockIdx.y * gridDim.x + blockIdx.x));
    int4 slo = sb[0], shi = sb[1];
    if (slo.w == 0 || !box_may_touch(p, slo, shi)) return;
    const int32_t tx = blockIdx.x * LCL_SUPER + (threadIdx.x % LCL_SUPER);
    const int32_t ty = blockIdx.y * LCL_SUPER + (threadIdx.x / LCL_SUPER);
    bool cand = false;
    if (tx < a.tiles_x && ty < a.tiles_y) {
        const int4 *tb = reinterpret_cast<const int4 *>(a.tile_box + 8 * ((int64_t)ty * a.tiles_x + tx));
        int4 lo = tb[0], hi = tb[1];
        cand = lo.w > 0 && box_may_touch(p, lo, hi);
    }
    append_candidate(cand, (uint32_t)(ty * a.tiles_x + tx), counter, list);
}

// The lasso test of one texel, in the exact FP32 order of the definition.
__device__ __forceinline__ bool lasso_hit(const LassoArg &p, const float *vx, const float *vy,
                                          const float *__restrict__ depth, int32_t X, int32_t Y, int32_t Z) {
    if (X == INT32_MIN) return false;  // uncovered
    const float fx = (float)X, fy = (float)Y, fz = (float)Z;
    const float cw = clip_row(p.m + 12, fx, fy, fz);
    if (!(cw > 0.0f)) return false;
    const float zn = __fdiv_rn(clip_row(p.m + 8, fx, fy, fz), cw);
    if (!(zn >= 0.0f && zn <= 1.0f)) return false;
    const float xs = screen_of(__fdiv_rn(clip_row(p.m, fx, fy, fz), cw), p.ws);
    const float ys = screen_of(__fdiv_rn(clip_row(p.m + 4, fx, fy, fz), cw), p.hs);
    if (!(xs >= 0.0f && xs < p.ws && ys >= 0.0f && ys < p.hs)) return false;
    bool inside = false;
#pragma unroll 4
    for (int e = 0; e < p.nv; ++e) {
        const float ax = vx[e], ay = vy[e], bx = vx[e + 1], by = vy[e + 1];
        if ((ay > ys) != (by > ys)) {
            const float xi = __fadd_rn(__fdiv_rn(__fmul_rn(__fsub_rn(bx, ax), __fsub_rn(ys, ay)), __fsub_rn(by, ay)), ax);
            if (xs < xi) inside = !inside;
        }
    }
    if (!inside) return false;
    const int32_t ix = __float2int_rz(xs), iy = __float2int_rz(ys);
    const float d = __ldg(depth + (int64_t)iy * p.w_s + ix);
    return zn <= __fadd_rn(d, p.bias);
}

template <typename L>
__global__ void __launch_bounds__(kThreads) k_lasso_apply(AtlasDev a, L *__restrict__ layer,
                                                          const __grid_constant__ LassoArg p,
                                                          const float *__restrict__ depth,
                                                          const uint32_t *__restrict__ counter,
                                                          const uint32_t *__restrict__ list,
                                                          unsigned long long *hits) {
    __shared__ float vx[LCL_MAX_LASSO_VERTICES + 1], vy[LCL_MAX_LASSO_VERTICES + 1];
    for (int e = threadIdx.x; e <= p.nv; e += kThreads) {
        vx[e] = p.vx[e];
        vy[e] = p.vy[e];
    }
    __syncthreads();
    const uint32_t n = *counter;
    const int32_t qpr = a.T / 4, nq = a.T * qpr;
    uint32_t cnt = 0;
    for (uint32_t i = blockIdx.x; i < n; i += gridDim.x) {
        const uint32_t tile = list[i];
        const int32_t tx = tile % a.tiles_x, ty = tile / a.tiles_x;
        for (int32_t qd = threadIdx.x; qd < nq; qd += kThreads) {
            const int32_t x = tx * a.T + 4 * (qd % qpr), y = ty * a.T + qd / qpr;
            if (x >= a.w || y >= a.h) continue;
            const int64_t l = (int64_t)y * a.w + x;
            const int4 X = __ldg(reinterpret_cast<const int4 *>(a.px + l));
            const int4 Y = __ldg(reinterpret_cast<const int4 *>(a.py + l));
            const int4 Z = __ldg(reinterpret_cast<const int4 *>(a.pz + l));
            uint32_t m = 0;
            m |= lasso_hit(p, vx, vy, depth, X.x, Y.x, Z.x) ? 1u : 0u;
            m |= lasso_hit(p, vx, vy, depth, X.y, Y.y, Z.y) ? 2u : 0u;
            m |= lasso_hit(p, vx, vy, depth, X.z, Y.z, Z.z) ? 4u : 0u;
            m |= lasso_hit(p, vx, vy, depth, X.w, Y.w, Z.w) ? 8u : 0u;
            if (m) {
                store_hits<L>(layer, l, m, p.label);
                cnt += __popc(m);
            }
        }
    }
    add_hits(hits, cnt);
}

struct SelWs {
    uint32_t *counters, *list;
};

SelWs sel_ws(const lcl_atlas *a, int32_t n, void *ws) {
    SelWs w;
    char *base = static_cast<char *>(ws);
    w.counters = reinterpret_cast<uint32_t *>(base);
    w.list = reinterpret_cast<uint32_t *>(base + align256((size_t)(n + 1) * 4));
    return w;
}

int apply_grid(int32_t T) {
    (void)T;
    return sm_count() * 8;
}

}  // namespace

size_t select_ws_bytes(const lcl_atlas *a, int32_t n) {
    return align256((size_t)(n + 1) * 4) + align256((size_t)a->tiles_x * a->tiles_y * 4);
}

lcl_status select_sphere_impl(const lcl_atlas *atlas, void *layer, int dtype_bytes, const lcl_sphere *strokes,
                              int32_t n, uint64_t *hits, void *ws, cudaStream_t st) {
    const AtlasDev a = dev_view(atlas);
    const SelWs w = sel_ws(atlas, n, ws);
    unsigned long long *h = reinterpret_cast<unsigned long long *>(hits);
    k_sel_init<<<(n + kThreads - 1) / kThreads, kThreads, 0, st>>>(w.counters, n, h);
    const dim3 cg(atlas->supers_x, atlas->supers_y);
    const int ag = apply_grid(atlas->tile);
    for (int32_t k = 0; k < n; ++k) {
        SphereArg s;
        s.cx = strokes[k].cx;
        s.cy = strokes[k].cy;
        s.cz = strokes[k].cz;
        s.r2 = strokes[k].r2 > kR2Cap ? kR2Cap : strokes[k].r2;
        s.label = strokes[k].label;
        k_sphere_cull<<<cg, kThreads, 0, st>>>(a, s, w.counters + k, w.list);
        if (dtype_bytes == 1)
            k_sphere_apply<uint8_t><<<ag, kThreads, 0, st>>>(a, static_cast<uint8_t *>(layer), s, w.counters + k, w.list,
                                                            h ? h + k : nullptr);
        else
            k_sphere_apply<uint16_t><<<ag, kThreads, 0, st>>>(a, static_cast<uint16_t *>(layer), s, w.counters + k,
                                                             w.list, h ? h + k : nullptr);
    }
    count_launches(1 + 2 * n);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "lcl_select_sphere launch");
    return LCL_OK;
}

lcl_status select_lasso_impl(const lcl_atlas *atlas, void *layer, int dtype_bytes, const lcl_camera *cam,
                             const float *depth, const float *poly, int32_t nv, uint32_t label, float bias,
                             uint64_t *hits, void *ws, cudaStream_t st) {
    const AtlasDev a = dev_view(atlas);
    const SelWs w = sel_ws(atlas, 1, ws);
    unsigned long long *h = reinterpret_cast<unsigned long long *>(hits);
    LassoArg p;
    for (int i = 0; i < 16; ++i) p.m[i] = cam->m[i];
    p.ws = (float)cam->width;
    p.hs = (float)cam->height;
    p.w_s = cam->width;
    p.h_s = cam->height;
    p.bias = bias;
    p.label = label;
    p.nv = nv;
    float x0 = INFINITY, x1 = -INFINITY, y0 = INFINITY, y1 = -INFINITY;
    for (int i = 0; i < nv; ++i) {
        p.vx[i] = poly[2 * i];
        p.vy[i] = poly[2 * i + 1];
        x0 = std::fmin(x0, p.vx[i]);
        x1 = std::fmax(x1, p.vx[i]);
        y0 = std::fmin(y0, p.vy[i]);
        y1 = std::fmax(y1, p.vy[i]);
    }
    for (int i = nv; i <= LCL_MAX_LASSO_VERTICES; ++i) {
        p.vx[i] = p.vx[0];
        p.vy[i] = p.vy[0];
    }
    // The culling margin covers FP32 rounding of projected box corners (far below a pixel).
    const float margin = 2.0f + 1e-3f * (float)std::max(cam->width, cam->height);
    p.bx0 = std::fmax(x0, 0.0f) - margin;
    p.bx1 = std::fmin(x1, (float)cam->width) + margin;
    p.by0 = std::fmax(y0, 0.0f) - margin;
    p.by1 = std::fmin(y1, (float)cam->height) + margin;
    k_sel_init<<<1, kThreads, 0, st>>>(w.counters, 1, h);
    const dim3 cg(atlas->supers_x, atlas->supers_y);
    k_lasso_cull<<<cg, kThreads, 0, st>>>(a, p, w.counters, w.list);
    const int ag = apply_grid(atlas->tile);
    if (dtype_bytes == 1)
        k_lasso_apply<uint8_t><<<ag, kThreads, 0, st>>>(a, static_cast<uint8_t *>(layer), p, depth, w.counters, w.list, h);
    else
        k_lasso_apply<uint16_t><<<ag, kThreads, 0, st>>>(a, static_cast<uint16_t *>(layer), p, depth, w.counters,
                                                        w.list, h);
    count_launches(3);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "lcl_select_lasso launch");
    return LCL_OK;
}

}  // namespace lcl
