// select.cu -- per-texel selection edits: the sphere brush and the screen-space lasso
// (arXiv 2501.14807, Section 4.3.1, Fig. 3: depth test, projection of the tool, shape mask,
// then the selected value is stored in the texels that survive).
//
// Culling: a stroke is tested against the box of every super-tile (16 x 16 tiles); where the
// super-tile's box can touch the stroke, each of its tiles' boxes is tested, one per thread, and
// the candidate tiles are appended to a list with one atomic per warp (ballot + popc).  Both
// tests are conservative, so culling never changes a result.
//
// Apply: a persistent grid (8 CTAs per SM) walks the candidate list; each thread owns four
// consecutive texels of a tile row: three 16-byte loads of the position planes, the per-texel
// test, and one 4-byte (uint8) or 8-byte (uint16) label word written only if a texel in it was
// hit (read first only if some of its texels were not).  The loads of the thread's next work
// item are issued before the current one is tested, so two items are in flight per thread.
//
// Sphere strokes take one launch each: the kernel that applies stroke k also culls stroke k + 1
// into the other of two candidate lists, and every launch is a programmatic dependent launch, so
// the next grid is scheduled while the current one drains and waits (griddepcontrol.wait) only
// for its completion.  Strokes of one call run in stream order, so a later stroke overwrites an
// earlier one.  Lassos take a cull and an apply launch.  Hit counts are per-warp popcounts
// reduced per CTA into one 64-bit atomic.
#include <algorithm>
#include <cmath>

#include "lcl_impl.cuh"

namespace lcl {
namespace {

struct AtlasDev {
    const int32_t *px, *py, *pz;
    const int32_t *tile_box, *super_box;
    int32_t w, h, T, tiles_x, tiles_y, supers_x, supers_y;
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
    d.supers_x = a->supers_x;
    d.supers_y = a->supers_y;
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

// Culls stroke s against super-tile `sidx`, appending its candidate tiles.  Uniform per CTA.
__device__ __forceinline__ void cull_super_sphere(const AtlasDev &a, const SphereArg &s, int32_t sidx,
                                                  uint32_t *counter, uint32_t *list) {
    const int4 *sb = reinterpret_cast<const int4 *>(a.super_box + 8 * (int64_t)sidx);
    const int4 slo = sb[0], shi = sb[1];
    if (slo.w == 0 || box_dist2(slo, shi, s) > s.r2) return;
    const int32_t tx = (sidx % a.supers_x) * LCL_SUPER + (threadIdx.x % LCL_SUPER);
    const int32_t ty = (sidx / a.supers_x) * LCL_SUPER + (threadIdx.x / LCL_SUPER);
    bool cand = false;
    if (tx < a.tiles_x && ty < a.tiles_y) {
        const int4 *tb = reinterpret_cast<const int4 *>(a.tile_box + 8 * ((int64_t)ty * a.tiles_x + tx));
        const int4 lo = tb[0], hi = tb[1];
        cand = lo.w > 0 && box_dist2(lo, hi, s) <= s.r2;
    }
    append_candidate(cand, (uint32_t)(ty * a.tiles_x + tx), counter, list);
}

// Programmatic dependent launch: wait for the previous grid on the stream to complete (its
// memory is then visible); let the next grid be scheduled.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_allow_next() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Culls the first stroke of a call.
__global__ void __launch_bounds__(kThreads) k_sphere_cull(AtlasDev a, SphereArg s, uint32_t *counter,
                                                          uint32_t *list) {
    pdl_wait();
    const int32_t n_super = a.supers_x * a.supers_y;
    for (int32_t sidx = blockIdx.x; sidx < n_super; sidx += gridDim.x) cull_super_sphere(a, s, sidx, counter, list);
    pdl_allow_next();
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

// One work item = one tile, or a 256-quad chunk of a larger tile; this thread's quad of it.
struct Item {
    int64_t l;  // linear index of the quad's first texel, -1 if the thread has no quad here
    int4 X, Y, Z;
};

__device__ __forceinline__ Item load_item(const AtlasDev &a, const uint32_t *__restrict__ list, uint32_t item,
                                          int cpt_log2, int32_t qpr, int32_t nq) {
    Item it;
    it.l = -1;
    const uint32_t tile = __ldg(list + (item >> cpt_log2));
    const int32_t qd = (int32_t)((item & ((1u << cpt_log2) - 1)) * kThreads + threadIdx.x);
    const int32_t tx = tile % a.tiles_x, ty = tile / a.tiles_x;
    const int32_t x = tx * a.T + 4 * (qd % qpr), y = ty * a.T + qd / qpr;
    if (qd < nq && x < a.w && y < a.h) {
        it.l = (int64_t)y * a.w + x;
        it.X = __ldg(reinterpret_cast<const int4 *>(a.px + it.l));
        it.Y = __ldg(reinterpret_cast<const int4 *>(a.py + it.l));
        it.Z = __ldg(reinterpret_cast<const int4 *>(a.pz + it.l));
    }
    return it;
}

// Hit mask of a quad.  Uncovered texels hold x = INT32_MIN, y = z = 0: their squared distance
// exceeds 2^61, above every accepted r2 (<= 2^50), so they never test as hit.
__device__ __forceinline__ uint32_t sphere_mask(const Item &it, const SphereArg &s) {
    const int32_t xs[4] = {it.X.x, it.X.y, it.X.z, it.X.w}, ys[4] = {it.Y.x, it.Y.y, it.Y.z, it.Y.w};
    const int32_t zs[4] = {it.Z.x, it.Z.y, it.Z.z, it.Z.w};
    uint32_t m = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int64_t dx = (int64_t)xs[k] - s.cx, dy = (int64_t)ys[k] - s.cy, dz = (int64_t)zs[k] - s.cz;
        m |= (dx * dx + dy * dy + dz * dz <= s.r2 ? 1u : 0u) << k;
    }
    return m;
}

// Applies stroke `s` from its candidate list and culls stroke `nxt` (if has_next) into the other list.
template <typename L>
__global__ void __launch_bounds__(kThreads) k_sphere_step(AtlasDev a, L *__restrict__ layer, SphereArg s,
                                                          const uint32_t *__restrict__ counter,
                                                          const uint32_t *__restrict__ list,
                                                          unsigned long long *hits, int has_next, SphereArg nxt,
                                                          uint32_t *next_counter, uint32_t *next_list) {
    pdl_wait();
    if (has_next) {
        const int32_t n_super = a.supers_x * a.supers_y;
        for (int32_t sidx = blockIdx.x; sidx < n_super; sidx += gridDim.x)
            cull_super_sphere(a, nxt, sidx, next_counter, next_list);
    }
    pdl_allow_next();
    const int32_t qpr = a.T / 4, nq = a.T * qpr;
    const int cpt_log2 = nq > kThreads ? 31 - __clz(nq / kThreads) : 0;
    const uint32_t n_items = *counter << cpt_log2;
    uint32_t cnt = 0;
    uint32_t item = blockIdx.x;
    Item cur;
    cur.l = -1;
    if (item < n_items) cur = load_item(a, list, item, cpt_log2, qpr, nq);
    for (; item < n_items; item += gridDim.x) {
        const uint32_t after = item + gridDim.x;
        Item next;
        next.l = -1;
        if (after < n_items) next = load_item(a, list, after, cpt_log2, qpr, nq);
        if (cur.l >= 0) {
            const uint32_t m = sphere_mask(cur, s);
            if (m) {
                store_hits<L>(layer, cur.l, m, s.label);
                cnt += __popc(m);
            }
        }
        cur = next;
    }
    add_hits(hits, cnt);
}

template <typename... K, typename... A>
cudaError_t launch_pdl(void (*kernel)(K...), dim3 grid, cudaStream_t st, A... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// ---- lasso ---------------------------------------------------------------------------

constexpr int kBands = 32;                                    // y-bands of lasso edges
constexpr int kBandEdgesMax = kBands * LCL_MAX_LASSO_VERTICES;

struct LassoArg {
    float m[16];
    float ws, hs;           // screen size as float
    int32_t w_s, h_s;
    float bias;
    uint32_t label;
    int32_t nv;
    float bx0, by0, bx1, by1;  // polygon bbox (clipped to the screen) widened by a margin, pixels
    float nx0, nx1, ny0, ny1;  // the same widened bbox in NDC, for the division-free reject
    float ymin, ymax;          // exact vertical extent of the polygon
    float band_y0, band_inv_h; // band of a point: floor((y - band_y0) * band_inv_h), clamped
    float vx[LCL_MAX_LASSO_VERTICES + 1], vy[LCL_MAX_LASSO_VERTICES + 1];  // vertex nv = vertex 0
    uint16_t band_off[kBands + 1];
    uint8_t band_edge[kBandEdgesMax];  // edge e runs from vertex e to vertex e + 1
};

struct LassoShared {
    float vx[LCL_MAX_LASSO_VERTICES + 1], vy[LCL_MAX_LASSO_VERTICES + 1];
    uint16_t band_off[kBands + 1];
    uint8_t band_edge[kBandEdgesMax];
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

// The lasso test of one texel.  The conditions of the definition are all required, so they are
// evaluated cheapest first; every value that decides the result is computed in the exact FP32
// order of the definition.  Two shortcuts are exact as well:
//  - a point more than the margin outside the polygon's bounding box (clipped to the screen) is
//    off screen or outside the polygon: left of every vertex each straddling edge counts, and a
//    closed polygon has an even number of those; right of every vertex none counts.  The test
//    compares clip-space x with the widened box times w (w > 0), so it needs no division; its
//    rounding is far below the 2-pixel margin;
//  - only edges listed for the point's y-band are tested: an edge can count only if its y-range
//    contains y, and each band lists every edge whose y-range comes within a margin of the band.
__device__ __forceinline__ bool lasso_hit(const LassoArg &p, const LassoShared &sh, const float *__restrict__ depth,
                                          int32_t X, int32_t Y, int32_t Z) {
    if (X == INT32_MIN) return false;  // uncovered
    const float fx = (float)X, fy = (float)Y, fz = (float)Z;
    const float cw = clip_row(p.m + 12, fx, fy, fz);
    if (!(cw > 0.0f)) return false;
    const float cx = clip_row(p.m, fx, fy, fz);
    if (cx < __fmul_rn(p.nx0, cw) || cx > __fmul_rn(p.nx1, cw)) return false;
    const float cy = clip_row(p.m + 4, fx, fy, fz);
    if (cy < __fmul_rn(p.ny0, cw) || cy > __fmul_rn(p.ny1, cw)) return false;
    const float xs = screen_of(__fdiv_rn(cx, cw), p.ws);
    const float ys = screen_of(__fdiv_rn(cy, cw), p.hs);
    if (!(xs >= 0.0f && xs < p.ws && ys >= 0.0f && ys < p.hs)) return false;
    if (!(ys >= p.ymin && ys < p.ymax)) return false;  // no edge straddles y
    int band = __float2int_rz(__fmul_rn(__fsub_rn(ys, p.band_y0), p.band_inv_h));
    band = band < 0 ? 0 : (band >= kBands ? kBands - 1 : band);
    bool inside = false;
    for (int k = sh.band_off[band]; k < sh.band_off[band + 1]; ++k) {
        const int e = sh.band_edge[k];
        const float ax = sh.vx[e], ay = sh.vy[e], bx = sh.vx[e + 1], by = sh.vy[e + 1];
        if ((ay > ys) != (by > ys)) {
            const float xi = __fadd_rn(__fdiv_rn(__fmul_rn(__fsub_rn(bx, ax), __fsub_rn(ys, ay)), __fsub_rn(by, ay)), ax);
            if (xs < xi) inside = !inside;
        }
    }
    if (!inside) return false;
    const float zn = __fdiv_rn(clip_row(p.m + 8, fx, fy, fz), cw);
    if (!(zn >= 0.0f && zn <= 1.0f)) return false;
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
    __shared__ LassoShared sh;
    for (int e = threadIdx.x; e <= p.nv; e += kThreads) {
        sh.vx[e] = p.vx[e];
        sh.vy[e] = p.vy[e];
    }
    for (int k = threadIdx.x; k <= kBands; k += kThreads) sh.band_off[k] = p.band_off[k];
    for (int k = threadIdx.x; k < p.band_off[kBands]; k += kThreads) sh.band_edge[k] = p.band_edge[k];
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
            m |= lasso_hit(p, sh, depth, X.x, Y.x, Z.x) ? 1u : 0u;
            m |= lasso_hit(p, sh, depth, X.y, Y.y, Z.y) ? 2u : 0u;
            m |= lasso_hit(p, sh, depth, X.z, Y.z, Z.z) ? 4u : 0u;
            m |= lasso_hit(p, sh, depth, X.w, Y.w, Z.w) ? 8u : 0u;
            if (m) {
                store_hits<L>(layer, l, m, p.label);
                cnt += __popc(m);
            }
        }
    }
    add_hits(hits, cnt);
}

struct SelWs {
    uint32_t *counters, *list, *list2;  // two candidate lists: strokes alternate between them
};

SelWs sel_ws(const lcl_atlas *a, int32_t n, void *ws) {
    SelWs w;
    char *base = static_cast<char *>(ws);
    w.counters = reinterpret_cast<uint32_t *>(base);
    w.list = reinterpret_cast<uint32_t *>(base + align256((size_t)(n + 1) * 4));
    w.list2 = reinterpret_cast<uint32_t *>(base + align256((size_t)(n + 1) * 4) +
                                           align256((size_t)a->tiles_x * a->tiles_y * 4));
    return w;
}

int apply_grid(int32_t T) {
    (void)T;
    return sm_count() * 8;
}

// A grid of as many CTAs as fit on the GPU at once (persistent loops need no second wave).
template <typename K>
int resident_grid(K kernel) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kThreads, 0) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    return per_sm * sm_count();
}

}  // namespace

size_t select_ws_bytes(const lcl_atlas *a, int32_t n) {
    return align256((size_t)(n + 1) * 4) + 2 * align256((size_t)a->tiles_x * a->tiles_y * 4);
}

lcl_status select_sphere_impl(const lcl_atlas *atlas, void *layer, int dtype_bytes, const lcl_sphere *strokes,
                              int32_t n, uint64_t *hits, void *ws, cudaStream_t st) {
    const AtlasDev a = dev_view(atlas);
    const SelWs w = sel_ws(atlas, n, ws);
    unsigned long long *h = reinterpret_cast<unsigned long long *>(hits);
    auto arg = [&](int32_t k) {
        SphereArg s;
        s.cx = strokes[k].cx;
        s.cy = strokes[k].cy;
        s.cz = strokes[k].cz;
        s.r2 = strokes[k].r2 > kR2Cap ? kR2Cap : strokes[k].r2;
        s.label = strokes[k].label;
        return s;
    };
    k_sel_init<<<(n + kThreads - 1) / kThreads, kThreads, 0, st>>>(w.counters, n, h);
    const int ag = dtype_bytes == 1 ? resident_grid(k_sphere_step<uint8_t>) : resident_grid(k_sphere_step<uint16_t>);
    const int n_super = atlas->supers_x * atlas->supers_y;
    cudaError_t e = launch_pdl(k_sphere_cull, dim3(std::min(n_super, ag)), st, a, arg(0), w.counters, w.list);
    for (int32_t k = 0; k < n && e == cudaSuccess; ++k) {
        uint32_t *cur_list = (k & 1) ? w.list2 : w.list, *next_list = (k & 1) ? w.list : w.list2;
        const int has_next = k + 1 < n;
        const SphereArg nxt = arg(has_next ? k + 1 : k);
        unsigned long long *hk = h ? h + k : nullptr;
        if (dtype_bytes == 1)
            e = launch_pdl(k_sphere_step<uint8_t>, dim3(ag), st, a, static_cast<uint8_t *>(layer), arg(k),
                           (const uint32_t *)(w.counters + k), (const uint32_t *)cur_list, hk, has_next, nxt,
                           w.counters + k + 1, next_list);
        else
            e = launch_pdl(k_sphere_step<uint16_t>, dim3(ag), st, a, static_cast<uint16_t *>(layer), arg(k),
                           (const uint32_t *)(w.counters + k), (const uint32_t *)cur_list, hk, has_next, nxt,
                           w.counters + k + 1, next_list);
    }
    count_launches(2 + n);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "lcl_select_sphere launch");
    return LCL_OK;
}

lcl_status select_lasso_impl(const lcl_atlas *atlas, void *layer, int dtype_bytes, const lcl_camera *cam,
                             const float *depth, const float *poly, int32_t nv, uint32_t label, float bias,
                             uint64_t *hits, void *ws, cudaStream_t st) {
    const AtlasDev a = dev_view(atlas);
    const SelWs w = sel_ws(atlas, 1, ws);
    unsigned long long *h = reinterpret_cast<unsigned long long *>(hits);
    static thread_local LassoArg p;  // ~2.8 KB: kept off the stack
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
    // Culling and the division-free reject use the bbox widened by a margin far above the FP32
    // rounding of projected points (well under a thousandth of a pixel at these sizes).
    const float margin = 2.0f + 1e-3f * (float)std::max(cam->width, cam->height);
    p.bx0 = std::fmax(x0, 0.0f) - margin;
    p.bx1 = std::fmin(x1, (float)cam->width) + margin;
    p.by0 = std::fmax(y0, 0.0f) - margin;
    p.by1 = std::fmin(y1, (float)cam->height) + margin;
    p.nx0 = (float)(2.0 * p.bx0 / cam->width - 1.0);
    p.nx1 = (float)(2.0 * p.bx1 / cam->width - 1.0);
    p.ny0 = (float)(2.0 * p.by0 / cam->height - 1.0);
    p.ny1 = (float)(2.0 * p.by1 / cam->height - 1.0);
    p.ymin = y0;
    p.ymax = y1;
    // y-bands of edges; each band lists the edges whose y-range comes within `slack` of it
    const double bh = std::max((double)y1 - (double)y0, 1e-3) / kBands;
    const double slack = 1e-3 * bh + 1e-3;
    p.band_y0 = y0;
    p.band_inv_h = (float)(1.0 / bh);
    int cnt = 0;
    for (int b = 0; b < kBands; ++b) {
        p.band_off[b] = (uint16_t)cnt;
        const double lo = (double)y0 + b * bh - slack, hi = (double)y0 + (b + 1) * bh + slack;
        for (int e = 0; e < nv; ++e) {
            const double ea = p.vy[e], eb = p.vy[e + 1];
            if (ea == eb) continue;  // horizontal edges never straddle
            if (std::min(ea, eb) <= hi && std::max(ea, eb) >= lo) p.band_edge[cnt++] = (uint8_t)e;
        }
    }
    p.band_off[kBands] = (uint16_t)cnt;
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
