// select_common.cuh -- device pieces shared by the single-stroke edits (select.cu) and the
// batched multi-model edits (batch.cu): stroke arguments, conservative box tests, the exact
// per-texel lasso test, label stores, candidate lists and launch helpers.  Not part of the ABI.
#pragma once

#include <algorithm>
#include <cmath>

#include "lcl_impl.cuh"

namespace lcl {

struct AtlasDev {
    const int32_t *px, *py, *pz;
    const uint32_t *cover;
    const int32_t *tile_box, *super_box;
    int32_t w, h, T, tiles_x, tiles_y, supers_x, supers_y;
    uint32_t tdiv_m, tdiv_s;  // tile index t -> tile row: (t tdiv_m) >> tdiv_s = t / tiles_x (tile_row)
};

// Multiplier and shift that divide every n < 2^24 exactly by d, 1 <= d <= 2^24, without a division
// (Granlund and Montgomery, "Division by invariant integers using multiplication", 1994, Thm 4.2):
// with l = ceil(log2 d) and m = ceil(2^(24+l) / d), m d = 2^(24+l) + e with 0 <= e < d <= 2^l, so
// n m / 2^(24+l) = n / d + n e / (d 2^(24+l)) and the second term is below 1/d for n < 2^24, which
// leaves the floor unchanged; m <= 2^25, so n m < 2^49.  Tile indices are below 2^22.
inline void tile_divisor(int32_t d, uint32_t *m, uint32_t *s) {
    int l = 0;
    while ((int64_t(1) << l) < d) ++l;
    *m = (uint32_t)(((uint64_t(1) << (24 + l)) + (uint64_t)d - 1) / (uint64_t)d);
    *s = (uint32_t)(24 + l);
}

inline AtlasDev dev_view(const lcl_atlas *a) {
    AtlasDev d;
    d.px = a->pos_x;
    d.py = a->pos_y;
    d.pz = a->pos_z;
    d.cover = a->cover;
    d.tile_box = a->tile_box;
    d.super_box = a->super_box;
    d.w = a->width;
    d.h = a->height;
    d.T = a->tile;
    d.tiles_x = a->tiles_x;
    d.tiles_y = a->tiles_y;
    d.supers_x = a->supers_x;
    d.supers_y = a->supers_y;
    tile_divisor(d.tiles_x > 0 ? d.tiles_x : 1, &d.tdiv_m, &d.tdiv_s);
    return d;
}

// Column and row of tile t (t < 2^24) of the atlas's tile grid.
__device__ __forceinline__ void tile_xy(const AtlasDev &a, uint32_t t, int32_t &tx, int32_t &ty) {
    ty = (int32_t)(((uint64_t)t * a.tdiv_m) >> a.tdiv_s);
    tx = (int32_t)t - ty * a.tiles_x;
}

struct SphereArg {
    int64_t cx, cy, cz, r2;
    uint32_t label;
    int32_t pad_r, pad_t;  // texture padding: kernel radius and outline thickness (0: no padding)
};



__device__ __forceinline__ int64_t box_dist2(int4 lo, int4 hi, const SphereArg &s) {
    int64_t ex = max(max((int64_t)lo.x - s.cx, s.cx - (int64_t)hi.x), (int64_t)0);
    int64_t ey = max(max((int64_t)lo.y - s.cy, s.cy - (int64_t)hi.y), (int64_t)0);
    int64_t ez = max(max((int64_t)lo.z - s.cz, s.cz - (int64_t)hi.z), (int64_t)0);
    return ex * ex + ey * ey + ez * ez;
}

// Squared distance from the sphere's centre to the box's farthest point: at most r2 means the sphere
// contains the whole box.
__device__ __forceinline__ int64_t box_far2(int4 lo, int4 hi, const SphereArg &s) {
    const int64_t fx = max(s.cx - (int64_t)lo.x, (int64_t)hi.x - s.cx);
    const int64_t fy = max(s.cy - (int64_t)lo.y, (int64_t)hi.y - s.cy);
    const int64_t fz = max(s.cz - (int64_t)lo.z, (int64_t)hi.z - s.cz);
    return fx * fx + fy * fy + fz * fz;
}

// Any box of the 3 x 3 neighbourhood of (bx, by) in a grid of nx x ny boxes within the sphere's
// reach (used when padding may write texels next to the selected ones).
__device__ __forceinline__ bool near_box_3x3(const int32_t *boxes, int32_t nx, int32_t ny, int32_t bx, int32_t by,
                                             const SphereArg &s) {
    bool any = false;
    for (int32_t y = max(by - 1, 0); y <= min(by + 1, ny - 1); ++y)
        for (int32_t x = max(bx - 1, 0); x <= min(bx + 1, nx - 1); ++x) {
            if (!LCL_IN((int64_t)y * nx + x, (int64_t)nx * ny)) continue;
            const int4 *b = reinterpret_cast<const int4 *>(boxes + 8 * ((int64_t)y * nx + x));
            const int4 lo = b[0], hi = b[1];
            any |= lo.w > 0 && box_dist2(lo, hi, s) <= s.r2;
        }
    return any;
}

// Appends this lane's tile to the candidate list (room for `cap` entries) if `cand`; one atomic
// per warp.
__device__ __forceinline__ void append_candidate(bool cand, uint32_t tile, uint32_t *counter, uint32_t *list,
                                                 int64_t cap) {
    uint32_t m = __ballot_sync(0xffffffffu, cand);
    if (!m) return;
    const int lane = threadIdx.x & 31;
    uint32_t base = 0;
    if (lane == __ffs(m) - 1) base = atomicAdd(counter, (uint32_t)__popc(m));
    base = __shfl_sync(0xffffffffu, base, __ffs(m) - 1);
    const uint32_t slot = base + __popc(m & ((1u << lane) - 1));
    if (cand && LCL_IN(slot, cap)) list[slot] = tile;
    (void)cap;
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

// Appends this lane's tile to the back of the list (slots cap - 1, cap - 2, ... counted by `counter`)
// if `cand`; one atomic per warp.  A list filled from both ends holds at most cap entries in all.
__device__ __forceinline__ void append_candidate_back(bool cand, uint32_t tile, uint32_t *counter, uint32_t *list,
                                                      int64_t cap) {
    uint32_t m = __ballot_sync(0xffffffffu, cand);
    if (!m) return;
    const int lane = threadIdx.x & 31;
    uint32_t base = 0;
    if (lane == __ffs(m) - 1) base = atomicAdd(counter, (uint32_t)__popc(m));
    base = __shfl_sync(0xffffffffu, base, __ffs(m) - 1);
    const int64_t slot = cap - 1 - (int64_t)(base + __popc(m & ((1u << lane) - 1)));
    if (cand && LCL_IN(slot, cap)) list[slot] = tile;
}

// Writes `label` into the covered texels (bits of `cov`) of the 32 texels starting at l (l a
// multiple of 32, the layer 16-byte aligned): 16-byte stores, read first only where some texel of
// the 16 bytes is not written.
template <typename L>
__device__ __forceinline__ void store_word32(L *layer, int64_t l, uint32_t cov, uint32_t label) {
    constexpr int kPer = 16 / (int)sizeof(L);  // texels per 16-byte store
    const uint32_t rep = sizeof(L) == 1 ? label * 0x01010101u : sizeof(L) == 2 ? label * 0x00010001u : label;
    uint4 *p = reinterpret_cast<uint4 *>(layer + l);
#pragma unroll
    for (int g = 0; g < 32 / kPer; ++g) {
        const uint32_t bits = (cov >> (g * kPer)) & (kPer == 32 ? 0xFFFFFFFFu : ((1u << kPer) - 1u));
        if (!bits) continue;
        if (bits == ((1u << kPer) - 1u)) {
            p[g] = make_uint4(rep, rep, rep, rep);
            continue;
        }
        uint32_t wm[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (sizeof(L) == 1) wm[j] = (((bits >> (4 * j)) & 0xFu) * 0x00204081u & 0x01010101u) * 0xFFu;
            else if (sizeof(L) == 2) wm[j] = (((bits >> (2 * j)) & 1u) ? 0x0000FFFFu : 0u) | (((bits >> (2 * j)) & 2u) ? 0xFFFF0000u : 0u);
            else wm[j] = ((bits >> j) & 1u) ? 0xFFFFFFFFu : 0u;
        }
        const uint4 o = p[g];
        p[g] = make_uint4((o.x & ~wm[0]) | (rep & wm[0]), (o.y & ~wm[1]) | (rep & wm[1]), (o.z & ~wm[2]) | (rep & wm[2]),
                          (o.w & ~wm[3]) | (rep & wm[3]));
    }
}

// Programmatic dependent launch: wait for the previous grid on the stream to complete (its
// memory is then visible); let the next grid be scheduled.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_allow_next() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }


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

template <>
__device__ __forceinline__ void store_hits<uint32_t>(uint32_t *layer, int64_t l, uint32_t m, uint32_t value) {
    if (m == 0xFu) {
        *reinterpret_cast<uint4 *>(layer + l) = make_uint4(value, value, value, value);
        return;
    }
#pragma unroll
    for (int k = 0; k < 4; ++k)
        if (m & (1u << k)) layer[l + k] = value;
}

// Mask texture of a numeric layer (Section 4.2): one bit per texel, bit (y * width + x) of a linear
// uint32 array like the coverage bits.  An edit sets the bits of the texels it writes (or clears
// them when it erases).
struct ValMask {
    uint32_t *bits;
    uint32_t set;  // 1: set the written texels' bits, 0: clear them
};

// Updates the mask bits of one quad (bits m at texel l, l a multiple of 4) with one atomic; the
// mask has a bit for each of n_tex texels.
__device__ __forceinline__ void valid_update_atomic(const ValMask &vm, int64_t l, uint32_t m, int64_t n_tex) {
    const uint32_t b = m << (l & 31);
    if (!LCL_IN(l >> 5, (n_tex + 31) >> 5)) return;
    if (vm.set) atomicOr(vm.bits + (l >> 5), b);
    else atomicAnd(vm.bits + (l >> 5), ~b);
    (void)n_tex;
}

// Updates the mask bits of the quads of a whole warp; every lane calls it (l < 0: no quad).
// GROUPED: the eight lanes 8g..8g+7 hold the 32 texels of one mask word, all of them or none (a
// tile side of at least 32 and a width that is a multiple of 32); their bits are merged with three
// shuffles and the word is written by its first lane, which owns it during the launch (one edit
// per launch), so no atomic is needed.  Otherwise each quad updates its bits with one atomic.
template <bool GROUPED>
__device__ __forceinline__ void valid_update_warp(const ValMask &vm, int64_t l, uint32_t m, int64_t n_tex) {
    if (GROUPED) {
        uint32_t b = (l >= 0) ? (m << (l & 31)) : 0u;
        b |= __shfl_xor_sync(0xffffffffu, b, 1);
        b |= __shfl_xor_sync(0xffffffffu, b, 2);
        b |= __shfl_xor_sync(0xffffffffu, b, 4);
        if ((threadIdx.x & 7u) == 0 && l >= 0 && b && LCL_IN(l >> 5, (n_tex + 31) >> 5)) {
            uint32_t *p = vm.bits + (l >> 5);
            if (vm.set) *p = (b == 0xFFFFFFFFu) ? b : (*p | b);
            else *p = (b == 0xFFFFFFFFu) ? 0u : (*p & ~b);
        }
    } else if (l >= 0 && m) {
        valid_update_atomic(vm, l, m, n_tex);
    }
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


template <typename... K, typename... A>
cudaError_t launch_pdl_shape(void (*kernel)(K...), dim3 grid, dim3 block, cudaStream_t st, A... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// Programmatic dependent launch of `kernel` with kThreads threads per CTA.
template <typename... K, typename... A>
cudaError_t launch_pdl(void (*kernel)(K...), dim3 grid, cudaStream_t st, A... args) {
    return launch_pdl_shape(kernel, grid, dim3(kThreads), st, args...);
}


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

// A CTA's copy of the polygon and its bands, plus one record per edge e (vertex e to e + 1):
// {ay, by, lo, hi}, lo and hi its x-range widened by the margin of edge_xrange.
struct LassoShared {
    float4 rec[LCL_MAX_LASSO_VERTICES];
    float vx[LCL_MAX_LASSO_VERTICES + 1], vy[LCL_MAX_LASSO_VERTICES + 1];
    uint16_t band_off[kBands + 1];
    uint8_t band_edge[kBandEdgesMax];
};

// The crossing x of the even-odd rule, xi = ((bx - ax)(ys - ay)) / (by - ay) + ax in FP32, lies
// within [min(ax, bx) - d, max(ax, bx) + d] with d = 4.01 u (|ax| + |bx|), u = 2^-24, whenever ys
// lies between ay and by: (ys - ay) / (by - ay) is then in [0, 1] and each of the five roundings
// adds at most u.  A point left or right of that range by more than m = 1e-6 (|ax| + |bx| + 1)
// >= 16 u (|ax| + |bx| + 1) (which also covers the roundings of the bounds) takes the same
// decision as the division.  Returns the widened range {lo, hi}.
__device__ __forceinline__ float2 edge_xrange(float ax, float bx) {
    const float m = __fmul_rn(1e-6f, __fadd_rn(__fadd_rn(fabsf(ax), fabsf(bx)), 1.0f));
    return make_float2(__fsub_rn(fminf(ax, bx), m), __fadd_rn(fmaxf(ax, bx), m));
}

// Whether (xs, ys), with ys between ay and by, lies left of edge e's crossing (the definition's
// `xs < xi`); the division runs only inside the widened x-range [lo, hi].
__device__ __forceinline__ bool edge_left(const float *__restrict__ vx, int e, float xs, float ys, float ay, float by,
                                          float lo, float hi) {
    if (xs < lo) return true;
    if (xs > hi) return false;
    const float ax = vx[e], bx = vx[e + 1];
    const float xi = __fadd_rn(div_rn(__fmul_rn(__fsub_rn(bx, ax), __fsub_rn(ys, ay)), __fsub_rn(by, ay)), ax);
    return xs < xi;
}

// Copies the polygon and its bands into shared memory and builds the edge records (one CTA).
__device__ __forceinline__ void stage_lasso(LassoShared &sh, const LassoArg &p) {
    for (int e = threadIdx.x; e <= p.nv; e += blockDim.x) {
        sh.vx[e] = p.vx[e];
        sh.vy[e] = p.vy[e];
        if (e < p.nv) {
            const float2 r = edge_xrange(p.vx[e], p.vx[e + 1]);
            sh.rec[e] = make_float4(p.vy[e], p.vy[e + 1], r.x, r.y);
        }
    }
    for (int k = threadIdx.x; k <= kBands; k += blockDim.x) sh.band_off[k] = p.band_off[k];
    for (int k = threadIdx.x; k < p.band_off[kBands]; k += blockDim.x) sh.band_edge[k] = p.band_edge[k];
}

// Conservative: false only if no texel of the box can be selected by the lasso.  Two exact tests:
//  - the box's projected corners (all with w > 0) bound the projection of every point of the box
//    (a projective map keeps a convex box convex); if their bounding box, widened by the margin,
//    misses the polygon's widened bounding box, no texel can be inside the polygon;
//  - with a depth map: NDC depth z/w is linear-fractional along every segment of the box, so its
//    minimum over the box is at a corner; if that minimum (less 1e-4 for FP32 rounding) exceeds
//    the largest depth-map value over the box's widened pixel footprint plus the bias, every texel
//    of the box fails the depth test.  Footprints above 1024 pixels are not scanned (kept).
// sbox (optional): as for box_may_touch8.
__device__ inline bool box_may_touch(const LassoArg &p, int4 lo, int4 hi, const float *__restrict__ depth = nullptr,
                                     float4 *sbox = nullptr) {
    float xmin = INFINITY, xmax = -INFINITY, ymin = INFINITY, ymax = -INFINITY, zmin = INFINITY;
    bool finite = true;
    if (sbox) *sbox = make_float4(NAN, NAN, NAN, NAN);
#pragma unroll 1
    for (int c = 0; c < 8; ++c) {
        float x = (float)((c & 1) ? hi.x : lo.x), y = (float)((c & 2) ? hi.y : lo.y), z = (float)((c & 4) ? hi.z : lo.z);
        float cw = clip_row(p.m + 12, x, y, z);
        if (!(cw > 0.0f)) return true;
        float xs = screen_of(div_rn(clip_row(p.m, x, y, z), cw), p.ws);
        float ys = screen_of(div_rn(clip_row(p.m + 4, x, y, z), cw), p.hs);
        finite = finite && isfinite(xs) && isfinite(ys);
        float zn = div_rn(clip_row(p.m + 8, x, y, z), cw);
        xmin = fminf(xmin, xs); xmax = fmaxf(xmax, xs);
        ymin = fminf(ymin, ys); ymax = fmaxf(ymax, ys);
        zmin = fminf(zmin, zn);
    }
    if (xmax < p.bx0 || xmin > p.bx1 || ymax < p.by0 || ymin > p.by1) return false;
    if (sbox && finite) *sbox = make_float4(xmin, xmax, ymin, ymax);
    if (!depth) return true;
    const float margin = 2.0f;
    const int ix0 = max(0, __float2int_rd(xmin - margin)), ix1 = min(p.w_s - 1, __float2int_rd(xmax + margin));
    const int iy0 = max(0, __float2int_rd(ymin - margin)), iy1 = min(p.h_s - 1, __float2int_rd(ymax + margin));
    if (ix0 > ix1 || iy0 > iy1) return false;  // the whole footprint is off screen
    if ((ix1 - ix0 + 1) * (iy1 - iy0 + 1) > 1024) return true;
    float dmax = -INFINITY;
    for (int iy = iy0; iy <= iy1; ++iy)
        for (int ix = ix0; ix <= ix1; ++ix)
            if (LCL_IN((int64_t)iy * p.w_s + ix, (int64_t)p.w_s * p.h_s))
                dmax = fmaxf(dmax, __ldg(depth + (int64_t)iy * p.w_s + ix));
    return !(zmin - 1e-4f > dmax + p.bias);
}


// box_may_touch evaluated by an aligned group of 8 lanes for one box (all 8 call it with the same
// box): lane c projects corner c, the group reduces the screen box and the nearest depth, and the
// depth-footprint scan is split by rows over the group.  The tests of box_may_touch, with
// footprints of up to 2048 px scanned (1024 there) before the test gives up and keeps the box.
// sbox (optional): the screen box {xmin, xmax, ymin, ymax} of the projected corners when every
// corner lies in front of the camera and projects to finite coordinates, else NaNs.
// Tile classes for a lasso (the texels of a box projected to screen box `sb`, by box_may_touch8).
enum : int { kTileOut = 0, kTileTest = 1, kTileIn = 2 };

template <int LANES>
__device__ __forceinline__ int lasso_tile_class8(const LassoArg &p, const float *vx, const float *vy, float4 sb);

// CLASSIFY (with vx, vy, *cls): between the screen-box test and the depth-footprint scan, the tile is
// classified by lasso_tile_class8 (its class in *cls, kTileTest where it cannot be); a tile outside the
// polygon returns false at once, without the scan.
template <bool CLASSIFY = false>
__device__ __forceinline__ bool box_may_touch8(const LassoArg &p, int4 lo, int4 hi, const float *__restrict__ depth,
                                               float4 *sbox = nullptr, const float *vx = nullptr,
                                               const float *vy = nullptr, int *cls = nullptr) {
    const unsigned lane = threadIdx.x & 31u, sub = lane & 7u;
    const unsigned gm = 0xFFu << (lane & 24u);
    const float x = (float)((sub & 1u) ? hi.x : lo.x), y = (float)((sub & 2u) ? hi.y : lo.y);
    const float z = (float)((sub & 4u) ? hi.z : lo.z);
    const float cw = clip_row(p.m + 12, x, y, z);
    if (sbox) *sbox = make_float4(NAN, NAN, NAN, NAN);
    if (__any_sync(gm, !(cw > 0.0f))) return true;
    // each lane folds its corner into empty bounds exactly as the serial loop does (NaN ignored)
    const float xs = screen_of(div_rn(clip_row(p.m, x, y, z), cw), p.ws);
    const float ys = screen_of(div_rn(clip_row(p.m + 4, x, y, z), cw), p.hs);
    const bool finite = __all_sync(gm, isfinite(xs) && isfinite(ys));
    float xmin = fminf(INFINITY, xs), xmax = fmaxf(-INFINITY, xs);
    float ymin = fminf(INFINITY, ys), ymax = fmaxf(-INFINITY, ys);
    float zmin = fminf(INFINITY, div_rn(clip_row(p.m + 8, x, y, z), cw));
    for (int o = 1; o < 8; o <<= 1) {
        xmin = fminf(xmin, __shfl_xor_sync(gm, xmin, o));
        xmax = fmaxf(xmax, __shfl_xor_sync(gm, xmax, o));
        ymin = fminf(ymin, __shfl_xor_sync(gm, ymin, o));
        ymax = fmaxf(ymax, __shfl_xor_sync(gm, ymax, o));
        zmin = fminf(zmin, __shfl_xor_sync(gm, zmin, o));
    }
    if (xmax < p.bx0 || xmin > p.bx1 || ymax < p.by0 || ymin > p.by1) return false;
    if (sbox && finite) *sbox = make_float4(xmin, xmax, ymin, ymax);
    if (CLASSIFY) {
        *cls = finite ? lasso_tile_class8<8>(p, vx, vy, make_float4(xmin, xmax, ymin, ymax)) : kTileTest;
        if (*cls == kTileOut) return false;  // outside the polygon: no texel can be selected
    }
    if (!depth) return true;
    const float margin = 2.0f;
    const int ix0 = max(0, __float2int_rd(xmin - margin)), ix1 = min(p.w_s - 1, __float2int_rd(xmax + margin));
    const int iy0 = max(0, __float2int_rd(ymin - margin)), iy1 = min(p.h_s - 1, __float2int_rd(ymax + margin));
    if (ix0 > ix1 || iy0 > iy1) return false;  // the whole footprint is off screen
    if ((ix1 - ix0 + 1) * (iy1 - iy0 + 1) > 2048) return true;
    float dmax = -INFINITY;
    for (int iy = iy0 + (int)sub; iy <= iy1; iy += 8)
        for (int ix = ix0; ix <= ix1; ++ix)
            if (LCL_IN((int64_t)iy * p.w_s + ix, (int64_t)p.w_s * p.h_s))
                dmax = fmaxf(dmax, __ldg(depth + (int64_t)iy * p.w_s + ix));
    for (int o = 1; o < 8; o <<= 1) dmax = fmaxf(dmax, __shfl_xor_sync(gm, dmax, o));
    return !(zmin - 1e-4f > dmax + p.bias);
}


// Classifies a box whose projection lies in the screen box sb, by the aligned group of 8 lanes of
// box_may_touch8 (all 8 call it; lane c takes edges c, c + 8, ...):
//   kTileOut   no edge of the polygon comes near the box and its centre is outside: no texel of the
//              box is inside (the tile is dropped);
//   kTileIn    no edge comes near the box, its centre is inside and the box lies on screen: every
//              texel of the box that projects is inside, so the texels skip the edge tests;
//   kTileTest  otherwise (every texel is tested).
// Why this is exact for the per-texel test in FP32: each texel's FP32 screen point lies in sb up to
// far less than the margin m = 1 px (a few ulps of coordinates below 2^15), and no edge segment meets
// sb widened by m, so along any straddled edge the crossing lies more than m - 0.05 px from the point,
// beyond the error bound of the FP32 crossing (edge_xrange's 4.01 u (|ax| + |bx|) < 0.01 px); every
// per-texel edge decision is then the exact one at that point, and the exact even-odd parity is the
// same at every point of a region no edge meets -- the parity at the centre.  The segment-box test is
// conservative: an FP32 side value whose magnitude is within its error bound counts as meeting.
// vx, vy: the polygon's vertices (vertex nv = vertex 0), staged in shared memory by the caller so
// that the lanes' different edges are not serialised on the parameter bank.  LANES: 8 (an aligned
// group of 8 lanes shares the work, as after box_may_touch8) or 1 (one thread does it alone).
template <int LANES>
__device__ __forceinline__ int lasso_tile_class8(const LassoArg &p, const float *vx, const float *vy, float4 sb) {
    const unsigned lane = threadIdx.x & 31u, sub = LANES == 8 ? (lane & 7u) : 0u;
    const unsigned gm = 0xFFu << (lane & 24u);
    if (!(isfinite(sb.x) && isfinite(sb.y) && isfinite(sb.z) && isfinite(sb.w))) return kTileTest;  // uniform
    const float m = 1.0f;
    const float x0 = sb.x - m, x1 = sb.y + m, y0 = sb.z - m, y1 = sb.w + m;
    const float cx = __fmul_rn(0.5f, __fadd_rn(sb.x, sb.y)), cy = __fmul_rn(0.5f, __fadd_rn(sb.z, sb.w));
    const float u5 = 5.0f * 5.9604645e-8f;  // 5 u, u = 2^-24
    bool meets = false, parity = false;
    for (int e = (int)sub; e < p.nv; e += LANES) {
        const float ax = vx[e], ay = vy[e], bx = vx[e + 1], by = vy[e + 1];
        if (!(fmaxf(ax, bx) < x0 || fminf(ax, bx) > x1 || fmaxf(ay, by) < y0 || fminf(ay, by) > y1)) {
            const float dx = __fsub_rn(bx, ax), dy = __fsub_rn(by, ay);
            bool pos = false, neg = false;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const float X = (c & 1) ? x1 : x0, Y = (c & 2) ? y1 : y0;
                const float a1 = __fmul_rn(dx, __fsub_rn(Y, ay)), a2 = __fmul_rn(dy, __fsub_rn(X, ax));
                const float side = __fsub_rn(a1, a2), err = __fmul_rn(u5, __fadd_rn(fabsf(a1), fabsf(a2)));
                if (side > err) pos = true;
                else if (side < -err) neg = true;
                else pos = neg = true;
            }
            meets = meets || (pos && neg);
        }
        if ((ay > cy) != (by > cy)) {  // the definition's crossing test at the centre
            const float xi = __fadd_rn(div_rn(__fmul_rn(__fsub_rn(bx, ax), __fsub_rn(cy, ay)), __fsub_rn(by, ay)), ax);
            if (cx < xi) parity = !parity;
        }
    }
    uint32_t bits = (meets ? 1u : 0u) | (parity ? 2u : 0u);
    for (int o = 1; o < LANES; o <<= 1) {
        const uint32_t t = __shfl_xor_sync(gm, bits, o);
        bits = (bits | (t & 1u)) ^ (t & 2u);
    }
    (void)gm;
    if (bits & 1u) return kTileTest;
    if (!(bits & 2u)) return kTileOut;
    const bool on_screen = x0 >= 0.0f && x1 < p.ws && y0 >= 0.0f && y1 < p.hs;
    return on_screen ? kTileIn : kTileTest;
}

// Decisions on the correctly rounded quotient q = RN(a / b), b > 0, made exactly without dividing
// when a product says enough (the correctly rounded division runs only in the narrow band left):
//   q >= 0:  a >= 0 gives a / b >= 0; a < 0 takes the division (a quotient that underflows to -0
//            passes);
//   q <= t:  e = RN(a - t b) (one rounding, an FMA) has the sign of a - t b, so e < 0 means a / b < t
//            and then q <= t (rounding is monotone and t is a float).  For t, b and t b normal, e above
//            RN(t b) 2^-20 means a / b > t + t 2^-21 > t + ulp(t) / 2, beyond the rounding boundary
//            above t, so q > t.  Otherwise (e near 0, or an operand too small or not finite) the
//            quotient is computed.
__device__ __forceinline__ bool quot_ge0(float a, float b) { return a >= 0.0f || div_rn(a, b) >= 0.0f; }

__device__ __forceinline__ bool quot_le(float a, float b, float t) {
    const float e = __fmaf_rn(-t, b, a);
    if (e < 0.0f) return true;
    const float tb = __fmul_rn(t, b);
    if (t >= 0x1p-126f && b >= 0x1p-126f && tb >= 0x1p-100f && tb <= 0x1p100f && e > __fmul_rn(tb, 0x1p-20f))
        return false;
    return div_rn(a, b) <= t;
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
// INSIDE: the texel's tile is known to lie inside the polygon (lasso_tile_class8): the edge tests,
// whose outcome would be "inside", are skipped.
template <bool INSIDE = false, typename Edges>
__device__ __forceinline__ bool lasso_hit(const LassoArg &p, const Edges &sh, const float *__restrict__ depth,
                                          int32_t X, int32_t Y, int32_t Z) {
    if (X == INT32_MIN) return false;  // uncovered
    const float fx = (float)X, fy = (float)Y, fz = (float)Z;
    const float cw = clip_row(p.m + 12, fx, fy, fz);
    if (!(cw > 0.0f)) return false;
    const float cx = clip_row(p.m, fx, fy, fz);
    if (cx < __fmul_rn(p.nx0, cw) || cx > __fmul_rn(p.nx1, cw)) return false;
    const float cy = clip_row(p.m + 4, fx, fy, fz);
    if (cy < __fmul_rn(p.ny0, cw) || cy > __fmul_rn(p.ny1, cw)) return false;
    const float xs = screen_of(div_rn(cx, cw), p.ws);
    const float ys = screen_of(div_rn(cy, cw), p.hs);
    if (!(xs >= 0.0f && xs < p.ws && ys >= 0.0f && ys < p.hs)) return false;
    if (!(ys >= p.ymin && ys < p.ymax)) return false;  // no edge straddles y
    int band = __float2int_rz(__fmul_rn(__fsub_rn(ys, p.band_y0), p.band_inv_h));
    band = band < 0 ? 0 : (band >= kBands ? kBands - 1 : band);
    bool inside = INSIDE;
    for (int k = sh.band_off[band]; !INSIDE && k < sh.band_off[band + 1]; ++k) {
        if (!LCL_IN(k, kBandEdgesMax)) break;
        const int e = sh.band_edge[k];
        if (!LCL_IN(e, LCL_MAX_LASSO_VERTICES)) continue;
        const float ax = sh.vx[e], ay = sh.vy[e], bx = sh.vx[e + 1], by = sh.vy[e + 1];
        if ((ay > ys) != (by > ys)) {
            const float2 r = edge_xrange(ax, bx);
            if (edge_left(sh.vx, e, xs, ys, ay, by, r.x, r.y)) inside = !inside;
        }
    }
    if (!inside) return false;
    // NDC depth zn = RN(cz / cw) in [0, 1] and zn <= depth + bias, decided as quot_* describes
    const float cz = clip_row(p.m + 8, fx, fy, fz);
    if (!(quot_ge0(cz, cw) && quot_le(cz, cw, 1.0f))) return false;
    const int32_t ix = __float2int_rz(xs), iy = __float2int_rz(ys);
    if (!LCL_IN((int64_t)iy * p.w_s + ix, (int64_t)p.w_s * p.h_s)) return false;
    const float d = __ldg(depth + (int64_t)iy * p.w_s + ix);
    return quot_le(cz, cw, __fadd_rn(d, p.bias));
}


// The depth test (Fig. 3a) of the texels `live` of a quad that passed the other steps: NDC depth in
// [0, 1] and z <= depth[floor(ys)][floor(xs)] + bias.
__device__ __forceinline__ uint32_t lasso_depth_quad(const LassoArg &p, const float *__restrict__ depth,
                                                     const int32_t (&xq)[4], const int32_t (&yq)[4],
                                                     const int32_t (&zq)[4], const float (&xs)[4],
                                                     const float (&ys)[4], const float (&cw)[4], uint32_t live) {
    uint32_t m = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        if (!(live & (1u << k))) continue;
        const float cz = clip_row(p.m + 8, (float)xq[k], (float)yq[k], (float)zq[k]);
        if (!(quot_ge0(cz, cw[k]) && quot_le(cz, cw[k], 1.0f))) continue;
        const int32_t ix = __float2int_rz(xs[k]), iy = __float2int_rz(ys[k]);
        if (!LCL_IN((int64_t)iy * p.w_s + ix, (int64_t)p.w_s * p.h_s)) continue;
        const float d = __ldg(depth + (int64_t)iy * p.w_s + ix);
        if (quot_le(cz, cw[k], __fadd_rn(d, p.bias))) m |= 1u << k;
    }
    return m;
}

// Candidate-list entry bit of a tile whose projecting texels all lie inside the lasso polygon.
constexpr uint32_t kInsideTile = 0x80000000u;

// lasso_hit for the four texels of a quad (bit k: texel k).  Each texel takes the steps of
// lasso_hit up to its band; when the quad's live texels share a band (nearly always: they are
// neighbours on the surface) one pass over that band's edge records tests all of them.  Texels
// that failed a step carry ys = NaN, which straddles no edge.  INSIDE: the quad's tile is known to
// lie inside the polygon (lasso_tile_class8), so the edge tests are skipped: their outcome for
// every texel that reaches them is "inside".
template <bool INSIDE>
__device__ __forceinline__ uint32_t lasso_quad(const LassoArg &p, const LassoShared &sh,
                                               const float *__restrict__ depth, int4 X, int4 Y, int4 Z) {
    const int32_t xq[4] = {X.x, X.y, X.z, X.w}, yq[4] = {Y.x, Y.y, Y.z, Y.w}, zq[4] = {Z.x, Z.y, Z.z, Z.w};
    float xs[4], ys[4], cw[4];
    int band[4];
    uint32_t live = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        xs[k] = 0.0f;
        ys[k] = __int_as_float(0x7fc00000);
        cw[k] = 1.0f;
        band[k] = -1;
        if (xq[k] == INT32_MIN) continue;  // uncovered
        const float fx = (float)xq[k], fy = (float)yq[k], fz = (float)zq[k];
        const float w = clip_row(p.m + 12, fx, fy, fz);
        if (!(w > 0.0f)) continue;
        const float cx = clip_row(p.m, fx, fy, fz);
        if (!INSIDE && (cx < __fmul_rn(p.nx0, w) || cx > __fmul_rn(p.nx1, w))) continue;
        const float cy = clip_row(p.m + 4, fx, fy, fz);
        if (!INSIDE && (cy < __fmul_rn(p.ny0, w) || cy > __fmul_rn(p.ny1, w))) continue;
        const float x = screen_of(div_rn(cx, w), p.ws);
        const float y = screen_of(div_rn(cy, w), p.hs);
        // INSIDE: the tile's class already settles the viewport, the polygon's box and its y-range
        // (the projected box widened by the margin lies on screen and inside the polygon)
        if (!INSIDE && !(x >= 0.0f && x < p.ws && y >= 0.0f && y < p.hs)) continue;
        if (!INSIDE && !(y >= p.ymin && y < p.ymax)) continue;
        int b = 0;
        if (!INSIDE) {
            b = __float2int_rz(__fmul_rn(__fsub_rn(y, p.band_y0), p.band_inv_h));
            b = b < 0 ? 0 : (b >= kBands ? kBands - 1 : b);
        }
        xs[k] = x;
        ys[k] = y;
        cw[k] = w;
        band[k] = b;
        live |= 1u << k;
    }
    if (!live) return 0;
    if (INSIDE) return lasso_depth_quad(p, depth, xq, yq, zq, xs, ys, cw, live);
    const int b0 = (live & 1u) ? band[0] : (live & 2u) ? band[1] : (live & 4u) ? band[2] : band[3];
    bool same = true;
#pragma unroll
    for (int k = 0; k < 4; ++k) same = same && (band[k] < 0 || band[k] == b0);
    uint32_t inside = 0;
    if (same) {
        for (int j = sh.band_off[b0]; j < sh.band_off[b0 + 1]; ++j) {
            if (!LCL_IN(j, kBandEdgesMax)) break;
            const int e = sh.band_edge[j];
            if (!LCL_IN(e, LCL_MAX_LASSO_VERTICES)) continue;
            const float4 r = sh.rec[e];
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if ((r.x > ys[k]) != (r.y > ys[k]) && edge_left(sh.vx, e, xs[k], ys[k], r.x, r.y, r.z, r.w))
                    inside ^= 1u << k;
        }
    } else {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (band[k] < 0) continue;
            for (int j = sh.band_off[band[k]]; j < sh.band_off[band[k] + 1]; ++j) {
                if (!LCL_IN(j, kBandEdgesMax)) break;
                const int e = sh.band_edge[j];
                if (!LCL_IN(e, LCL_MAX_LASSO_VERTICES)) continue;
                const float4 r = sh.rec[e];
                if ((r.x > ys[k]) != (r.y > ys[k]) && edge_left(sh.vx, e, xs[k], ys[k], r.x, r.y, r.z, r.w))
                    inside ^= 1u << k;
            }
        }
    }
    return lasso_depth_quad(p, depth, xq, yq, zq, xs, ys, cw, live & inside);
}


// The paper's editing tool (Section 4.3.1): window and shape, with the FP32 constants of the
// tool-space map precomputed on the host (each from double, rounded once).
struct ToolArg {
    float px, py;    // tool position (window centre), pixels
    float kx, ky;    // 2 / tw, 2 / th (inscribed circle)
    float x0, y0;    // window corner px - tw/2, py - th/2
    float su, sv;    // shape texels per pixel
    float fw, fh;    // shape size as float
    const uint8_t *shape;  // null: inscribed circle
    int32_t sw, sh;
    int32_t pad_r, pad_t;  // texture padding: kernel radius and outline thickness (0: no padding)
};

// Tool test of one texel: projection, viewport and depth test as for lassos (the window's
// bounding box, widened, in p's division-free reject), then the shape (MASK) or the circle.
template <bool MASK>
__device__ __forceinline__ bool tool_hit(const LassoArg &p, const ToolArg &t, const float *__restrict__ depth,
                                         int32_t X, int32_t Y, int32_t Z) {
    if (X == INT32_MIN) return false;  // uncovered
    const float fx = (float)X, fy = (float)Y, fz = (float)Z;
    const float cw = clip_row(p.m + 12, fx, fy, fz);
    if (!(cw > 0.0f)) return false;
    const float cx = clip_row(p.m, fx, fy, fz);
    if (cx < __fmul_rn(p.nx0, cw) || cx > __fmul_rn(p.nx1, cw)) return false;
    const float cy = clip_row(p.m + 4, fx, fy, fz);
    if (cy < __fmul_rn(p.ny0, cw) || cy > __fmul_rn(p.ny1, cw)) return false;
    const float xs = screen_of(div_rn(cx, cw), p.ws);
    const float ys = screen_of(div_rn(cy, cw), p.hs);
    if (!(xs >= 0.0f && xs < p.ws && ys >= 0.0f && ys < p.hs)) return false;
    if (MASK) {
        const float fu = __fmul_rn(__fsub_rn(xs, t.x0), t.su), fv = __fmul_rn(__fsub_rn(ys, t.y0), t.sv);
        if (!(fu >= 0.0f && fu < t.fw && fv >= 0.0f && fv < t.fh)) return false;
        const int64_t si = (int64_t)__float2int_rz(fv) * t.sw + __float2int_rz(fu);
        if (!LCL_IN(si, (int64_t)t.sw * t.sh)) return false;
        if (__ldg(t.shape + si) == 0) return false;
    } else {
        const float ex = __fmul_rn(__fsub_rn(xs, t.px), t.kx), ey = __fmul_rn(__fsub_rn(ys, t.py), t.ky);
        if (!(__fadd_rn(__fmul_rn(ex, ex), __fmul_rn(ey, ey)) <= 1.0f)) return false;
    }
    const float cz = clip_row(p.m + 8, fx, fy, fz);  // zn = RN(cz / cw), decided as quot_* describes
    if (!(quot_ge0(cz, cw) && quot_le(cz, cw, 1.0f))) return false;
    const int32_t ix = __float2int_rz(xs), iy = __float2int_rz(ys);
    if (!LCL_IN((int64_t)iy * p.w_s + ix, (int64_t)p.w_s * p.h_s)) return false;
    const float d = __ldg(depth + (int64_t)iy * p.w_s + ix);
    return quot_le(cz, cw, __fadd_rn(d, p.bias));
}

// CTAs of `threads` threads that fit on one SM at once (at least 1).
template <typename K>
inline int resident_per_sm(K kernel, int threads) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    return per_sm;
}

// A grid of as many CTAs as fit on the GPU at once (persistent loops need no second wave).
template <typename K>
inline int resident_grid(K kernel) {
    return resident_per_sm(kernel, kThreads) * sm_count();
}


// y-bands of edges: band b lists the edges whose y-range comes within `slack` of it, in edge order.
__host__ __device__ inline double lasso_band_height(const LassoArg &p) {
    return fmax((double)p.ymax - (double)p.ymin, 1e-3) / kBands;
}

// The lasso argument without its y-bands: matrix, screen, polygon (vertex nv repeated as vertex
// 0), the widened bounding box in pixels and NDC, the band mapping.  Host and device run the same
// code (batched edits build their lassos on the device), so both get identical fields.
__host__ __device__ inline void lasso_arg_head(LassoArg &p, const float *m16, int32_t w_s, int32_t h_s,
                                               const float *poly, int32_t nv, uint32_t label, float bias) {
    for (int i = 0; i < 16; ++i) p.m[i] = m16[i];
    p.ws = (float)w_s;
    p.hs = (float)h_s;
    p.w_s = w_s;
    p.h_s = h_s;
    p.bias = bias;
    p.label = label;
    p.nv = nv;
    float x0 = INFINITY, x1 = -INFINITY, y0 = INFINITY, y1 = -INFINITY;
    for (int i = 0; i < nv; ++i) {
        p.vx[i] = poly[2 * i];
        p.vy[i] = poly[2 * i + 1];
        x0 = fminf(x0, p.vx[i]);
        x1 = fmaxf(x1, p.vx[i]);
        y0 = fminf(y0, p.vy[i]);
        y1 = fmaxf(y1, p.vy[i]);
    }
    for (int i = nv; i <= LCL_MAX_LASSO_VERTICES; ++i) {
        p.vx[i] = p.vx[0];
        p.vy[i] = p.vy[0];
    }
    // Culling and the division-free reject use the bbox widened by a margin far above the FP32
    // rounding of projected points (well under a thousandth of a pixel at these sizes).
    const float margin = 2.0f + 1e-3f * (float)(w_s > h_s ? w_s : h_s);
    p.bx0 = fmaxf(x0, 0.0f) - margin;
    p.bx1 = fminf(x1, (float)w_s) + margin;
    p.by0 = fmaxf(y0, 0.0f) - margin;
    p.by1 = fminf(y1, (float)h_s) + margin;
    p.nx0 = (float)(2.0 * p.bx0 / w_s - 1.0);
    p.nx1 = (float)(2.0 * p.bx1 / w_s - 1.0);
    p.ny0 = (float)(2.0 * p.by0 / h_s - 1.0);
    p.ny1 = (float)(2.0 * p.by1 / h_s - 1.0);
    p.ymin = y0;
    p.ymax = y1;
    p.band_y0 = y0;
    p.band_inv_h = (float)(1.0 / lasso_band_height(p));
}

__host__ __device__ inline bool lasso_band_has(const LassoArg &p, int b, int e, double bh) {
    const double slack = 1e-3 * bh + 1e-3;
    const double lo = (double)p.ymin + b * bh - slack, hi = (double)p.ymin + (b + 1) * bh + slack;
    const double ea = p.vy[e], eb = p.vy[e + 1];
    if (ea == eb) return false;  // horizontal edges never straddle
    return fmin(ea, eb) <= hi && fmax(ea, eb) >= lo;
}

// The whole lasso argument, on the host.
inline void fill_lasso_arg(LassoArg &p, const lcl_camera *cam, const float *poly, int32_t nv, uint32_t label,
                           float bias) {
    lasso_arg_head(p, cam->m, cam->width, cam->height, poly, nv, label, bias);
    const double bh = lasso_band_height(p);
    int cnt = 0;
    for (int b = 0; b < kBands; ++b) {
        p.band_off[b] = (uint16_t)cnt;
        for (int e = 0; e < nv; ++e)
            if (lasso_band_has(p, b, e, bh)) p.band_edge[cnt++] = (uint8_t)e;
    }
    p.band_off[kBands] = (uint16_t)cnt;
}

// Tool argument and the culling argument (the window as a 4-vertex polygon) from a tool.
inline void fill_tool_arg(ToolArg &t, LassoArg &p, const lcl_camera *cam, const lcl_tool *tool, uint32_t label,
                          float bias) {
    const double px = tool->px, py = tool->py, tw = tool->tw, th = tool->th;
    t.px = tool->px;
    t.py = tool->py;
    t.kx = (float)(2.0 / tw);
    t.ky = (float)(2.0 / th);
    t.x0 = (float)(px - 0.5 * tw);
    t.y0 = (float)(py - 0.5 * th);
    t.shape = tool->shape;
    t.sw = tool->shape ? tool->shape_w : 0;
    t.sh = tool->shape ? tool->shape_h : 0;
    t.su = tool->shape ? (float)((double)tool->shape_w / tw) : 0.0f;
    t.sv = tool->shape ? (float)((double)tool->shape_h / th) : 0.0f;
    t.fw = (float)t.sw;
    t.fh = (float)t.sh;
    t.pad_r = (int32_t)(tool->flags & 15u);
    t.pad_t = (int32_t)((tool->flags >> 4) & 15u);
    // the window's corners, widened by a pixel so rounding of x0 + tw cannot cut it
    const float win[8] = {(float)(px - 0.5 * tw - 1.0), (float)(py - 0.5 * th - 1.0),
                          (float)(px + 0.5 * tw + 1.0), (float)(py - 0.5 * th - 1.0),
                          (float)(px + 0.5 * tw + 1.0), (float)(py + 0.5 * th + 1.0),
                          (float)(px - 0.5 * tw - 1.0), (float)(py + 0.5 * th + 1.0)};
    fill_lasso_arg(p, cam, win, 4, label, bias);
}

}  // namespace lcl
