// layers.cu -- whole-layer operations: boolean overlays and per-label surface area.
// Layer systems combine layers with logic operations (arXiv 2501.14807, Section 3.4.2) and
// measure what they hold (Section 5, Table 1 gives the area one texel stands for).
// Both are pure HBM streams over the texture:
//   k_overlay  16 bytes of each operand and of the output per thread step, coverage bits
//              expanded to byte / half-word masks in registers (SWAR), no shared memory
//   k_area4    four consecutive texels per lane and step, a contiguous range of steps per warp
//              (128 consecutive texels per warp and step, coalesced loads of triangle ids and
//              labels, the next step's issued ahead); the four weight gathers of a lane are
//              independent loads; texels carrying the warp's current label add to per-lane
//              sums in registers (a quad whose four labels are that label is recognised by one
//              compare of its label word), reduced across the warp only when another label appears;
//              the histogram lives in shared memory (64-bit shared atomics) and goes into the
//              outputs with one global atomic per non-zero bin per CTA.  All sums are
//              integers, so the result does not depend on the order.
#include <algorithm>
#include <type_traits>

#include "lcl_impl.cuh"

namespace lcl {
namespace {

constexpr uint32_t kSmemLabels = 2048;  // histograms up to this size live in shared memory

// Byte (or half-word) lanes of x that are non-zero -> all-ones lanes.
__device__ __forceinline__ uint32_t nonzero_lanes(uint32_t x, int bytes) {
    if (bytes == 1) {
        uint32_t t = ((x & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | x;
        return ((t & 0x80808080u) >> 7) * 0xFFu;
    }
    uint32_t t = ((x & 0x7FFF7FFFu) + 0x7FFF7FFFu) | x;
    return ((t & 0x80008000u) >> 15) * 0xFFFFu;
}

// Coverage bits of the lanes of one 32-bit word -> all-ones lanes.
__device__ __forceinline__ uint32_t cover_lanes(uint32_t bits, int bytes) {
    if (bytes == 1) return ((bits * 0x00204081u) & 0x01010101u) * 0xFFu;
    return ((bits & 1u) ? 0x0000FFFFu : 0u) | ((bits & 2u) ? 0xFFFF0000u : 0u);
}

__device__ __forceinline__ uint32_t overlay_word(uint32_t a, uint32_t b, uint32_t cov, int op, uint32_t flags,
                                                 int bytes) {
    if (flags & LCL_NOT_A) a = ~a;
    if (flags & LCL_NOT_B) b = ~b;
    uint32_t r;
    switch (op) {
    case LCL_AND: r = a & b; break;
    case LCL_OR: r = a | b; break;
    case LCL_XOR: r = a ^ b; break;
    default: r = a & nonzero_lanes(b, bytes); break;
    }
    if (flags & LCL_NOT_OUT) r = ~r;
    return r & cover_lanes(cov, bytes);
}

template <int BYTES>
__global__ void __launch_bounds__(kThreads) k_overlay(const uint32_t *__restrict__ a, const uint32_t *__restrict__ b,
                                                      uint32_t *__restrict__ out, const uint32_t *__restrict__ cover,
                                                      int64_t n_words, int op, uint32_t flags) {
    constexpr int kLanes = 4 / BYTES;  // texels per 32-bit word
    const int64_t n_vec = n_words / 4;
    const int64_t n_cover = (n_words * kLanes + 31) / 32;  // coverage words of the texture
    (void)n_cover;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n_vec; v += stride) {
        if (!LCL_IN(4 * v + 3, n_words) || !LCL_IN((v * 4 * kLanes) >> 5, n_cover)) continue;
        const uint4 A = __ldcs(reinterpret_cast<const uint4 *>(a) + v);
        const uint4 B = __ldcs(reinterpret_cast<const uint4 *>(b) + v);
        const int64_t t0 = v * 4 * kLanes;  // first texel of this 16-byte chunk
        const uint32_t cw = __ldg(cover + (t0 >> 5)) >> (t0 & 31);
        uint4 R;
        R.x = overlay_word(A.x, B.x, cw & ((1u << kLanes) - 1), op, flags, BYTES);
        R.y = overlay_word(A.y, B.y, (cw >> kLanes) & ((1u << kLanes) - 1), op, flags, BYTES);
        R.z = overlay_word(A.z, B.z, (cw >> (2 * kLanes)) & ((1u << kLanes) - 1), op, flags, BYTES);
        R.w = overlay_word(A.w, B.w, (cw >> (3 * kLanes)) & ((1u << kLanes) - 1), op, flags, BYTES);
        __stcs(reinterpret_cast<uint4 *>(out) + v, R);
    }
    // tail: the last n_words % 4 words
    const int64_t w = n_vec * 4 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (w < n_words && LCL_IN(w, n_words) && LCL_IN((w * kLanes) >> 5, n_cover)) {
        const int64_t t0 = w * kLanes;
        const uint32_t cw = (cover[t0 >> 5] >> (t0 & 31)) & ((1u << kLanes) - 1);
        out[w] = overlay_word(a[w], b[w], cw, op, flags, BYTES);
    }
}

__global__ void k_zero2(unsigned long long *x, unsigned long long *y, uint32_t n) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        x[i] = 0;
        y[i] = 0;
    }
}

// Sums of the warp's lanes: counts below 2^28 in all; a lane's area below 2^63 (at most 2^28 texels
// of weight below 2^35), cut into three 21-bit pieces whose sums over 32 lanes stay below 2^26, so
// four 32-bit warp reductions give the exact 64-bit sum.
__device__ __forceinline__ void warp_sums(uint32_t &c, unsigned long long &a) {
    c = __reduce_add_sync(0xffffffffu, c);
    const uint32_t a0 = __reduce_add_sync(0xffffffffu, (uint32_t)(a & 0x1FFFFFull));
    const uint32_t a1 = __reduce_add_sync(0xffffffffu, (uint32_t)((a >> 21) & 0x1FFFFFull));
    const uint32_t a2 = __reduce_add_sync(0xffffffffu, (uint32_t)(a >> 42));
    a = (unsigned long long)a0 + ((unsigned long long)a1 << 21) + ((unsigned long long)a2 << 42);
}

// Per-label area, four consecutive texels (a quad) per lane and step: a warp reads 128 consecutive
// texels per step, one 16-byte load of triangle ids and one 4- or 8-byte load of labels per lane.
// The four weight gathers of a lane are independent loads (a texel whose triangle is its left
// neighbour's reuses that weight), so they are in flight together.
// Texels carrying the warp's current label add to per-lane sums in registers; when a step holds
// other labels, the warp's sums are reduced into the histogram, the warp takes the label of the
// step's last such texel, and texels of any third label go to the histogram one by one.
template <typename L, bool SMEM>
__global__ void __launch_bounds__(kThreads, 5) k_area4(const L *__restrict__ layer, const uint32_t *__restrict__ tri,
                                                    const uint64_t *__restrict__ area_w, int64_t n_tri,
                                                    int64_t n_texels, uint32_t n_labels,
                                                    unsigned long long *__restrict__ count,
                                                    unsigned long long *__restrict__ area) {
    extern __shared__ unsigned long long sh[];
    unsigned long long *hc = SMEM ? sh : count;
    unsigned long long *ha = SMEM ? sh + n_labels : area;
    if (SMEM) {
        for (uint32_t i = threadIdx.x; i < 2 * n_labels; i += blockDim.x) sh[i] = 0;
        __syncthreads();
    }
    const unsigned long long *aw = reinterpret_cast<const unsigned long long *>(area_w);
    const int lane = threadIdx.x & 31;
    const int64_t n_quads = n_texels / 4;  // the width is a multiple of 4
    const int64_t n_steps = (n_quads + 31) / 32;
    const int64_t n_warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t per = (n_steps + n_warps - 1) / n_warps;
    const int64_t s0 = warp * per, s1 = min(n_steps, s0 + per);
    using LV = typename std::conditional<sizeof(L) == 1, uint32_t, uint2>::type;  // a lane's four labels
    // step s: quad 32 s + lane; the next step's loads are issued before this step is summed
    uint4 T = make_uint4(kNone, kNone, kNone, kNone);
    LV V{};
    auto load = [&](int64_t st) {
        const int64_t q = st * 32 + lane;
        T = make_uint4(kNone, kNone, kNone, kNone);
        if (q < n_quads && LCL_IN(4 * q + 3, n_texels)) {
            T = __ldcs(reinterpret_cast<const uint4 *>(tri) + q);
            V = __ldcs(reinterpret_cast<const LV *>(layer) + q);
        }
    };
    uint32_t wlabel = kNone, wcnt = 0;  // the warp's label; this lane's share of its count and area
    unsigned long long warea = 0;
    // a quad whose four labels are the warp's label matches wl4 (the label in every lane of a word);
    // wvalid is false until the warp has a label
    uint32_t wl4 = 0;
    bool wvalid = false;
    // tri ids are 32-bit and kNone = 0xFFFFFFFF is not below any 32-bit count, so one compare with
    // the count decides whether a texel is covered by a valid triangle
    const uint32_t ntri = n_tri < (int64_t)0xFFFFFFFFu ? (uint32_t)n_tri : 0xFFFFFFFFu;
    if (s0 < s1) load(s0);
    for (int64_t st = s0; st < s1; ++st) {
        const uint32_t ts[4] = {T.x, T.y, T.z, T.w};
        const LV Vc = V;
        if (st + 1 < s1) load(st + 1);
        unsigned long long w[4];
        bool vt[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            vt[k] = ts[k] < ntri;
            w[k] = (vt[k] && (k == 0 || ts[k] != ts[k - 1])) ? __ldg(aw + ts[k]) : 0ull;
        }
#pragma unroll
        for (int k = 1; k < 4; ++k)
            if (vt[k] && ts[k] == ts[k - 1]) w[k] = w[k - 1];
        bool same;
        if constexpr (sizeof(L) == 1) same = wvalid && Vc == wl4;
        else same = wvalid && Vc.x == wl4 && Vc.y == wl4;
        uint32_t odd = 0;
        uint32_t lab[4] = {0u, 0u, 0u, 0u};
        if (same) {  // every texel of the quad carries the warp's label (below n_labels): w is 0 off the mesh
            wcnt += (uint32_t)vt[0] + (uint32_t)vt[1] + (uint32_t)vt[2] + (uint32_t)vt[3];
            warea += (w[0] + w[1]) + (w[2] + w[3]);
        } else {
            if constexpr (sizeof(L) == 1) {
#pragma unroll
                for (int k = 0; k < 4; ++k) lab[k] = (Vc >> (8 * k)) & 0xFFu;
            } else {
                lab[0] = Vc.x & 0xFFFFu;
                lab[1] = Vc.x >> 16;
                lab[2] = Vc.y & 0xFFFFu;
                lab[3] = Vc.y >> 16;
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                if (!vt[k] || lab[k] >= n_labels) continue;
                if (lab[k] == wlabel) {
                    wcnt += 1;
                    warea += w[k];
                } else {
                    odd |= 1u << k;
                }
            }
        }
        const uint32_t bal = __ballot_sync(0xffffffffu, odd != 0);
        if (bal) {  // uniform over the warp
            uint32_t c = wcnt;
            unsigned long long a = warea;
            warp_sums(c, a);
            if (lane == 0 && c && LCL_IN(wlabel, n_labels)) {
                atomicAdd(hc + wlabel, (unsigned long long)c);
                atomicAdd(ha + wlabel, a);
            }
            uint32_t last = kNone;
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if (odd & (1u << k)) last = lab[k];
            wlabel = __shfl_sync(0xffffffffu, last, 31 - __clz(bal));
            wvalid = true;
            wl4 = sizeof(L) == 1 ? wlabel * 0x01010101u : wlabel * 0x00010001u;
            wcnt = 0;
            warea = 0;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                if (!(odd & (1u << k))) continue;
                if (lab[k] == wlabel) {
                    wcnt += 1;
                    warea += w[k];
                } else if (LCL_IN(lab[k], n_labels)) {
                    atomicAdd(hc + lab[k], 1ull);
                    atomicAdd(ha + lab[k], w[k]);
                }
            }
        }
    }
    {
        uint32_t c = wcnt;
        unsigned long long a = warea;
        warp_sums(c, a);
        if (lane == 0 && c && LCL_IN(wlabel, n_labels)) {
            atomicAdd(hc + wlabel, (unsigned long long)c);
            atomicAdd(ha + wlabel, a);
        }
    }
    if (SMEM) {
        __syncthreads();
        for (uint32_t i = threadIdx.x; i < n_labels; i += blockDim.x) {
            if (sh[i]) {
                atomicAdd(count + i, sh[i]);
                atomicAdd(area + i, sh[n_labels + i]);
            }
        }
    }
}

}  // namespace

lcl_status overlay_impl(const lcl_atlas *atlas, const void *a, const void *b, void *out, int dtype_bytes, int op,
                        uint32_t flags, cudaStream_t st) {
    const int64_t n_tex = (int64_t)atlas->width * atlas->height;
    const int64_t n_words = n_tex * dtype_bytes / 4;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(sm_count() * 8, (n_words / 4 + kThreads - 1) / kThreads));
    if (dtype_bytes == 1)
        k_overlay<1><<<grid, kThreads, 0, st>>>(static_cast<const uint32_t *>(a), static_cast<const uint32_t *>(b),
                                                static_cast<uint32_t *>(out), atlas->cover, n_words, op, flags);
    else
        k_overlay<2><<<grid, kThreads, 0, st>>>(static_cast<const uint32_t *>(a), static_cast<const uint32_t *>(b),
                                                static_cast<uint32_t *>(out), atlas->cover, n_words, op, flags);
    count_launches(1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "lcl_overlay launch");
    return LCL_OK;
}

lcl_status label_area_impl(const lcl_atlas *atlas, const void *layer, int dtype_bytes, uint32_t n_labels,
                           uint64_t *count, uint64_t *area, cudaStream_t st) {
    const int64_t n_tex = (int64_t)atlas->width * atlas->height;
    unsigned long long *c = reinterpret_cast<unsigned long long *>(count);
    unsigned long long *ar = reinterpret_cast<unsigned long long *>(area);
    k_zero2<<<std::max(1u, std::min(1024u, (n_labels + kThreads - 1) / kThreads)), kThreads, 0, st>>>(c, ar, n_labels);
    const bool smem = n_labels <= kSmemLabels;
    const size_t shb = smem ? 2 * (size_t)n_labels * sizeof(unsigned long long) : 0;
    // as many CTAs as fit at once (one wave), fewer for small textures
    auto fit = [&](auto kernel) {
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kThreads, shb) != cudaSuccess || per_sm < 1)
            per_sm = 1;
        return (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)sm_count() * per_sm,
                                                           (n_tex / 16 + kThreads - 1) / kThreads));
    };
    const uint32_t *tri = atlas->tri;
    if (dtype_bytes == 1) {
        const uint8_t *l = static_cast<const uint8_t *>(layer);
        if (smem) k_area4<uint8_t, true><<<fit(k_area4<uint8_t, true>), kThreads, shb, st>>>(l, tri, atlas->area_w, atlas->n_tri,
                                                                                          n_tex, n_labels, c, ar);
        else k_area4<uint8_t, false><<<fit(k_area4<uint8_t, false>), kThreads, 0, st>>>(l, tri, atlas->area_w, atlas->n_tri,
                                                                                      n_tex, n_labels, c, ar);
    } else {
        const uint16_t *l = static_cast<const uint16_t *>(layer);
        if (smem) k_area4<uint16_t, true><<<fit(k_area4<uint16_t, true>), kThreads, shb, st>>>(l, tri, atlas->area_w,
                                                                                            atlas->n_tri, n_tex,
                                                                                            n_labels, c, ar);
        else k_area4<uint16_t, false><<<fit(k_area4<uint16_t, false>), kThreads, 0, st>>>(l, tri, atlas->area_w, atlas->n_tri,
                                                                                        n_tex, n_labels, c, ar);
    }
    count_launches(2);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "lcl_label_area launch");
    return LCL_OK;
}

}  // namespace lcl
