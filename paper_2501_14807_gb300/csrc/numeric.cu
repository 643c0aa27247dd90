// numeric.cu -- numeric layers (arXiv 2501.14807, Section 4.2): a data texture of 8/16/32-bit
// integers or 16/32-bit floats plus a mask texture (here one bit per texel).  Whole-layer
// operations, all HBM streams over the texture:
//   k_num_arith   arithmetic overlay a <op> b (or a <op> scalar): each lane takes a 16-byte chunk of
//                 data (warp-contiguous), the mask bits of its texels come from the word shared by
//                 the 2, 4 or 8 lanes of its group, and the group's output word is merged with
//                 shuffles and written by its first lane
//   k_num_select  selection by value into a label layer (the lane owns its texels' label bytes)
//   k_num_stats   zonal statistics: a warp takes 512 texels per step (lane l: texels 4l + 128k),
//                 runs of equal zone labels are accumulated in registers and flushed into a
//                 shared-memory table (or the output, for many zones); min / max through
//                 order-preserving 64-bit keys, sums in double
#include <algorithm>
#include <type_traits>

#include <cuda_fp16.h>

#include "lcl_impl.cuh"

namespace lcl {
namespace {

constexpr int kKindUnsigned = 1, kKindSigned = 2, kKindFloat = 3;
constexpr uint32_t kSmemZones = 1024;  // zone tables up to this size live in shared memory (48 KB)

template <int S>
__device__ __forceinline__ uint32_t width_mask() {
    return S == 4 ? 0xFFFFFFFFu : ((1u << (8 * S)) - 1u);
}

template <int S>
__device__ __forceinline__ int32_t sext(uint32_t v) {
    if (S == 1) return (int32_t)(int8_t)(uint8_t)v;
    if (S == 2) return (int32_t)(int16_t)(uint16_t)v;
    return (int32_t)v;
}

template <int S>
__device__ __forceinline__ float to_float(uint32_t v) {
    if (S == 2) return __half2float(__ushort_as_half((unsigned short)v));
    return __uint_as_float(v);
}

template <int S>
__device__ __forceinline__ uint32_t from_float(float f) {
    if (S == 2) return (uint32_t)__half_as_ushort(__float2half_rn(f));
    return __float_as_uint(f);
}

// One arithmetic operation on the bits of two values of the type (S bytes, KIND).
template <int S, int KIND>
__device__ __forceinline__ uint32_t arith(uint32_t a, uint32_t b, int op) {
    if (KIND == kKindFloat) {
        const float x = to_float<S>(a), y = to_float<S>(b);
        float r;
        switch (op) {
        case LCL_ADD: r = __fadd_rn(x, y); break;
        case LCL_SUB: r = __fsub_rn(x, y); break;
        case LCL_MUL: r = __fmul_rn(x, y); break;
        case LCL_DIV: r = __fdiv_rn(x, y); break;
        case LCL_MIN: r = x < y ? x : y; break;
        default: r = x > y ? x : y; break;
        }
        return from_float<S>(r);
    }
    uint32_t r;
    switch (op) {
    case LCL_ADD: r = a + b; break;
    case LCL_SUB: r = a - b; break;
    case LCL_MUL: r = a * b; break;
    case LCL_MIN: r = (KIND == kKindSigned ? sext<S>(a) < sext<S>(b) : a < b) ? a : b; break;
    default: r = (KIND == kKindSigned ? sext<S>(a) > sext<S>(b) : a > b) ? a : b; break;
    }
    return r & width_mask<S>();
}

// Element k of a 16-byte chunk of S-byte values.
template <int S>
__device__ __forceinline__ uint32_t elem(const uint32_t (&w)[4], int k) {
    if (S == 4) return w[k];
    if (S == 2) return (w[k >> 1] >> (16 * (k & 1))) & 0xFFFFu;
    return (w[k >> 2] >> (8 * (k & 3))) & 0xFFu;
}

template <int S>
__device__ __forceinline__ void set_elem(uint32_t (&w)[4], int k, uint32_t v) {
    if (S == 4) {
        w[k] = v;
    } else if (S == 2) {
        const int sh = 16 * (k & 1);
        w[k >> 1] = (w[k >> 1] & ~(0xFFFFu << sh)) | (v << sh);
    } else {
        const int sh = 8 * (k & 3);
        w[k >> 2] = (w[k >> 2] & ~(0xFFu << sh)) | (v << sh);
    }
}

struct ArithArgs {
    const uint4 *a, *b;
    uint4 *out;
    const uint32_t *ma, *mb, *cover;
    uint32_t *mout;
    uint32_t b_value;
    int op;
    int64_t n_chunks;  // 16-byte chunks over whole mask words: (n_texels / 32) * 32 texels
    int64_t n_texels;
};

// Texels of one lane's chunk: 16 / S, starting at texel c * (16 / S), inside mask word
// (c * (16 / S)) / 32 at bit (c * (16 / S)) % 32; 2S consecutive lanes share that word.
template <int S, int KIND>
__global__ void __launch_bounds__(kThreads) k_num_arith(ArithArgs p) {
    constexpr int kPer = 16 / S;
    constexpr int kGroup = 32 / kPer;  // lanes per mask word
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    // whole warps iterate together (the group merge uses shuffles over the full warp)
    const int64_t n_iter = (p.n_chunks + 31) & ~int64_t(31);
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c - (threadIdx.x & 31) < n_iter; c += stride) {
        const bool live = c < p.n_chunks;
        uint32_t bits = 0;
        int64_t t0 = c * kPer;
        if (live) {
            const uint4 A = __ldcs(p.a + c);
            uint4 B;
            if (p.b) B = __ldcs(p.b + c);
            const uint32_t word = (uint32_t)(t0 >> 5);
            const int off = (int)(t0 & 31);
            uint32_t valid = __ldg(p.ma + word) & __ldg(p.cover + word);
            if (p.b) valid &= __ldg(p.mb + word);
            valid = (valid >> off) & (kPer == 32 ? 0xFFFFFFFFu : ((1u << kPer) - 1u));
            const uint32_t aw[4] = {A.x, A.y, A.z, A.w};
            uint32_t bw[4] = {0u, 0u, 0u, 0u};
            if (p.b) {
                bw[0] = B.x;
                bw[1] = B.y;
                bw[2] = B.z;
                bw[3] = B.w;
            }
            uint32_t rw[4] = {0u, 0u, 0u, 0u};
#pragma unroll
            for (int k = 0; k < kPer; ++k) {
                const uint32_t bv = p.b ? elem<S>(bw, k) : p.b_value;
                const uint32_t r = (valid >> k) & 1u ? arith<S, KIND>(elem<S>(aw, k), bv, p.op) : 0u;
                set_elem<S>(rw, k, r);
            }
            __stcs(p.out + c, make_uint4(rw[0], rw[1], rw[2], rw[3]));
            bits = valid << off;
        }
#pragma unroll
        for (int o = 1; o < kGroup; o <<= 1) bits |= __shfl_xor_sync(0xffffffffu, bits, o);
        if (live && (threadIdx.x & (kGroup - 1)) == 0) p.mout[t0 >> 5] = bits;
    }
    // the last n_texels % 32 texels (one partial mask word), by the grid's first thread
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const int64_t t_begin = (p.n_texels >> 5) << 5;
        if (t_begin < p.n_texels) {
            const uint32_t word = (uint32_t)(t_begin >> 5);
            uint32_t valid = p.ma[word] & p.cover[word];
            if (p.b) valid &= p.mb[word];
            uint32_t bits = 0;
            for (int64_t t = t_begin; t < p.n_texels; ++t) {
                const int k = (int)(t - t_begin);
                uint32_t av, bv = p.b_value;
                if (S == 1) {
                    av = reinterpret_cast<const uint8_t *>(p.a)[t];
                    if (p.b) bv = reinterpret_cast<const uint8_t *>(p.b)[t];
                } else if (S == 2) {
                    av = reinterpret_cast<const uint16_t *>(p.a)[t];
                    if (p.b) bv = reinterpret_cast<const uint16_t *>(p.b)[t];
                } else {
                    av = reinterpret_cast<const uint32_t *>(p.a)[t];
                    if (p.b) bv = reinterpret_cast<const uint32_t *>(p.b)[t];
                }
                const bool v = (valid >> k) & 1u;
                const uint32_t r = v ? arith<S, KIND>(av, bv, p.op) : 0u;
                if (S == 1) reinterpret_cast<uint8_t *>(p.out)[t] = (uint8_t)r;
                else if (S == 2) reinterpret_cast<uint16_t *>(p.out)[t] = (uint16_t)r;
                else reinterpret_cast<uint32_t *>(p.out)[t] = r;
                bits |= (v ? 1u : 0u) << k;
            }
            p.mout[word] = bits;
        }
    }
}

// ---- selection by value ----------------------------------------------------------------------

template <int S, int KIND>
__device__ __forceinline__ bool compare(uint32_t v, uint32_t t, int cmp) {
    if (KIND == kKindFloat) {
        const float x = to_float<S>(v), y = to_float<S>(t);
        switch (cmp) {
        case LCL_LT: return x < y;
        case LCL_LE: return x <= y;
        case LCL_GT: return x > y;
        case LCL_GE: return x >= y;
        case LCL_EQ: return x == y;
        default: return x != y;
        }
    }
    if (KIND == kKindSigned) {
        const int32_t x = sext<S>(v), y = sext<S>(t);
        switch (cmp) {
        case LCL_LT: return x < y;
        case LCL_LE: return x <= y;
        case LCL_GT: return x > y;
        case LCL_GE: return x >= y;
        case LCL_EQ: return x == y;
        default: return x != y;
        }
    }
    switch (cmp) {
    case LCL_LT: return v < t;
    case LCL_LE: return v <= t;
    case LCL_GT: return v > t;
    case LCL_GE: return v >= t;
    case LCL_EQ: return v == t;
    default: return v != t;
    }
}

struct SelectArgs {
    const uint4 *data;
    const uint32_t *mask, *cover;
    void *layer;
    uint32_t threshold, label;
    int cmp;
    int64_t n_chunks;  // whole 16-byte chunks
    int64_t n_texels;
    unsigned long long *hits;
};

// Writes `label` (LB bytes) into the texels t0 .. t0 + n - 1 whose bit is set in `sel`.
template <int LB>
__device__ __forceinline__ void store_labels(void *layer, int64_t t0, int n, uint32_t sel, uint32_t label) {
    if (!sel) return;
    if (LB == 1) {
        uint8_t *l = static_cast<uint8_t *>(layer) + t0;
        for (int w = 0; w < n; w += 4) {  // t0 and n are multiples of 4
            const uint32_t m4 = (sel >> w) & 0xFu;
            if (!m4) continue;
            uint32_t *p = reinterpret_cast<uint32_t *>(l + w);
            uint32_t bm = ((m4 * 0x00204081u) & 0x01010101u) * 0xFFu;
            const uint32_t rep = label * 0x01010101u;
            *p = m4 == 0xFu ? rep : ((*p & ~bm) | (rep & bm));
        }
    } else {
        uint16_t *l = static_cast<uint16_t *>(layer) + t0;
        for (int w = 0; w < n; w += 2) {
            const uint32_t m2 = (sel >> w) & 0x3u;
            if (!m2) continue;
            uint32_t *p = reinterpret_cast<uint32_t *>(l + w);
            const uint32_t bm = ((m2 & 1u) ? 0x0000FFFFu : 0u) | ((m2 & 2u) ? 0xFFFF0000u : 0u);
            const uint32_t rep = label * 0x00010001u;
            *p = m2 == 0x3u ? rep : ((*p & ~bm) | (rep & bm));
        }
    }
}

template <int S, int KIND, int LB>
__global__ void __launch_bounds__(kThreads) k_num_select(SelectArgs p) {
    constexpr int kPer = 16 / S;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    uint32_t cnt = 0;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < p.n_chunks; c += stride) {
        const uint4 D = __ldcs(p.data + c);
        const int64_t t0 = c * kPer;
        const uint32_t word = (uint32_t)(t0 >> 5);
        const uint32_t valid = ((__ldg(p.mask + word) & __ldg(p.cover + word)) >> (t0 & 31)) &
                               (kPer == 32 ? 0xFFFFFFFFu : ((1u << kPer) - 1u));
        if (!valid) continue;
        const uint32_t dw[4] = {D.x, D.y, D.z, D.w};
        uint32_t sel = 0;
#pragma unroll
        for (int k = 0; k < kPer; ++k)
            if ((valid >> k) & 1u) sel |= (compare<S, KIND>(elem<S>(dw, k), p.threshold, p.cmp) ? 1u : 0u) << k;
        store_labels<LB>(p.layer, t0, kPer, sel, p.label);
        cnt += __popc(sel);
    }
    // tail texels after the whole chunks (fewer than 16 / S), by the grid's first thread
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        for (int64_t t = p.n_chunks * kPer; t < p.n_texels; ++t) {
            const uint32_t word = (uint32_t)(t >> 5);
            if (!(((p.mask[word] & p.cover[word]) >> (t & 31)) & 1u)) continue;
            uint32_t v;
            if (S == 1) v = reinterpret_cast<const uint8_t *>(p.data)[t];
            else if (S == 2) v = reinterpret_cast<const uint16_t *>(p.data)[t];
            else v = reinterpret_cast<const uint32_t *>(p.data)[t];
            if (!compare<S, KIND>(v, p.threshold, p.cmp)) continue;
            if (LB == 1) static_cast<uint8_t *>(p.layer)[t] = (uint8_t)p.label;
            else static_cast<uint16_t *>(p.layer)[t] = (uint16_t)p.label;
            ++cnt;
        }
    }
    if (p.hits) {
        for (int o = 16; o; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
        if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(p.hits, (unsigned long long)cnt);
    }
}

// ---- zonal statistics ------------------------------------------------------------------------

// Order-preserving 64-bit key of a double (atomicMin / atomicMax on doubles).
__device__ __forceinline__ unsigned long long dkey(double v) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(v);
    return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}
__device__ __forceinline__ double key_double(unsigned long long k) {
    return __longlong_as_double((long long)((k >> 63) ? (k & 0x7FFFFFFFFFFFFFFFull) : ~k));
}

// Accumulator layout of one zone while the kernel runs (same 48 bytes as lcl_zone_stats, with
// order-preserving keys in place of vmin / vmax).
struct ZoneAcc {
    unsigned long long count, area, kmin, kmax;
    double sum, wsum;
};
static_assert(sizeof(ZoneAcc) == sizeof(lcl_zone_stats), "zone accumulator must alias lcl_zone_stats");

__global__ void k_stats_init(ZoneAcc *z, uint32_t n) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        z[i].count = 0;
        z[i].area = 0;
        z[i].kmin = ~0ull;
        z[i].kmax = 0;
        z[i].sum = 0.0;
        z[i].wsum = 0.0;
    }
}

__global__ void k_stats_final(ZoneAcc *z, uint32_t n) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        lcl_zone_stats *o = reinterpret_cast<lcl_zone_stats *>(z + i);
        const unsigned long long kmin = z[i].kmin, kmax = z[i].kmax;
        const bool empty = z[i].count == 0;
        o->vmin = empty ? __longlong_as_double(0x7FF0000000000000ll) : key_double(kmin);
        o->vmax = empty ? __longlong_as_double((long long)0xFFF0000000000000ull) : key_double(kmax);
    }
}

struct StatsRun {
    uint32_t zone;
    uint32_t cnt;
    unsigned long long area;
    double vmin, vmax, sum, wsum;
};

__device__ __forceinline__ void flush_run(const StatsRun &r, ZoneAcc *tab) {
    if (r.cnt == 0) return;
    ZoneAcc *z = tab + r.zone;
    atomicAdd(&z->count, (unsigned long long)r.cnt);
    atomicAdd(&z->area, r.area);
    atomicMin(&z->kmin, dkey(r.vmin));
    atomicMax(&z->kmax, dkey(r.vmax));
    atomicAdd(&z->sum, r.sum);
    atomicAdd(&z->wsum, r.wsum);
}

struct StatsArgs {
    const void *data;
    const uint32_t *mask, *cover, *tri;
    const unsigned long long *area_w;
    const void *zones;  // NULL: one zone
    uint32_t n_labels;
    int64_t n_texels;
    ZoneAcc *out;
};

template <int S, int KIND>
__device__ __forceinline__ double value_of(uint32_t bits) {
    if (KIND == kKindFloat) return (double)to_float<S>(bits);
    if (KIND == kKindSigned) return (double)sext<S>(bits);
    return (double)bits;
}

// Four consecutive S-byte values starting at texel t (t a multiple of 4).
template <int S>
__device__ __forceinline__ void load4(const void *data, int64_t t, uint32_t (&v)[4]) {
    if (S == 1) {
        const uint32_t w = __ldcs(reinterpret_cast<const unsigned int *>(static_cast<const uint8_t *>(data) + t));
        for (int k = 0; k < 4; ++k) v[k] = (w >> (8 * k)) & 0xFFu;
    } else if (S == 2) {
        const uint2 w = __ldcs(reinterpret_cast<const uint2 *>(static_cast<const uint16_t *>(data) + t));
        v[0] = w.x & 0xFFFFu;
        v[1] = w.x >> 16;
        v[2] = w.y & 0xFFFFu;
        v[3] = w.y >> 16;
    } else {
        const uint4 w = __ldcs(reinterpret_cast<const uint4 *>(static_cast<const uint32_t *>(data) + t));
        v[0] = w.x;
        v[1] = w.y;
        v[2] = w.z;
        v[3] = w.w;
    }
}

template <int S, int KIND, int ZB, bool SMEM>
__global__ void __launch_bounds__(kThreads) k_num_stats(StatsArgs p) {
    extern __shared__ ZoneAcc sh_zone[];
    ZoneAcc *tab = SMEM ? sh_zone : p.out;
    if (SMEM) {
        for (uint32_t i = threadIdx.x; i < p.n_labels; i += blockDim.x) {
            sh_zone[i].count = 0;
            sh_zone[i].area = 0;
            sh_zone[i].kmin = ~0ull;
            sh_zone[i].kmax = 0;
            sh_zone[i].sum = 0.0;
            sh_zone[i].wsum = 0.0;
        }
        __syncthreads();
    }
    StatsRun run;
    run.zone = 0;
    run.cnt = 0;
    uint32_t last_t = kNone;
    unsigned long long last_w = 0;
    auto visit = [&](uint32_t z, uint32_t t, uint32_t bits, bool valid) {
        if (!valid || t == kNone || z >= p.n_labels) return;
        double v = value_of<S, KIND>(bits);
        if (v != v) return;  // NaN
        if (v == 0.0) v = 0.0;
        if (t != last_t) {
            last_t = t;
            last_w = __ldg(p.area_w + t);
        }
        const double wv = __dmul_rn((double)last_w, v);
        if (z != run.zone || run.cnt == 0) {
            flush_run(run, tab);
            run.zone = z;
            run.cnt = 0;
            run.area = 0;
            run.vmin = v;
            run.vmax = v;
            run.sum = 0.0;
            run.wsum = 0.0;
        }
        run.cnt += 1;
        run.area += last_w;
        run.vmin = v < run.vmin ? v : run.vmin;
        run.vmax = v > run.vmax ? v : run.vmax;
        run.sum = __dadd_rn(run.sum, v);
        run.wsum = __dadd_rn(run.wsum, wv);
    };
    // a warp takes 512 texels per step: lane l holds texels 4l + 128k .. + 3, k = 0..3
    constexpr int64_t kChunk = 512;
    const int lane = threadIdx.x & 31;
    const int64_t gthread = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t n_warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t n_chunks = p.n_texels / kChunk;
    for (int64_t c = gthread >> 5; c < n_chunks; c += n_warps) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int64_t t = c * kChunk + 128 * k + 4 * lane;
            const uint4 T = __ldcs(reinterpret_cast<const uint4 *>(p.tri + t));
            uint32_t v[4];
            load4<S>(p.data, t, v);
            uint32_t z[4] = {0u, 0u, 0u, 0u};
            if (p.zones) {
                if (ZB == 1) {
                    const uint32_t w = __ldcs(reinterpret_cast<const unsigned int *>(static_cast<const uint8_t *>(p.zones) + t));
                    for (int j = 0; j < 4; ++j) z[j] = (w >> (8 * j)) & 0xFFu;
                } else {
                    const uint2 w = __ldcs(reinterpret_cast<const uint2 *>(static_cast<const uint16_t *>(p.zones) + t));
                    z[0] = w.x & 0xFFFFu;
                    z[1] = w.x >> 16;
                    z[2] = w.y & 0xFFFFu;
                    z[3] = w.y >> 16;
                }
            }
            const uint32_t word = (uint32_t)(t >> 5);
            const uint32_t valid = ((__ldg(p.mask + word) & __ldg(p.cover + word)) >> (t & 31)) & 0xFu;
            visit(z[0], T.x, v[0], valid & 1u);
            visit(z[1], T.y, v[1], valid & 2u);
            visit(z[2], T.z, v[2], valid & 4u);
            visit(z[3], T.w, v[3], valid & 8u);
        }
    }
    // tail texels (n_texels % 512), one per thread
    for (int64_t t = n_chunks * kChunk + gthread; t < p.n_texels; t += (int64_t)gridDim.x * blockDim.x) {
        uint32_t bits, z = 0;
        if (S == 1) bits = static_cast<const uint8_t *>(p.data)[t];
        else if (S == 2) bits = static_cast<const uint16_t *>(p.data)[t];
        else bits = static_cast<const uint32_t *>(p.data)[t];
        if (p.zones) z = ZB == 1 ? static_cast<const uint8_t *>(p.zones)[t] : static_cast<const uint16_t *>(p.zones)[t];
        const uint32_t word = (uint32_t)(t >> 5);
        const bool valid = ((p.mask[word] & p.cover[word]) >> (t & 31)) & 1u;
        visit(z, p.tri[t], bits, valid);
    }
    flush_run(run, tab);
    if (SMEM) {
        __syncthreads();
        for (uint32_t i = threadIdx.x; i < p.n_labels; i += blockDim.x) {
            const ZoneAcc &a = sh_zone[i];
            if (a.count == 0) continue;
            ZoneAcc *o = p.out + i;
            atomicAdd(&o->count, a.count);
            atomicAdd(&o->area, a.area);
            atomicMin(&o->kmin, a.kmin);
            atomicMax(&o->kmax, a.kmax);
            atomicAdd(&o->sum, a.sum);
            atomicAdd(&o->wsum, a.wsum);
        }
    }
}

int stream_grid(int64_t work, int per_thread_units) {
    const int64_t threads = (work + per_thread_units - 1) / per_thread_units;
    return (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)sm_count() * 8, (threads + kThreads - 1) / kThreads));
}

template <int S, int KIND>
void launch_arith(const ArithArgs &p, cudaStream_t st) {
    k_num_arith<S, KIND><<<stream_grid(std::max<int64_t>(p.n_chunks, 1), 1), kThreads, 0, st>>>(p);
}

template <int S, int KIND, int LB>
void launch_select(const SelectArgs &p, cudaStream_t st) {
    k_num_select<S, KIND, LB><<<stream_grid(std::max<int64_t>(p.n_chunks, 1), 1), kThreads, 0, st>>>(p);
}

template <int S, int KIND, int ZB, bool SMEM>
void launch_stats_smem(const StatsArgs &p, size_t shb, cudaStream_t st) {
    auto kernel = k_num_stats<S, KIND, ZB, SMEM>;
    if (SMEM && shb > 48 * 1024) cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shb);
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kThreads, shb) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    const int64_t warps = p.n_texels / 512 + 1;
    const int grid = (int)std::max<int64_t>(
        1, std::min<int64_t>((int64_t)sm_count() * per_sm, (warps + kThreads / 32 - 1) / (kThreads / 32)));
    kernel<<<grid, kThreads, shb, st>>>(p);
}

template <int S, int KIND, int ZB>
void launch_stats(const StatsArgs &p, cudaStream_t st) {
    if (p.n_labels <= kSmemZones)
        launch_stats_smem<S, KIND, ZB, true>(p, (size_t)p.n_labels * sizeof(ZoneAcc), st);
    else
        launch_stats_smem<S, KIND, ZB, false>(p, 0, st);
}

template <int S, int KIND>
void launch_stats_z(const StatsArgs &p, int zb, cudaStream_t st) {
    if (zb == 2) launch_stats<S, KIND, 2>(p, st);
    else launch_stats<S, KIND, 1>(p, st);
}

}  // namespace

lcl_status numeric_arith_impl(const lcl_atlas *atlas, int type, const void *a, const uint32_t *ma, const void *b,
                              const uint32_t *mb, uint32_t b_value, void *out, uint32_t *mout, int op,
                              cudaStream_t st) {
    ArithArgs p;
    p.a = static_cast<const uint4 *>(a);
    p.b = static_cast<const uint4 *>(b);
    p.out = static_cast<uint4 *>(out);
    p.ma = ma;
    p.mb = mb;
    p.cover = atlas->cover;
    p.mout = mout;
    p.b_value = b_value;
    p.op = op;
    p.n_texels = (int64_t)atlas->width * atlas->height;
    const int bytes = type & 15;
    p.n_chunks = ((p.n_texels >> 5) << 5) * bytes / 16;
    switch (type) {
    case LCL_NUM_U8: launch_arith<1, kKindUnsigned>(p, st); break;
    case LCL_NUM_I8: launch_arith<1, kKindSigned>(p, st); break;
    case LCL_NUM_U16: launch_arith<2, kKindUnsigned>(p, st); break;
    case LCL_NUM_I16: launch_arith<2, kKindSigned>(p, st); break;
    case LCL_NUM_U32: launch_arith<4, kKindUnsigned>(p, st); break;
    case LCL_NUM_I32: launch_arith<4, kKindSigned>(p, st); break;
    case LCL_NUM_F16: launch_arith<2, kKindFloat>(p, st); break;
    default: launch_arith<4, kKindFloat>(p, st); break;
    }
    count_launches(1);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "lcl_numeric_arith launch");
    return LCL_OK;
}

lcl_status numeric_select_impl(const lcl_atlas *atlas, int type, const void *data, const uint32_t *mask, int cmp,
                               uint32_t threshold, void *layer, int label_bytes, uint32_t label, uint64_t *hits,
                               cudaStream_t st) {
    SelectArgs p;
    p.data = static_cast<const uint4 *>(data);
    p.mask = mask;
    p.cover = atlas->cover;
    p.layer = layer;
    p.threshold = threshold;
    p.label = label;
    p.cmp = cmp;
    p.n_texels = (int64_t)atlas->width * atlas->height;
    p.n_chunks = p.n_texels * (type & 15) / 16;
    p.hits = reinterpret_cast<unsigned long long *>(hits);
    if (hits) cudaMemsetAsync(hits, 0, sizeof(uint64_t), st);
#define LCL_SEL(S, K)                                                          \
    do {                                                                       \
        if (label_bytes == 1) launch_select<S, K, 1>(p, st);                   \
        else launch_select<S, K, 2>(p, st);                                    \
    } while (0)
    switch (type) {
    case LCL_NUM_U8: LCL_SEL(1, kKindUnsigned); break;
    case LCL_NUM_I8: LCL_SEL(1, kKindSigned); break;
    case LCL_NUM_U16: LCL_SEL(2, kKindUnsigned); break;
    case LCL_NUM_I16: LCL_SEL(2, kKindSigned); break;
    case LCL_NUM_U32: LCL_SEL(4, kKindUnsigned); break;
    case LCL_NUM_I32: LCL_SEL(4, kKindSigned); break;
    case LCL_NUM_F16: LCL_SEL(2, kKindFloat); break;
    default: LCL_SEL(4, kKindFloat); break;
    }
#undef LCL_SEL
    count_launches(1);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "lcl_numeric_select launch");
    return LCL_OK;
}

lcl_status numeric_stats_impl(const lcl_atlas *atlas, int type, const void *data, const uint32_t *mask,
                              const void *zones, int zone_bytes, uint32_t n_labels, lcl_zone_stats *out,
                              cudaStream_t st) {
    StatsArgs p;
    p.data = data;
    p.mask = mask;
    p.cover = atlas->cover;
    p.tri = atlas->tri;
    p.area_w = reinterpret_cast<const unsigned long long *>(atlas->area_w);
    p.zones = zones;
    p.n_labels = n_labels;
    p.n_texels = (int64_t)atlas->width * atlas->height;
    p.out = reinterpret_cast<ZoneAcc *>(out);
    const unsigned zg = std::max(1u, std::min(1024u, (n_labels + kThreads - 1) / kThreads));
    k_stats_init<<<zg, kThreads, 0, st>>>(p.out, n_labels);
    switch (type) {
    case LCL_NUM_U8: launch_stats_z<1, kKindUnsigned>(p, zone_bytes, st); break;
    case LCL_NUM_I8: launch_stats_z<1, kKindSigned>(p, zone_bytes, st); break;
    case LCL_NUM_U16: launch_stats_z<2, kKindUnsigned>(p, zone_bytes, st); break;
    case LCL_NUM_I16: launch_stats_z<2, kKindSigned>(p, zone_bytes, st); break;
    case LCL_NUM_U32: launch_stats_z<4, kKindUnsigned>(p, zone_bytes, st); break;
    case LCL_NUM_I32: launch_stats_z<4, kKindSigned>(p, zone_bytes, st); break;
    case LCL_NUM_F16: launch_stats_z<2, kKindFloat>(p, zone_bytes, st); break;
    default: launch_stats_z<4, kKindFloat>(p, zone_bytes, st); break;
    }
    k_stats_final<<<zg, kThreads, 0, st>>>(p.out, n_labels);
    count_launches(3);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "lcl_numeric_stats launch");
    return LCL_OK;
}

}  // namespace lcl
