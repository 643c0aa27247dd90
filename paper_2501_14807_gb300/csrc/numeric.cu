// numeric.cu -- numeric layers (arXiv 2501.14807, Section 4.2): a data texture of 8/16/32-bit
// integers or 16/32-bit floats plus a mask texture (here one bit per texel).  Whole-layer
// operations, all HBM streams over the texture:
//   k_num_arith   arithmetic overlay a <op> b (or a <op> scalar): each lane takes a 16-byte chunk of
//                 data (warp-contiguous), the mask bits of its texels come from the word shared by
//                 the 2, 4 or 8 lanes of its group, and the group's output word is merged with
//                 shuffles and written by its first lane
//   k_num_select  selection by value into a label layer (the lane owns its texels' label bytes)
//   k_num_stats   zonal statistics: a contiguous range of 16-texel chunks per warp (one chunk per
//                 lane and step); runs of equal zone labels stay in registers until the warp
//                 meets another zone, then are reduced across the warp and flushed into a
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
        int64_t t0 = c * kPer;
        const bool live = c < p.n_chunks && LCL_IN(t0 + kPer - 1, p.n_texels);
        uint32_t bits = 0;
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
        if (t_begin < p.n_texels && LCL_IN(t_begin >> 5, (p.n_texels + 31) >> 5)) {
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
        if (!LCL_IN(c * kPer + kPer - 1, p.n_texels)) continue;
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
            if (!LCL_IN(t, p.n_texels)) break;
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

// ---- per-texel value handling for the statistics ------------------------------------------
// Order-preserving 32-bit key of a value in its own type (integer min / max, no FP64):
// unsigned: the value; signed: value ^ 2^31 (of the sign-extended value); floats: the float32
// bits with the sign folded.  key_value turns a key back into the exact double.
template <int S, int KIND>
__device__ __forceinline__ uint32_t vkey(uint32_t f32_or_int_bits) {
    if (KIND == kKindFloat) {
        const uint32_t b = f32_or_int_bits;
        return (b >> 31) ? ~b : (b | 0x80000000u);
    }
    if (KIND == kKindSigned) return (uint32_t)sext<S>(f32_or_int_bits) ^ 0x80000000u;
    return f32_or_int_bits;
}

template <int S, int KIND>
__device__ __forceinline__ double key_value(uint32_t k) {
    if (KIND == kKindFloat) return (double)__uint_as_float((k >> 31) ? (k & 0x7FFFFFFFu) : ~k);
    if (KIND == kKindSigned) return (double)(int32_t)(k ^ 0x80000000u);
    return (double)k;
}

// float32 bits -> double, by integer operations for normal numbers and zeros (FP64 throughput
// on this part is a small fraction of its integer throughput); subnormals and infinities through
// the conversion instruction.
__device__ __forceinline__ double f32_bits_to_double(uint32_t b) {
    const uint32_t e = (b >> 23) & 0xFFu;
    if (e == 0 || e == 0xFFu) {
        if ((b & 0x7FFFFFFFu) == 0) return __hiloint2double((int)(b & 0x80000000u), 0);
        return (double)__uint_as_float(b);
    }
    const uint32_t m = b & 0x7FFFFFu;
    const uint32_t hi = (b & 0x80000000u) | ((e + 896u) << 20) | (m >> 3);
    return __hiloint2double((int)hi, (int)(m << 29));
}

// Running sums of one (zone, triangle) stretch: integers and finite float16 values (integer
// multiples of 2^-24) exactly in int64, float32 values and float16 infinities in double; closed
// into the zone run as sum += s and wsum += w * s.
template <int S, int KIND>
struct TriSum {
    static constexpr bool kInt = !(KIND == kKindFloat && S == 4);
    long long i;
    double d;
    __device__ __forceinline__ void reset() {
        i = 0;
        d = 0.0;
    }
    __device__ __forceinline__ double value() const {
        if (!kInt) return d;
        if (KIND == kKindFloat) return __dadd_rn(__dmul_rn((double)i, 0x1p-24), d);  // exact: |i| < 2^45; d: infinities
        return (double)i;                                                             // exact: |i| < 2^37
    }
};

struct StatsRun {
    uint32_t zone;
    uint32_t cnt;
    unsigned long long area;
    uint32_t kmin, kmax;  // value keys (vkey) of the smallest and largest value
    double sum, wsum;
};

__device__ __forceinline__ void run_reset(StatsRun &r) {
    r.cnt = 0;
    r.area = 0;
    r.kmin = 0xFFFFFFFFu;
    r.kmax = 0u;
    r.sum = 0.0;
    r.wsum = 0.0;
}

__device__ __forceinline__ void run_merge(StatsRun &r, const StatsRun &o) {
    r.cnt += o.cnt;
    r.area += o.area;
    r.kmin = min(r.kmin, o.kmin);
    r.kmax = max(r.kmax, o.kmax);
    r.sum = __dadd_rn(r.sum, o.sum);
    r.wsum = __dadd_rn(r.wsum, o.wsum);
}

__device__ __forceinline__ void acc_add(ZoneAcc *z, unsigned long long cnt, unsigned long long area,
                                        unsigned long long kmin, unsigned long long kmax, double sum, double wsum) {
    atomicAdd(&z->count, cnt);
    atomicAdd(&z->area, area);
    atomicMin(&z->kmin, kmin);
    atomicMax(&z->kmax, kmax);
    atomicAdd(&z->sum, sum);
    atomicAdd(&z->wsum, wsum);
}

template <int S, int KIND>
__device__ __forceinline__ void flush_run(const StatsRun &r, ZoneAcc *tab, uint32_t n_zones) {
    if (r.cnt == 0) return;
    if (!LCL_IN(r.zone, n_zones)) return;
    (void)n_zones;
    acc_add(tab + r.zone, r.cnt, r.area, dkey(key_value<S, KIND>(r.kmin)), dkey(key_value<S, KIND>(r.kmax)), r.sum,
            r.wsum);
}

// Full-warp reductions (every lane gets the result).
__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long x) {
#pragma unroll
    for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}
__device__ __forceinline__ double warp_sum_f64(double x) {
#pragma unroll
    for (int o = 16; o; o >>= 1) x = __dadd_rn(x, __shfl_xor_sync(0xffffffffu, x, o));
    return x;
}

// Adds the runs of the lanes with `take` set (all of one zone) into zone `zone` of `tab`: one warp
// reduction per field, the atomics by lane `writer`.  Every lane of the warp calls it.
template <int S, int KIND>
__device__ __forceinline__ void warp_flush(const StatsRun &r, bool take, uint32_t zone, int writer, ZoneAcc *tab,
                                           uint32_t n_zones) {
    const bool t = take && r.cnt;
    const unsigned long long cnt = warp_sum_u64(t ? r.cnt : 0u);
    if (cnt == 0) return;  // uniform
    const unsigned long long area = warp_sum_u64(t ? r.area : 0ull);
    const uint32_t kmin = __reduce_min_sync(0xffffffffu, t ? r.kmin : 0xFFFFFFFFu);
    const uint32_t kmax = __reduce_max_sync(0xffffffffu, t ? r.kmax : 0u);
    const double sum = warp_sum_f64(t ? r.sum : 0.0);
    const double wsum = warp_sum_f64(t ? r.wsum : 0.0);
    if ((int)(threadIdx.x & 31) == writer && LCL_IN(zone, n_zones))
        acc_add(tab + zone, cnt, area, dkey(key_value<S, KIND>(kmin)), dkey(key_value<S, KIND>(kmax)), sum, wsum);
    (void)n_zones;
}

struct StatsArgs {
    const void *data;
    const uint32_t *mask, *cover, *tri;
    const unsigned long long *area_w;
    const void *zones;  // NULL: one zone
    uint32_t n_labels;
    int64_t n_texels;
    int64_t n_tri;
    ZoneAcc *out;
};

// Sixteen consecutive S-byte values starting at texel t (t a multiple of 16).
template <int S>
__device__ __forceinline__ void load16(const void *data, int64_t t, uint32_t (&v)[16]) {
    const uint4 *p = reinterpret_cast<const uint4 *>(static_cast<const uint8_t *>(data) + t * S);
#pragma unroll
    for (int q = 0; q < S; ++q) {
        const uint4 w = __ldcs(p + q);
        const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (S == 4) {
                v[4 * q + j] = ws[j];
            } else if (S == 2) {
                v[8 * q + 2 * j] = ws[j] & 0xFFFFu;
                v[8 * q + 2 * j + 1] = ws[j] >> 16;
            } else {
#pragma unroll
                for (int b = 0; b < 4; ++b) v[16 * q + 4 * j + b] = (ws[j] >> (8 * b)) & 0xFFu;
            }
        }
    }
}

// Zonal statistics.  A warp takes a contiguous range of iterations; in one iteration lane l takes
// the 16-texel chunk 32 it + l.  Each lane sums its chunk into a lane run (flushed by itself with
// atomics only if the zone changes inside the chunk): count, area, min / max as integer keys of
// the value's own type, and per stretch of texels of one triangle the value sum (exact in int64 for
// integer and float16 layers, in double for float32) which is closed as sum += s, wsum += w * s.
// While every lane's chunk run has the warp's current zone, the lane merges it into its share of
// the warp run, in registers; when an iteration brings another zone, the warp run is reduced
// across the warp and written by one lane, the iteration's chunk runs are reduced zone by zone,
// and the zone of lane 31 becomes the warp's zone.
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
    StatsRun run, wrun;
    run.zone = kNone;
    run_reset(run);
    run_reset(wrun);
    TriSum<S, KIND> ts_acc;
    ts_acc.reset();
    uint32_t last_t = kNone;
    unsigned long long last_w = 0;
    bool open = false;  // ts_acc holds texels of triangle last_t in zone run.zone
    auto close_tri = [&]() {
        if (!open) return;
        const double sv = ts_acc.value();
        run.sum = __dadd_rn(run.sum, sv);
        run.wsum = __dadd_rn(run.wsum, __dmul_rn((double)last_w, sv));
        ts_acc.reset();
        open = false;
    };
    auto visit = [&](uint32_t z, uint32_t t, uint32_t bits, bool valid) {
        if (!valid || t == kNone || z >= p.n_labels) return;
        uint32_t fb = bits;  // float layers: the float32 bits of the value
        if (KIND == kKindFloat) {
            if (S == 2) fb = __float_as_uint(__half2float(__ushort_as_half((unsigned short)bits)));
            if ((fb & 0x7FFFFFFFu) > 0x7F800000u) return;  // NaN
            if ((fb & 0x7FFFFFFFu) == 0) fb = 0;           // -0 counts as +0
        }
        if (z != run.zone && run.cnt) {
            close_tri();
            flush_run<S, KIND>(run, tab, p.n_labels);
            run_reset(run);
        }
        if (!LCL_IN(t, p.n_tri)) return;
        run.zone = z;
        if (t != last_t) {
            close_tri();
            last_t = t;
            last_w = __ldg(p.area_w + t);
        }
        open = true;
        run.cnt += 1;
        run.area += last_w;
        const uint32_t k = vkey<S, KIND>(fb);
        run.kmin = min(run.kmin, k);
        run.kmax = max(run.kmax, k);
        if (KIND == kKindFloat && S == 4) ts_acc.d = __dadd_rn(ts_acc.d, f32_bits_to_double(fb));
        else if (KIND == kKindFloat && (fb & 0x7FFFFFFFu) == 0x7F800000u) ts_acc.d = __dadd_rn(ts_acc.d, (double)__uint_as_float(fb));
        else if (KIND == kKindFloat) ts_acc.i += __float2ll_rn(__fmul_rn(__uint_as_float(fb), 0x1p24f));  // exact
        else if (KIND == kKindSigned) ts_acc.i += sext<S>(bits);
        else ts_acc.i += bits;
    };
    const int lane = threadIdx.x & 31;
    const int64_t n_chunks = p.n_texels / 16;
    const int64_t n_warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t n_iter = (n_chunks + 31) / 32;
    const int64_t per = (n_iter + n_warps - 1) / n_warps;
    const int64_t it0 = warp * per, it1 = min(n_iter, it0 + per);
    uint32_t wzone = kNone;
    for (int64_t it = it0; it < it1; ++it) {
        const int64_t c = it * 32 + lane;
        if (c < n_chunks && LCL_IN(16 * c + 15, p.n_texels)) {
            const int64_t t = 16 * c;
            uint32_t v[16];
            load16<S>(p.data, t, v);
            const uint4 *tp = reinterpret_cast<const uint4 *>(p.tri + t);
            const uint4 T0 = __ldcs(tp), T1 = __ldcs(tp + 1), T2 = __ldcs(tp + 2), T3 = __ldcs(tp + 3);
            const uint32_t ts[16] = {T0.x, T0.y, T0.z, T0.w, T1.x, T1.y, T1.z, T1.w,
                                     T2.x, T2.y, T2.z, T2.w, T3.x, T3.y, T3.z, T3.w};
            uint32_t z[16];
            if (p.zones) {
                const uint4 *zp = reinterpret_cast<const uint4 *>(static_cast<const uint8_t *>(p.zones) + t * ZB);
#pragma unroll
                for (int q = 0; q < ZB; ++q) {
                    const uint4 w = __ldcs(zp + q);
                    const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        if (ZB == 1) {
#pragma unroll
                            for (int b = 0; b < 4; ++b) z[4 * j + b] = (ws[j] >> (8 * b)) & 0xFFu;
                        } else {
                            z[8 * q + 2 * j] = ws[j] & 0xFFFFu;
                            z[8 * q + 2 * j + 1] = ws[j] >> 16;
                        }
                    }
                }
            } else {
#pragma unroll
                for (int k = 0; k < 16; ++k) z[k] = 0;
            }
            const uint32_t word = (uint32_t)(t >> 5);
            const uint32_t valid = (__ldg(p.mask + word) & __ldg(p.cover + word)) >> (t & 31);
#pragma unroll
            for (int k = 0; k < 16; ++k) visit(z[k], ts[k], v[k], (valid >> k) & 1u);
            close_tri();
        }
        const uint32_t key = run.cnt ? run.zone : kNone;
        if (__all_sync(0xffffffffu, key == wzone || key == kNone)) {
            if (run.cnt) run_merge(wrun, run);
        } else {
            warp_flush<S, KIND>(wrun, true, wzone, 0, tab, p.n_labels);
            run_reset(wrun);
            // this iteration's chunk runs, zone by zone
            unsigned left = __ballot_sync(0xffffffffu, key != kNone);
            while (left) {
                const int leader = __ffs(left) - 1;
                const uint32_t zk = __shfl_sync(0xffffffffu, key, leader);
                const bool mine = key == zk;
                warp_flush<S, KIND>(run, mine, zk, leader, tab, p.n_labels);
                left &= ~__ballot_sync(0xffffffffu, mine);
            }
            wzone = __shfl_sync(0xffffffffu, key, 31);
        }
        run_reset(run);
    }
    warp_flush<S, KIND>(wrun, true, wzone, 0, tab, p.n_labels);
    // tail texels (n_texels % 16), one per thread
    for (int64_t t = n_chunks * 16 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < p.n_texels;
         t += (int64_t)gridDim.x * blockDim.x) {
        if (!LCL_IN(t, p.n_texels)) break;
        uint32_t bits, z = 0;
        if (S == 1) bits = static_cast<const uint8_t *>(p.data)[t];
        else if (S == 2) bits = static_cast<const uint16_t *>(p.data)[t];
        else bits = static_cast<const uint32_t *>(p.data)[t];
        if (p.zones) z = ZB == 1 ? static_cast<const uint8_t *>(p.zones)[t] : static_cast<const uint16_t *>(p.zones)[t];
        const uint32_t word = (uint32_t)(t >> 5);
        const bool valid = ((p.mask[word] & p.cover[word]) >> (t & 31)) & 1u;
        visit(z, p.tri[t], bits, valid);
    }
    close_tri();
    flush_run<S, KIND>(run, tab, p.n_labels);
    if (SMEM) {
        __syncthreads();
        for (uint32_t i = threadIdx.x; i < p.n_labels; i += blockDim.x) {
            const ZoneAcc &a = sh_zone[i];
            if (a.count == 0) continue;
            acc_add(p.out + i, a.count, a.area, a.kmin, a.kmax, a.sum, a.wsum);
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
    const int64_t threads = p.n_texels / 16 + 1;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)sm_count() * per_sm,
                                                                 (threads + kThreads - 1) / kThreads));
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
    p.n_tri = atlas->n_tri;
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
