// atlas.cu -- UV atlas build: the mesh rasterised in texture space once per model
// (arXiv 2501.14807, Section 4.3.1: the mesh is drawn with its texture coordinates as
// vertex positions, so each fragment is one texel of the layer).  The paper repeats that
// rasterisation on every edit; here it runs once and its result -- per texel the covering
// triangle and the 21-bit grid position of the surface point -- is kept in HBM so that
// every later edit is a streaming pass over the texels.
//
// Kernels, in launch order:
//   k_init        tri plane := none, coverage bits := 0, header reset
//   k_bbox        float bbox of all positions (order-preserving integer atomics)
//   k_scale       grid scale (2^21-1)/extent, one thread
//   k_quant       every vertex to the grid (double, rounded once per operation)
//   k_snap        every texture coordinate to 1/256 texel (round half to even)
//   k_raster      one thread per triangle: set-up record, area weight, and the texels of
//                 small triangles (atomicMin of the triangle id: smallest id wins); big
//                 triangles are split into 16x16-texel blocks appended to a work list
//   k_raster_big  one CTA per (triangle, block) entry
//   k_resolve     one CTA per tile, one texel per thread and step: exact barycentric position of
//                 every covered texel, coverage bits, tile box
//   k_super       one CTA per super-tile: union of its tile boxes
#include <algorithm>
#include <cstring>

#include "lcl_impl.cuh"

namespace lcl {
namespace {

__global__ void k_init(uint32_t *__restrict__ tri, int64_t n_texels, uint32_t *__restrict__ cover, int64_t n_words,
                       AtlasHdr *hdr) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    uint4 none = make_uint4(kNone, kNone, kNone, kNone);
    for (int64_t k = i; k < n_texels / 4; k += stride)
        if (LCL_IN(4 * k + 3, n_texels)) reinterpret_cast<uint4 *>(tri)[k] = none;
    for (int64_t k = i; k < n_words; k += stride)
        if (LCL_IN(k, n_words)) cover[k] = 0u;
    if (i == 0) {
        for (int a = 0; a < 3; ++a) {
            hdr->key_min[a] = 0x7FFFFFFF;
            hdr->key_max[a] = (int32_t)0x80000000;
        }
        hdr->flags = 0;
        hdr->n_big = 0;
    }
}

__global__ void k_bbox(const float *__restrict__ pos, int64_t n_pos, AtlasHdr *hdr) {
    float mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
    bool bad = false;
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n_pos; v += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if (!LCL_IN(3 * v + a, 3 * n_pos)) continue;
            float p = pos[3 * v + a];
            bad |= !isfinite(p);
            mn[a] = fminf(mn[a], p);
            mx[a] = fmaxf(mx[a], p);
        }
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        for (int o = 16; o; o >>= 1) {
            mn[a] = fminf(mn[a], __shfl_xor_sync(0xffffffffu, mn[a], o));
            mx[a] = fmaxf(mx[a], __shfl_xor_sync(0xffffffffu, mx[a], o));
        }
    }
    bad = __any_sync(0xffffffffu, bad);
    if ((threadIdx.x & 31) == 0) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if (mn[a] <= mx[a]) {
                atomicMin(&hdr->key_min[a], float_key(mn[a]));
                atomicMax(&hdr->key_max[a], float_key(mx[a]));
            }
        }
        if (bad) atomicOr(&hdr->flags, kBadPos);
    }
}

__global__ void k_scale(AtlasHdr *hdr) {
    double ext = 0.0;
    for (int a = 0; a < 3; ++a) {
        float lo = key_float(hdr->key_min[a]), hi = key_float(hdr->key_max[a]);
        double e = __dsub_rn((double)hi, (double)lo);
        ext = e > ext ? e : ext;
        hdr->mn[a] = lo;
    }
    if (!(ext > 0.0)) {
        hdr->flags |= kFlatBBox;
        hdr->scale = 1.0;
    } else {
        hdr->scale = __ddiv_rn((double)kGridMax, ext);
    }
}

__global__ void k_quant(const float *__restrict__ pos, int64_t n_pos, const AtlasHdr *__restrict__ hdr,
                        int4 *__restrict__ q) {
    int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (v >= n_pos) return;
    double S = hdr->scale;
    if (!LCL_IN(3 * v + 2, 3 * n_pos)) return;
    int4 r;
    r.x = quantize_coord(pos[3 * v + 0], hdr->mn[0], S);
    r.y = quantize_coord(pos[3 * v + 1], hdr->mn[1], S);
    r.z = quantize_coord(pos[3 * v + 2], hdr->mn[2], S);
    r.w = 0;
    q[v] = r;
}

__global__ void k_snap(const float *__restrict__ uv, int64_t n_uv, int32_t w, int32_t h, AtlasHdr *hdr,
                       int2 *__restrict__ out) {
    int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (v >= n_uv) return;
    if (!LCL_IN(2 * v + 1, 2 * n_uv)) return;
    float u = uv[2 * v], t = uv[2 * v + 1];
    bool ok = isfinite(u) && isfinite(t) && u >= -1.0f && u <= 2.0f && t >= -1.0f && t <= 2.0f;
    if (!ok) {
        atomicOr(&hdr->flags, kBadUV);
        out[v] = make_int2(0, 0);
        return;
    }
    // u * 256 * extent is exact in double (24 + 22 significant bits); rint = ties to even.
    long long X = __double2ll_rn(__dmul_rn((double)u, (double)(256 * (int64_t)w)));
    long long Y = __double2ll_rn(__dmul_rn((double)t, (double)(256 * (int64_t)h)));
    out[v] = make_int2((int32_t)X, (int32_t)Y);
}

// floor(sqrt(n)) for n < 2^88 (the squared length of a cross product of 21-bit differences,
// at most 3 * 2^86): a binary64 estimate, then exact integer corrections.  Converting n to binary64
// and the correctly rounded square root each err by at most half an ulp, so the estimate is within
// 2^-8 of sqrt(n) < 2^44, and its floor within one of the result.
__device__ uint64_t isqrt_u88(unsigned __int128 n) {
    const double d = (double)(uint64_t)(n >> 64) * 18446744073709551616.0 + (double)(uint64_t)n;
    uint64_t r = (uint64_t)__dsqrt_rn(d);
#pragma unroll 1
    for (int k = 0; k < 3 && (unsigned __int128)r * r > n; ++k) --r;
#pragma unroll 1
    for (int k = 0; k < 3 && (unsigned __int128)(r + 1) * (r + 1) <= n; ++k) ++r;
    return r;
}

struct RasterArgs {
    const uint32_t *tri_pos, *tri_uv;
    int64_t n_tri, n_pos, n_uv;
    const int4 *q;
    const int2 *uvs;
    int32_t w, h;        // texture size (h: rows of the whole texture)
    int32_t row0, rows;  // the rows this atlas holds: [row0, row0 + rows)
    TriSetup *setup;
    uint64_t *area_w;
    uint32_t *tri_plane;
    AtlasHdr *hdr;
    uint2 *big;
    int64_t big_cap;
};

// Texel-centre range [i0, i1] of sub-pixel interval [lo, hi] clamped to [first, last].
__device__ __forceinline__ void texel_range(int64_t lo, int64_t hi, int64_t first, int64_t last, int64_t &i0,
                                            int64_t &i1) {
    i0 = -floordiv(-(lo - 128), 256);
    i1 = floordiv(hi - 128, 256);
    i0 = i0 < first ? first : i0;
    i1 = i1 > last ? last : i1;
}

// raster_rect for a triangle whose corners span at most 2^14 sub-pixels (64 texels) on each axis.
// The scanned texel centres lie within the corners' bounding box (the texel range is cut from it),
// and the values computed one texel past the last column or row within one texel of it, so with
// ex, ey <= 2^14 the extents: |edge value| <= ex (ey + 256) + ey (ex + 256) + 1 < 2^30, and the
// steps are at most 256 * 2^14.  The scan therefore runs in 32-bit integers after an exact start.
__device__ void raster_rect_small(const TriSetup &s, uint32_t t, int64_t i0, int64_t i1, int64_t j0, int64_t j1,
                                  int32_t w, int32_t row0, int32_t rows, uint32_t *__restrict__ tri_plane) {
    const int32_t X0 = s.x[0], X1 = s.x[1], X2 = s.x[2], Y0 = s.y[0], Y1 = s.y[1], Y2 = s.y[2];
    const int32_t px = 256 * (int32_t)i0 + 128, py = 256 * (int32_t)j0 + 128;
    int32_t e0 = (int32_t)(edge_fn32(X1, Y1, X2, Y2, px, py) + edge_bias(X2 - X1, Y2 - Y1));
    int32_t e1 = (int32_t)(edge_fn32(X2, Y2, X0, Y0, px, py) + edge_bias(X0 - X2, Y0 - Y2));
    int32_t e2 = (int32_t)(edge_fn32(X0, Y0, X1, Y1, px, py) + edge_bias(X1 - X0, Y1 - Y0));
    const int32_t dx0 = -(Y2 - Y1) * 256, dy0 = (X2 - X1) * 256;
    const int32_t dx1 = -(Y0 - Y2) * 256, dy1 = (X0 - X2) * 256;
    const int32_t dx2 = -(Y1 - Y0) * 256, dy2 = (X1 - X0) * 256;
    const int32_t n_i = (int32_t)(i1 - i0);
#pragma unroll 1
    for (int64_t j = j0; j <= j1; ++j) {
        int32_t r0 = e0, r1 = e1, r2 = e2;
        uint32_t *row = tri_plane + (j - row0) * (int64_t)w + i0;
#pragma unroll 1
        for (int32_t i = 0; i <= n_i; ++i) {
            if (min(r0, min(r1, r2)) > 0 && LCL_IN((j - row0) * (int64_t)w + i0 + i, (int64_t)w * rows))
                atomicMin(row + i, t);
            r0 += dx0;
            r1 += dx1;
            r2 += dx2;
        }
        e0 += dy0;
        e1 += dy1;
        e2 += dy2;
    }
}

// Rasterises texels [i0, i1] x [j0, j1] (texture rows j) of a set-up triangle into a plane that
// holds rows [row0, row0 + rows): atomicMin of its id.
__device__ void raster_rect(const TriSetup &s, uint32_t t, int64_t i0, int64_t i1, int64_t j0, int64_t j1, int32_t w,
                            int32_t row0, int32_t rows, uint32_t *__restrict__ tri_plane) {
    int64_t X0 = s.x[0], X1 = s.x[1], X2 = s.x[2], Y0 = s.y[0], Y1 = s.y[1], Y2 = s.y[2];
    int64_t px = 256 * i0 + 128, py = 256 * j0 + 128;
    // w_k + bias_k > 0 <=> covered (integer edge values, owned edges get bias 1)
    int64_t e0 = edge_fn(X1, Y1, X2, Y2, px, py) + edge_bias(X2 - X1, Y2 - Y1);
    int64_t e1 = edge_fn(X2, Y2, X0, Y0, px, py) + edge_bias(X0 - X2, Y0 - Y2);
    int64_t e2 = edge_fn(X0, Y0, X1, Y1, px, py) + edge_bias(X1 - X0, Y1 - Y0);
    // steps per texel: dE/dx = -(by - ay) * 256, dE/dy = (bx - ax) * 256
    int64_t dx0 = -(Y2 - Y1) * 256, dy0 = (X2 - X1) * 256;
    int64_t dx1 = -(Y0 - Y2) * 256, dy1 = (X0 - X2) * 256;
    int64_t dx2 = -(Y1 - Y0) * 256, dy2 = (X1 - X0) * 256;
#pragma unroll 1
    for (int64_t j = j0; j <= j1; ++j) {
        int64_t r0 = e0, r1 = e1, r2 = e2;
        uint32_t *row = tri_plane + (j - row0) * (int64_t)w;
#pragma unroll 1
        for (int64_t i = i0; i <= i1; ++i) {
            if (r0 > 0 && r1 > 0 && r2 > 0 && LCL_IN((j - row0) * (int64_t)w + i, (int64_t)w * rows))
                atomicMin(row + i, t);
            r0 += dx0;
            r1 += dx1;
            r2 += dx2;
        }
        e0 += dy0;
        e1 += dy1;
        e2 += dy2;
    }
}

__global__ void k_raster(RasterArgs a) {
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= a.n_tri) return;
    TriSetup s;
    s.rden = 0.0f;
    uint32_t ip[3], iu[3];
    bool ok = true;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        ip[k] = a.tri_pos[3 * t + k];
        iu[k] = a.tri_uv[3 * t + k];
        ok &= ip[k] < (uint64_t)a.n_pos && iu[k] < (uint64_t)a.n_uv;
    }
    if (!ok) {
        atomicOr(&a.hdr->flags, kBadIndex);
        s.x[0] = INT32_MIN;
        a.setup[t] = s;
        a.area_w[t] = 0;
        return;
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        int2 c = a.uvs[iu[k]];
        int4 q = a.q[ip[k]];
        s.x[k] = c.x;
        s.y[k] = c.y;
        s.qx[k] = q.x;
        s.qy[k] = q.y;
        s.qz[k] = q.z;
    }
    int64_t A = edge_fn(s.x[0], s.y[0], s.x[1], s.y[1], s.x[2], s.y[2]);
    // area weight: 3D area over UV area, floor(isqrt(|n|^2) * 2^(16+F) / |A|), capped
    {
        int64_t d1x = (int64_t)s.qx[1] - s.qx[0], d1y = (int64_t)s.qy[1] - s.qy[0], d1z = (int64_t)s.qz[1] - s.qz[0];
        int64_t d2x = (int64_t)s.qx[2] - s.qx[0], d2y = (int64_t)s.qy[2] - s.qy[0], d2z = (int64_t)s.qz[2] - s.qz[0];
        int64_t nx = d1y * d2z - d1z * d2y, ny = d1z * d2x - d1x * d2z, nz = d1x * d2y - d1y * d2x;
        unsigned __int128 nn = (unsigned __int128)((__int128)nx * nx) + (unsigned __int128)((__int128)ny * ny) +
                               (unsigned __int128)((__int128)nz * nz);
        uint64_t wgt = 0;
        if (A != 0) {
            uint64_t a3 = isqrt_u88(nn);
            unsigned __int128 num = (unsigned __int128)a3 << (16 + LCL_AREA_FRAC_BITS);
            uint64_t den = (uint64_t)(A < 0 ? -A : A);
            unsigned __int128 wq = num / den;
            wgt = wq > kWeightCap ? kWeightCap : (uint64_t)wq;
        }
        a.area_w[t] = wgt;
    }
    if (A == 0) {
        s.x[0] = INT32_MIN;
        a.setup[t] = s;
        return;
    }
    s.rden = __frcp_rn((float)(2 * (A < 0 ? -A : A)));
    if (A < 0) {  // counter-clockwise: swap corners 1 and 2
        int32_t tmp;
        tmp = s.x[1]; s.x[1] = s.x[2]; s.x[2] = tmp;
        tmp = s.y[1]; s.y[1] = s.y[2]; s.y[2] = tmp;
        tmp = s.qx[1]; s.qx[1] = s.qx[2]; s.qx[2] = tmp;
        tmp = s.qy[1]; s.qy[1] = s.qy[2]; s.qy[2] = tmp;
        tmp = s.qz[1]; s.qz[1] = s.qz[2]; s.qz[2] = tmp;
    }
    a.setup[t] = s;
    int64_t xmin = min(s.x[0], min(s.x[1], s.x[2])), xmax = max(s.x[0], max(s.x[1], s.x[2]));
    int64_t ymin = min(s.y[0], min(s.y[1], s.y[2])), ymax = max(s.y[0], max(s.y[1], s.y[2]));
    int64_t i0, i1, j0, j1;
    texel_range(xmin, xmax, 0, a.w - 1, i0, i1);
    texel_range(ymin, ymax, a.row0, (int64_t)a.row0 + a.rows - 1, j0, j1);  // this atlas's rows only
    if (i0 > i1 || j0 > j1) return;
    int64_t nx = i1 - i0 + 1, ny = j1 - j0 + 1;
    if (nx * ny <= kSmallRaster) {
        if (xmax - xmin <= (1 << 14) && ymax - ymin <= (1 << 14))
            raster_rect_small(s, (uint32_t)t, i0, i1, j0, j1, a.w, a.row0, a.rows, a.tri_plane);
        else
            raster_rect(s, (uint32_t)t, i0, i1, j0, j1, a.w, a.row0, a.rows, a.tri_plane);
        return;
    }
    int64_t nbx = (nx + kBlockSide - 1) / kBlockSide, nby = (ny + kBlockSide - 1) / kBlockSide;
    int64_t nb = nbx * nby;
    unsigned long long base = atomicAdd(&a.hdr->n_big, (unsigned long long)nb);
    if ((int64_t)base + nb <= a.big_cap) {
        for (int64_t b = 0; b < nb; ++b)
            if (LCL_IN((int64_t)base + b, a.big_cap)) a.big[base + b] = make_uint2((uint32_t)t, (uint32_t)b);
    } else {
        // list full: the reserved slots that lie below the capacity are read by k_raster_big, so they
        // get empty entries, and this thread rasterises the triangle itself
        for (int64_t b = 0; b < nb && (int64_t)base + b < a.big_cap; ++b)
            if (LCL_IN((int64_t)base + b, a.big_cap)) a.big[base + b] = make_uint2(kNone, 0u);
        raster_rect(s, (uint32_t)t, i0, i1, j0, j1, a.w, a.row0, a.rows, a.tri_plane);
    }
}

__global__ void k_raster_big(const uint2 *__restrict__ big, const AtlasHdr *__restrict__ hdr, int64_t cap,
                             const TriSetup *__restrict__ setup, int64_t n_tri, int32_t w, int32_t row0,
                             int32_t rows, uint32_t *__restrict__ tri_plane) {
    int64_t n = min((int64_t)hdr->n_big, cap);
    for (int64_t e = blockIdx.x; e < n; e += gridDim.x) {
        if (!LCL_IN(e, cap)) break;
        uint2 ent = big[e];
        if (ent.x == kNone) continue;  // a slot of a reservation that did not fit
        if (!LCL_IN(ent.x, n_tri)) continue;
        TriSetup s = setup[ent.x];
        int64_t xmin = min(s.x[0], min(s.x[1], s.x[2])), xmax = max(s.x[0], max(s.x[1], s.x[2]));
        int64_t ymin = min(s.y[0], min(s.y[1], s.y[2])), ymax = max(s.y[0], max(s.y[1], s.y[2]));
        int64_t i0, i1, j0, j1;
        texel_range(xmin, xmax, 0, w - 1, i0, i1);
        texel_range(ymin, ymax, row0, (int64_t)row0 + rows - 1, j0, j1);  // as k_raster cut the blocks
        int64_t nbx = (i1 - i0 + 1 + kBlockSide - 1) / kBlockSide;
        int64_t bx = ent.y % nbx, by = ent.y / nbx;
        int64_t i = i0 + bx * kBlockSide + (threadIdx.x % kBlockSide);
        int64_t j = j0 + by * kBlockSide + (threadIdx.x / kBlockSide);
        if (i > i1 || j > j1) continue;
        int64_t px = 256 * i + 128, py = 256 * j + 128;
        int64_t X0 = s.x[0], X1 = s.x[1], X2 = s.x[2], Y0 = s.y[0], Y1 = s.y[1], Y2 = s.y[2];
        int64_t e0 = edge_fn(X1, Y1, X2, Y2, px, py) + edge_bias(X2 - X1, Y2 - Y1);
        int64_t e1 = edge_fn(X2, Y2, X0, Y0, px, py) + edge_bias(X0 - X2, Y0 - Y2);
        int64_t e2 = edge_fn(X0, Y0, X1, Y1, px, py) + edge_bias(X1 - X0, Y1 - Y0);
        if (e0 > 0 && e1 > 0 && e2 > 0 && LCL_IN((j - row0) * (int64_t)w + i, (int64_t)w * rows))
            atomicMin(tri_plane + (j - row0) * (int64_t)w + i, ent.x);
    }
}

// Exact rounded barycentric interpolation of one axis, relative to corner 0:
// q = q0 + floor((2 (w1 (q1-q0) + w2 (q2-q0)) + A) / (2A)), which equals
// floor((2 sum_k w_k q_k + A) / (2A)) because q0 is an integer.  The quotient is estimated in
// FP32 with `rden` ~ 1/(2A) (error well under 2 units) and then made exact with integer
// remainder corrections.
__device__ __forceinline__ int32_t interp_axis(int64_t w1, int64_t w2, int64_t A, float rden, int32_t q0, int32_t q1,
                                               int32_t q2) {
    const int32_t d1 = q1 - q0, d2 = q2 - q0;  // |d| < 2^21
    if (A < (int64_t(1) << 40)) {
        const int64_t num = 2 * (w1 * d1 + w2 * d2) + A;  // |num| < 2^63 since w <= A < 2^40, |d| < 2^21
        const int64_t den = 2 * A;
        // the quotient lies within the corners' range (|num / den| <= 2^21 + 1): an int32 floor of the
        // estimate, which four roundings (num and 2A to FP32, the reciprocal, the product) leave within
        // 1/2 of num / den, so the corrections below take at most one step and usually none
        int32_t est = __float2int_rd(__fmul_rn((float)num, rden));
        int64_t r = num - (int64_t)est * den;
#pragma unroll 1
        for (int k = 0; k < 4 && r < 0; ++k) { est -= 1; r += den; }
#pragma unroll 1
        for (int k = 0; k < 4 && r >= den; ++k) { est += 1; r -= den; }
        return q0 + (int32_t)est;
    }
    __int128 num = 2 * ((__int128)w1 * d1 + (__int128)w2 * d2) + A, den = 2 * (__int128)A;
    double dn = (double)(int64_t)(num >> 64) * 18446744073709551616.0 + (double)(uint64_t)num;
    double dd = (double)(int64_t)(den >> 64) * 18446744073709551616.0 + (double)(uint64_t)den;
    int64_t est = (int64_t)floor(dn / dd);
    __int128 r = num - (__int128)est * den;
#pragma unroll 1
    for (int k = 0; k < 4 && r < 0; ++k) { est -= 1; r += den; }
#pragma unroll 1
    for (int k = 0; k < 4 && r >= den; ++k) { est += 1; r -= den; }
    return q0 + (int32_t)est;
}

__global__ void __launch_bounds__(kThreads, 4) k_resolve(const TriSetup *__restrict__ setup, int64_t n_tri, int32_t w,
                                                      int32_t h, int32_t row0, int32_t T,
                                                      const uint32_t *__restrict__ tri_plane,
                                                      int32_t *__restrict__ px, int32_t *__restrict__ py,
                                                      int32_t *__restrict__ pz, uint32_t *__restrict__ cover,
                                                      int32_t *__restrict__ tile_box) {
    const int32_t tx = blockIdx.x, ty = blockIdx.y;
    int32_t mn[3] = {INT32_MAX, INT32_MAX, INT32_MAX}, mx[3] = {INT32_MIN, INT32_MIN, INT32_MIN};
    int32_t cnt = 0;
    // one texel per thread and step, a tile row after the other: warps read the triangle plane and
    // write the position planes in whole 128-byte rows, and the texels of one triangle, which lie
    // together, find its set-up record in L1
    const int32_t n_tex_tile = T * T;
    const int iters = (n_tex_tile + kThreads - 1) / kThreads;
    // tiles of 32 texels or more on a width that is a multiple of 32: each warp's 32 texels are one
    // aligned coverage word (uniform over the grid)
    const bool aligned = T >= 32 && (w & 31) == 0;
    // the triangle id of the thread's texel in step it + 1 is loaded during step it; T is a power of
    // two, so the texel's row and column in the tile come from a shift and a mask
    const int tshift = __ffs(T) - 1;
    auto texel = [&](int step, int32_t &x, int32_t &y, int64_t &l) {
        const int32_t i = step * kThreads + threadIdx.x;
        x = tx * T + (i & (T - 1));
        y = ty * T + (i >> tshift);
        const bool v = i < n_tex_tile && x < w && y < h && LCL_IN((int64_t)y * w + x, (int64_t)w * h);
        l = v ? (int64_t)y * w + x : -1;
    };
    int32_t nx, ny;
    int64_t nl;
    texel(0, nx, ny, nl);
    uint32_t nt = nl >= 0 ? __ldcs(tri_plane + nl) : kNone;
    for (int it = 0; it < iters; ++it) {
        const int32_t x = nx, y = ny;
        const bool valid = nl >= 0;
        const int64_t l = valid ? nl : 0;
        const uint32_t t = nt;
        if (it + 1 < iters) {
            texel(it + 1, nx, ny, nl);
            nt = nl >= 0 ? __ldcs(tri_plane + nl) : kNone;
        }
        bool covered = false;
        if (valid) {
            int32_t ox = INT32_MIN, oy = 0, oz = 0;
            if (t != kNone && LCL_IN(t, n_tri)) {
                const TriSetup s = setup[t];
                // sub-pixel coordinates and texel centres lie within [-2^22, 2^23] (sides <= 2^14,
                // UVs in [-1, 2]): differences fit in 32 bits, products in 64
                const int32_t cx = 256 * x + 128, cy = 256 * (y + row0) + 128;
                const int64_t A = edge_fn32(s.x[0], s.y[0], s.x[1], s.y[1], s.x[2], s.y[2]);
                const int64_t w1 = edge_fn32(s.x[2], s.y[2], s.x[0], s.y[0], cx, cy);
                const int64_t w2 = edge_fn32(s.x[0], s.y[0], s.x[1], s.y[1], cx, cy);
                const float rden = s.rden;
                ox = interp_axis(w1, w2, A, rden, s.qx[0], s.qx[1], s.qx[2]);
                oy = interp_axis(w1, w2, A, rden, s.qy[0], s.qy[1], s.qy[2]);
                oz = interp_axis(w1, w2, A, rden, s.qz[0], s.qz[1], s.qz[2]);
                mn[0] = min(mn[0], ox); mx[0] = max(mx[0], ox);
                mn[1] = min(mn[1], oy); mx[1] = max(mx[1], oy);
                mn[2] = min(mn[2], oz); mx[2] = max(mx[2], oz);
                ++cnt;
                covered = true;
            }
            __stcs(px + l, ox);
            __stcs(py + l, oy);
            __stcs(pz + l, oz);
        }
        // coverage bits
        const uint32_t word = (uint32_t)(l >> 5);
        if (aligned) {
            // the warp holds one whole 32-texel word of one tile row (lane k = texel k): a ballot is
            // the word, written by lane 0 (the tile's CTA is its only writer)
            const uint32_t bits = __ballot_sync(0xffffffffu, covered);
            if (valid && (threadIdx.x & 31) == 0 && LCL_IN(word, ((int64_t)w * h + 31) / 32)) cover[word] = bits;
        } else {
            // lanes writing the same 32-bit word combine, one atomicOr per word
            const uint32_t val = covered ? 1u << (uint32_t)(l & 31) : 0u;
            const uint32_t peers = __match_any_sync(0xffffffffu, valid ? word : 0xFFFFFFFFu);
            const uint32_t orv = __reduce_or_sync(peers, val);
            if (valid && orv != 0 && (threadIdx.x & 31) == (__ffs(peers) - 1) &&
                LCL_IN(word, ((int64_t)w * h + 31) / 32))
                atomicOr(cover + word, orv);
        }
    }
    // tile box: block reduction
    __shared__ int32_t red[7][kThreads / 32];
    int32_t v[7] = {mn[0], mn[1], mn[2], cnt, mx[0], mx[1], mx[2]};
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        v[0] = min(v[0], __shfl_xor_sync(0xffffffffu, v[0], o));
        v[1] = min(v[1], __shfl_xor_sync(0xffffffffu, v[1], o));
        v[2] = min(v[2], __shfl_xor_sync(0xffffffffu, v[2], o));
        v[3] += __shfl_xor_sync(0xffffffffu, v[3], o);
        v[4] = max(v[4], __shfl_xor_sync(0xffffffffu, v[4], o));
        v[5] = max(v[5], __shfl_xor_sync(0xffffffffu, v[5], o));
        v[6] = max(v[6], __shfl_xor_sync(0xffffffffu, v[6], o));
    }
    const int wid = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0)
        for (int k = 0; k < 7; ++k) red[k][wid] = v[k];
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int j = 1; j < kThreads / 32; ++j) {
            v[0] = min(v[0], red[0][j]); v[1] = min(v[1], red[1][j]); v[2] = min(v[2], red[2][j]);
            v[3] += red[3][j];
            v[4] = max(v[4], red[4][j]); v[5] = max(v[5], red[5][j]); v[6] = max(v[6], red[6][j]);
        }
        if (LCL_IN((int64_t)ty * gridDim.x + tx, (int64_t)((w + T - 1) / T) * ((h + T - 1) / T))) {
            int32_t *b = tile_box + 8 * ((int64_t)ty * gridDim.x + tx);
            reinterpret_cast<int4 *>(b)[0] = make_int4(v[0], v[1], v[2], v[3]);
            reinterpret_cast<int4 *>(b)[1] = make_int4(v[4], v[5], v[6], 0);
        }
    }
}

__global__ void __launch_bounds__(kThreads) k_super(const int32_t *__restrict__ tile_box, int32_t tiles_x,
                                                    int32_t tiles_y, int32_t *__restrict__ super_box) {
    const int32_t sx = blockIdx.x, sy = blockIdx.y;
    const int32_t tx = sx * LCL_SUPER + (threadIdx.x % LCL_SUPER), ty = sy * LCL_SUPER + (threadIdx.x / LCL_SUPER);
    int32_t v[7] = {INT32_MAX, INT32_MAX, INT32_MAX, 0, INT32_MIN, INT32_MIN, INT32_MIN};
    if (tx < tiles_x && ty < tiles_y && LCL_IN((int64_t)ty * tiles_x + tx, (int64_t)tiles_x * tiles_y)) {
        const int4 *b = reinterpret_cast<const int4 *>(tile_box + 8 * ((int64_t)ty * tiles_x + tx));
        int4 lo = b[0], hi = b[1];
        v[0] = lo.x; v[1] = lo.y; v[2] = lo.z; v[3] = lo.w; v[4] = hi.x; v[5] = hi.y; v[6] = hi.z;
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        v[0] = min(v[0], __shfl_xor_sync(0xffffffffu, v[0], o));
        v[1] = min(v[1], __shfl_xor_sync(0xffffffffu, v[1], o));
        v[2] = min(v[2], __shfl_xor_sync(0xffffffffu, v[2], o));
        v[3] += __shfl_xor_sync(0xffffffffu, v[3], o);
        v[4] = max(v[4], __shfl_xor_sync(0xffffffffu, v[4], o));
        v[5] = max(v[5], __shfl_xor_sync(0xffffffffu, v[5], o));
        v[6] = max(v[6], __shfl_xor_sync(0xffffffffu, v[6], o));
    }
    __shared__ int32_t red[7][kThreads / 32];
    const int wid = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0)
        for (int k = 0; k < 7; ++k) red[k][wid] = v[k];
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int j = 1; j < kThreads / 32; ++j) {
            v[0] = min(v[0], red[0][j]); v[1] = min(v[1], red[1][j]); v[2] = min(v[2], red[2][j]);
            v[3] += red[3][j];
            v[4] = max(v[4], red[4][j]); v[5] = max(v[5], red[5][j]); v[6] = max(v[6], red[6][j]);
        }
        const int64_t n_sup = (int64_t)((tiles_x + LCL_SUPER - 1) / LCL_SUPER) * ((tiles_y + LCL_SUPER - 1) / LCL_SUPER);
        if (LCL_IN((int64_t)sy * gridDim.x + sx, n_sup)) {
            int4 *b = reinterpret_cast<int4 *>(super_box + 8 * ((int64_t)sy * gridDim.x + sx));
            b[0] = make_int4(v[0], v[1], v[2], v[3]);
            b[1] = make_int4(v[4], v[5], v[6], 0);
        }
        (void)n_sup;
    }
}

struct WsLayout {
    size_t hdr, q, uvs, setup, big, total;
};

WsLayout ws_layout(int64_t n_pos, int64_t n_uv, int64_t n_tri, int32_t w, int32_t h) {
    WsLayout L;
    L.hdr = 0;
    L.q = align256(sizeof(AtlasHdr));
    L.uvs = L.q + align256((size_t)n_pos * sizeof(int4));
    L.setup = L.uvs + align256((size_t)n_uv * sizeof(int2));
    L.big = L.setup + align256((size_t)n_tri * sizeof(TriSetup));
    L.total = L.big + align256((size_t)big_capacity(n_tri, w, h) * sizeof(uint2));
    return L;
}

}  // namespace

size_t big_capacity(int64_t n_tri, int32_t w, int32_t h) {
    int64_t blocks = ((int64_t)w / kBlockSide + 2) * ((int64_t)h / kBlockSide + 2);
    return (size_t)std::max<int64_t>(4096, n_tri / 8 + 4 * blocks);
}

size_t atlas_ws_bytes(int64_t n_pos, int64_t n_uv, int64_t n_tri, int32_t w, int32_t h) {
    return ws_layout(n_pos, n_uv, n_tri, w, h).total;
}

lcl_status atlas_build_impl(const lcl_mesh *mesh, lcl_atlas *at, void *ws, size_t ws_bytes, cudaStream_t st) {
    const WsLayout L = ws_layout(mesh->n_pos, mesh->n_uv, mesh->n_tri, at->width, at->height);
    if (ws_bytes < L.total) return fail(LCL_ERR_OUT_OF_MEMORY, "atlas workspace smaller than lcl_atlas_workspace_bytes");
    char *base = static_cast<char *>(ws);
    AtlasHdr *hdr = reinterpret_cast<AtlasHdr *>(base + L.hdr);
    int4 *q = reinterpret_cast<int4 *>(base + L.q);
    int2 *uvs = reinterpret_cast<int2 *>(base + L.uvs);
    TriSetup *setup = reinterpret_cast<TriSetup *>(base + L.setup);
    uint2 *big = reinterpret_cast<uint2 *>(base + L.big);
    const int64_t n_tex = (int64_t)at->width * at->height;
    const int64_t n_words = (n_tex + 31) / 32;
    const int sms = sm_count();

    k_init<<<sms * 8, kThreads, 0, st>>>(at->tri, n_tex, at->cover, n_words, hdr);
    k_bbox<<<std::max(1, std::min<int>(sms * 4, (int)((mesh->n_pos + kThreads - 1) / kThreads))), kThreads, 0, st>>>(
        mesh->pos, mesh->n_pos, hdr);
    k_scale<<<1, 1, 0, st>>>(hdr);
    k_quant<<<(unsigned)((mesh->n_pos + kThreads - 1) / kThreads), kThreads, 0, st>>>(mesh->pos, mesh->n_pos, hdr, q);
    const int32_t tex_h = at->tex_height > 0 ? at->tex_height : at->height;  // snapped against the whole texture
    k_snap<<<(unsigned)((mesh->n_uv + kThreads - 1) / kThreads), kThreads, 0, st>>>(mesh->uv, mesh->n_uv, at->width,
                                                                                   tex_h, hdr, uvs);
    count_launches(5);
    if (mesh->n_tri > 0) {
        RasterArgs ra;
        ra.tri_pos = mesh->tri_pos;
        ra.tri_uv = mesh->tri_uv;
        ra.n_tri = mesh->n_tri;
        ra.n_pos = mesh->n_pos;
        ra.n_uv = mesh->n_uv;
        ra.q = q;
        ra.uvs = uvs;
        ra.w = at->width;
        ra.h = tex_h;
        ra.row0 = at->row0;
        ra.rows = at->height;
        ra.setup = setup;
        ra.area_w = at->area_w;
        ra.tri_plane = at->tri;
        ra.hdr = hdr;
        ra.big = big;
        ra.big_cap = (int64_t)big_capacity(mesh->n_tri, at->width, at->height);  // blocks of this atlas's rows
        k_raster<<<(unsigned)((mesh->n_tri + 127) / 128), 128, 0, st>>>(ra);
        k_raster_big<<<sms * 8, kThreads, 0, st>>>(big, hdr, ra.big_cap, setup, mesh->n_tri, at->width, at->row0,
                                                   at->height, at->tri);
        count_launches(2);
    }
    dim3 tg(at->tiles_x, at->tiles_y);
    k_resolve<<<tg, kThreads, 0, st>>>(setup, mesh->n_tri, at->width, at->height, at->row0, at->tile, at->tri,
                                       at->pos_x, at->pos_y, at->pos_z, at->cover, at->tile_box);
    dim3 sg(at->supers_x, at->supers_y);
    k_super<<<sg, kThreads, 0, st>>>(at->tile_box, at->tiles_x, at->tiles_y, at->super_box);
    count_launches(2);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "atlas build launch");
    AtlasHdr host;
    e = cudaMemcpyAsync(&host, hdr, sizeof(AtlasHdr), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "atlas build");
    if (host.flags & kBadPos) return fail(LCL_ERR_INVALID_ARG, "mesh positions contain a non-finite value");
    if (host.flags & kFlatBBox) return fail(LCL_ERR_INVALID_ARG, "mesh bounding box has zero extent");
    if (host.flags & kBadIndex) return fail(LCL_ERR_INVALID_ARG, "triangle index out of range");
    if (host.flags & kBadUV) return fail(LCL_ERR_INVALID_ARG, "texture coordinate outside [-1, 2] or non-finite");
    for (int a = 0; a < 3; ++a) at->bbox_min[a] = host.mn[a];
    at->scale = host.scale;
    return LCL_OK;
}

}  // namespace lcl
