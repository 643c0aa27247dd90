// depth.cu -- the depth texture the lasso's visibility test reads (arXiv 2501.14807,
// Section 4.3.1: scene depth from the current viewpoint, refreshed when the camera
// changes; Fig. 3a).  The paper draws it with the graphics pipeline; here it is a CUDA
// rasteriser with the same exact integer rules as the atlas build:
//   k_clear       depth := +inf
//   k_vertex      one thread per vertex: quantise and project it (FP32, fixed order, no FMA),
//                 snap to 1/256 px, flag it if it drops its triangles (w <= 0, NDC depth
//                 outside [0, 1], off the guard band); 16 bytes per vertex
//   k_raster      one thread per triangle: gather its three vertex records, and for small
//                 triangles test every pixel centre of the bounding box; depth = barycentric
//                 interpolation of NDC z in double, rounded to float; atomicMin on the float
//                 bits (all values >= 0)
//   k_raster_big  big triangles split into 16 x 16-pixel blocks, one CTA per block
#include <algorithm>

#include "lcl_impl.cuh"

namespace lcl {
namespace {

constexpr int64_t kGuardSub = int64_t(1) << 28;  // 2^20 px in sub-pixel units

struct DepthHdr {
    unsigned long long n_big;
};

// Projected vertex: snapped screen position (1/256 px), NDC depth; X == INT32_MIN marks a vertex
// whose triangles are dropped.
struct __align__(16) PVert {
    int32_t X, Y;
    float z;
    int32_t pad;
};

struct DepthArgs {
    const float *pos;
    const uint32_t *tri_pos;
    int64_t n_tri, n_pos;
    float m[16];
    float mn[3];
    double scale;
    int32_t w, h;
    float fw, fh;
    uint32_t *depth;  // float bits
    const PVert *pv;
    DepthHdr *hdr;
    uint2 *big;
    int64_t big_cap;
};

// A set-up triangle.  Snapped corners lie within the guard band (|X|, |Y| <= 2^28 sub-pixels) and
// pixel centres within [0, 2^22), so coordinate differences fit in 32 bits and the edge functions
// are 32 x 32 -> 64-bit products.
struct DTri {
    int32_t X[3], Y[3];
    float Z[3];
    int64_t A;
};

struct Mat16 {
    float v[16];
};

__global__ void k_vertex(const float *__restrict__ pos, int64_t n_pos, const Mat16 mat, float mn0, float mn1,
                         float mn2, double scale, float fw, float fh, PVert *__restrict__ out) {
    const int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (v >= n_pos) return;
    if (!LCL_IN(3 * v + 2, 3 * n_pos)) return;
    const float *m = mat.v;
    PVert r;
    r.X = INT32_MIN;
    r.Y = 0;
    r.z = 0.0f;
    r.pad = 0;
    const float qx = (float)quantize_coord(pos[3 * v + 0], mn0, scale);
    const float qy = (float)quantize_coord(pos[3 * v + 1], mn1, scale);
    const float qz = (float)quantize_coord(pos[3 * v + 2], mn2, scale);
    const float cw = clip_row(m + 12, qx, qy, qz);
    if (cw > 0.0f) {
        // div_rn: the correctly rounded quotient, the value of __fdiv_rn (checked by lcl_check_division)
        const float zn = div_rn(clip_row(m + 8, qx, qy, qz), cw);
        const float xs = __fmul_rn(screen_of(div_rn(clip_row(m, qx, qy, qz), cw), fw), 256.0f);
        const float ys = __fmul_rn(screen_of(div_rn(clip_row(m + 4, qx, qy, qz), cw), fh), 256.0f);
        if (zn >= 0.0f && zn <= 1.0f && fabsf(xs) <= (float)kGuardSub && fabsf(ys) <= (float)kGuardSub) {
            r.X = (int32_t)__float2ll_rn(xs);
            r.Y = (int32_t)__float2ll_rn(ys);
            r.z = zn;
        }
    }
    out[v] = r;
}

// Triangle t from its projected corners; false if it is dropped (bad index, a dropped corner, or
// zero screen area).  Corners are counter-clockwise on return.
__device__ bool depth_setup(const DepthArgs &a, int64_t t, DTri &d) {
    if (!LCL_IN(3 * t + 2, 3 * a.n_tri)) return false;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const uint32_t ip = a.tri_pos[3 * t + k];
        if (ip >= (uint64_t)a.n_pos) return false;
        const PVert p = a.pv[ip];
        if (p.X == INT32_MIN) return false;
        d.X[k] = p.X;
        d.Y[k] = p.Y;
        d.Z[k] = p.z;
    }
    d.A = edge_fn32(d.X[0], d.Y[0], d.X[1], d.Y[1], d.X[2], d.Y[2]);
    if (d.A == 0) return false;
    if (d.A < 0) {
        int32_t tx = d.X[1], ty = d.Y[1];
        float tz = d.Z[1];
        d.X[1] = d.X[2]; d.Y[1] = d.Y[2]; d.Z[1] = d.Z[2];
        d.X[2] = tx; d.Y[2] = ty; d.Z[2] = tz;
        d.A = -d.A;
    }
    return true;
}

__device__ __forceinline__ void pixel_range(const DTri &d, int32_t w, int32_t h, int64_t &i0, int64_t &i1, int64_t &j0,
                                            int64_t &j1) {
    int64_t xmin = min(d.X[0], min(d.X[1], d.X[2])), xmax = max(d.X[0], max(d.X[1], d.X[2]));
    int64_t ymin = min(d.Y[0], min(d.Y[1], d.Y[2])), ymax = max(d.Y[0], max(d.Y[1], d.Y[2]));
    i0 = -floordiv(-(xmin - 128), 256);
    i1 = floordiv(xmax - 128, 256);
    j0 = -floordiv(-(ymin - 128), 256);
    j1 = floordiv(ymax - 128, 256);
    i0 = max(i0, (int64_t)0);
    j0 = max(j0, (int64_t)0);
    i1 = min(i1, (int64_t)w - 1);
    j1 = min(j1, (int64_t)h - 1);
}

// The depth of a covered pixel as the definition computes it: v = ((w0 z0 + w1 z1) + w2 z2) / A in
// binary64 (each operation rounded), then rounded to binary32.  The FP64 pipe is slow on this part,
// so the result is first decided in FP32 pairs:
//  - w_k >= 0 and z_k >= 0 (a covered pixel), so no sum cancels and the binary64 result is within
//    6 * 2^-53 (relative) of the exact x = sum w_k z_k / A (one rounding per operation);
//  - w0 + w1 + w2 = A exactly, so with A < 2^24 every w_k and A are exact floats; each product is
//    an exact pair (RN(w z), its error by FMA), the pairs' high parts are added exactly (TwoSum) and
//    the rest rounds, and the quotient is qh = RN(sh / A) plus ql from the exact remainder:
//    |qh + ql - x| <= 2^-44 x;
//  - if qh + ql lies, with that margin and the binary64 one, strictly between the rounding boundaries
//    around qh (half an ulp above, half an ulp below -- a quarter below a power of two), every value
//    within the margins rounds to qh, the binary64 result included, so the result is qh.
// Otherwise (near a boundary, about 2^-19 of the pixels, or A >= 2^24: triangles above 256 px^2)
// the binary64 sequence itself runs.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {  // s + e = a + b exactly
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __noinline__ float depth_z_binary64(int64_t w0, int64_t w1, int64_t w2, float z0, float z1, float z2,
                                               int64_t A) {
    const double num = __dadd_rn(__dadd_rn(__dmul_rn(__ll2double_rn(w0), (double)z0), __dmul_rn(__ll2double_rn(w1), (double)z1)),
                                 __dmul_rn(__ll2double_rn(w2), (double)z2));
    return __double2float_rn(__ddiv_rn(num, __ll2double_rn(A)));
}

__device__ __forceinline__ float depth_z(int64_t w0, int64_t w1, int64_t w2, const DTri &d) {
    if (d.A < (int64_t(1) << 24)) {
        const float wf[3] = {__int2float_rn((int32_t)w0), __int2float_rn((int32_t)w1), __int2float_rn((int32_t)w2)};
        float ph[3], pl[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            ph[k] = __fmul_rn(wf[k], d.Z[k]);
            pl[k] = __fmaf_rn(wf[k], d.Z[k], -ph[k]);  // the product's rounding error, exactly
        }
        float a, e1, sh, e2;
        two_sum(ph[0], ph[1], a, e1);
        two_sum(a, ph[2], sh, e2);
        float sl = __fadd_rn(__fadd_rn(e1, e2), __fadd_rn(__fadd_rn(pl[0], pl[1]), pl[2]));
        const float t = __fadd_rn(sh, sl);  // renormalise (|sl| is far below sh)
        sl = __fsub_rn(sl, __fsub_rn(t, sh));
        sh = t;
        if (sh == 0.0f) return 0.0f;  // every term is 0: x = 0 exactly
        const float af = __int2float_rn((int32_t)d.A);
        const float qh = div_rn(sh, af);
        // sh - qh A is exactly representable (the remainder of a correctly rounded quotient)
        const float ql = __fdividef(__fadd_rn(__fmaf_rn(-qh, af, sh), sl), af);
        const uint32_t bits = __float_as_uint(qh);
        const uint32_t eb = (bits >> 23) & 0xFFu;
        if (eb > 26u && eb < 255u) {
            const float half = __uint_as_float((eb - 24u) << 23);                  // ulp(qh) / 2
            const float below = (bits & 0x7FFFFFu) ? half : __fmul_rn(half, 0.5f);  // half the gap below
            const float err = __fmul_rn(qh, 0x1p-40f);
            if (ql < __fsub_rn(half, err) && -ql < __fsub_rn(below, err)) return qh;
        }
    }
    return depth_z_binary64(w0, w1, w2, d.Z[0], d.Z[1], d.Z[2], d.A);
}

// Depth of the pixel centre (px, py) if covered; writes it with atomicMin.
__device__ __forceinline__ void depth_pixel(const DTri &d, int64_t i, int64_t j, int32_t w, int32_t h, uint32_t *depth) {
    const int32_t px = 256 * (int32_t)i + 128, py = 256 * (int32_t)j + 128;
    const int64_t w0 = edge_fn32(d.X[1], d.Y[1], d.X[2], d.Y[2], px, py);
    const int64_t w1 = edge_fn32(d.X[2], d.Y[2], d.X[0], d.Y[0], px, py);
    const int64_t w2 = edge_fn32(d.X[0], d.Y[0], d.X[1], d.Y[1], px, py);
    if (w0 + edge_bias(d.X[2] - d.X[1], d.Y[2] - d.Y[1]) <= 0) return;
    if (w1 + edge_bias(d.X[0] - d.X[2], d.Y[0] - d.Y[2]) <= 0) return;
    if (w2 + edge_bias(d.X[1] - d.X[0], d.Y[1] - d.Y[0]) <= 0) return;
    float z = depth_z(w0, w1, w2, d);
    z = __fadd_rn(z, 0.0f);  // no negative zero
    if (!LCL_IN(j * (int64_t)w + i, (int64_t)w * h)) return;
    atomicMin(depth + j * (int64_t)w + i, __float_as_uint(z));
    (void)h;
}

__global__ void k_clear(uint32_t *__restrict__ depth, int64_t n) {
    const uint32_t inf = 0x7F800000u;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        if (LCL_IN(i, n)) depth[i] = inf;
}

__global__ void k_hdr_reset(DepthHdr *hdr) { hdr->n_big = 0; }

__global__ void k_raster(const __grid_constant__ DepthArgs a) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= a.n_tri) return;
    DTri d;
    if (!depth_setup(a, t, d)) return;
    int64_t i0, i1, j0, j1;
    pixel_range(d, a.w, a.h, i0, i1, j0, j1);
    if (i0 > i1 || j0 > j1) return;
    const int64_t nx = i1 - i0 + 1, ny = j1 - j0 + 1;
    if (nx * ny > kSmallRaster) {
        const int64_t nb = ((nx + kBlockSide - 1) / kBlockSide) * ((ny + kBlockSide - 1) / kBlockSide);
        const unsigned long long base = atomicAdd(&a.hdr->n_big, (unsigned long long)nb);
        if ((int64_t)base + nb <= a.big_cap) {
            for (int64_t b = 0; b < nb; ++b)
                if (LCL_IN((int64_t)base + b, a.big_cap)) a.big[base + b] = make_uint2((uint32_t)t, (uint32_t)b);
            return;
        }
        // list full: the reserved slots below the capacity are read by k_raster_big, so they get
        // empty entries, and this thread rasterises the triangle itself (below)
        for (int64_t b = 0; b < nb && (int64_t)base + b < a.big_cap; ++b)
            if (LCL_IN((int64_t)base + b, a.big_cap)) a.big[base + b] = make_uint2(kNone, 0u);
    }
#pragma unroll 1
    for (int64_t j = j0; j <= j1; ++j)
#pragma unroll 1
        for (int64_t i = i0; i <= i1; ++i) depth_pixel(d, i, j, a.w, a.h, a.depth);
}

__global__ void __launch_bounds__(kThreads) k_raster_big(const __grid_constant__ DepthArgs a) {
    __shared__ DTri sd;
    __shared__ int ok;
    const int64_t n = min((int64_t)a.hdr->n_big, a.big_cap);
    for (int64_t e = blockIdx.x; e < n; e += gridDim.x) {
        if (!LCL_IN(e, a.big_cap)) break;  // uniform over the CTA
        const uint2 ent = a.big[e];
        if (threadIdx.x == 0) ok = ent.x != kNone && depth_setup(a, ent.x, sd) ? 1 : 0;
        __syncthreads();
        if (ok) {
            const DTri d = sd;
            int64_t i0, i1, j0, j1;
            pixel_range(d, a.w, a.h, i0, i1, j0, j1);
            const int64_t nbx = (i1 - i0 + 1 + kBlockSide - 1) / kBlockSide;
            const int64_t bx = ent.y % nbx, by = ent.y / nbx;
            const int64_t i = i0 + bx * kBlockSide + (threadIdx.x % kBlockSide);
            const int64_t j = j0 + by * kBlockSide + (threadIdx.x / kBlockSide);
            if (i <= i1 && j <= j1) depth_pixel(d, i, j, a.w, a.h, a.depth);
        }
        __syncthreads();
    }
}

}  // namespace

size_t depth_ws_bytes(int64_t n_pos, int64_t n_tri, int32_t w, int32_t h) {
    return align256(sizeof(DepthHdr)) + align256(big_capacity(n_tri, w, h) * sizeof(uint2)) +
           align256((size_t)n_pos * sizeof(PVert));
}

lcl_status depth_render_impl(const lcl_mesh *mesh, const lcl_atlas *atlas, const lcl_camera *cam, float *depth,
                             void *ws, size_t ws_bytes, cudaStream_t st) {
    if (ws_bytes < depth_ws_bytes(mesh->n_pos, mesh->n_tri, cam->width, cam->height))
        return fail(LCL_ERR_OUT_OF_MEMORY, "depth workspace smaller than lcl_depth_workspace_bytes");
    DepthArgs a;
    a.pos = mesh->pos;
    a.tri_pos = mesh->tri_pos;
    a.n_tri = mesh->n_tri;
    a.n_pos = mesh->n_pos;
    for (int i = 0; i < 16; ++i) a.m[i] = cam->m[i];
    for (int i = 0; i < 3; ++i) a.mn[i] = atlas->bbox_min[i];
    a.scale = atlas->scale;
    a.w = cam->width;
    a.h = cam->height;
    a.fw = (float)cam->width;
    a.fh = (float)cam->height;
    a.depth = reinterpret_cast<uint32_t *>(depth);
    a.hdr = reinterpret_cast<DepthHdr *>(ws);
    a.big = reinterpret_cast<uint2 *>(static_cast<char *>(ws) + align256(sizeof(DepthHdr)));
    a.big_cap = (int64_t)big_capacity(mesh->n_tri, cam->width, cam->height);
    PVert *pv = reinterpret_cast<PVert *>(static_cast<char *>(ws) + align256(sizeof(DepthHdr)) +
                                          align256((size_t)a.big_cap * sizeof(uint2)));
    a.pv = pv;
    const int64_t n_px = (int64_t)cam->width * cam->height;
    const int sms = sm_count();
    k_clear<<<sms * 4, kThreads, 0, st>>>(a.depth, n_px);
    k_hdr_reset<<<1, 1, 0, st>>>(a.hdr);
    count_launches(2);
    if (mesh->n_tri > 0) {
        Mat16 mat;
        for (int i = 0; i < 16; ++i) mat.v[i] = cam->m[i];
        k_vertex<<<(unsigned)((mesh->n_pos + kThreads - 1) / kThreads), kThreads, 0, st>>>(
            mesh->pos, mesh->n_pos, mat, a.mn[0], a.mn[1], a.mn[2], a.scale, a.fw, a.fh, pv);
        k_raster<<<(unsigned)((mesh->n_tri + 127) / 128), 128, 0, st>>>(a);
        k_raster_big<<<sms * 8, kThreads, 0, st>>>(a);
        count_launches(3);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "lcl_depth_render launch");
    return LCL_OK;
}

}  // namespace lcl
