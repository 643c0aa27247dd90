/*
 * lcl_oracle.c -- plain, slow CPU oracle for the UV-atlas layer-editing path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's
 * CPU-baseline / reference arm may load this library.  It shares no code, header,
 * table or helper with the CUDA library: it restates, step by step, what each
 * operation computes, with plain loops over every texel (no tiles, no culling, no
 * batching), so that a reader can check it against the paper by eye.
 *
 * The paper (arXiv 2501.14807) stores thematic information layers as 2D textures
 * indexed by the mesh's texture coordinates (Section 4.1, 4.2) and edits them by
 * rasterising the mesh in UV space and testing every produced texel against the
 * editing tool and a depth texture (Section 4.3.1, Fig. 3).  Where the paper is
 * silent (grid size, sub-pixel precision, fill rule, rounding, tie-breaks), this
 * file takes one stated reading; each is marked READING below.
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fPIC -shared (no FMA contraction, so
 * every float/double operation is one IEEE rounding in the order written).
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef __int128 i128;
typedef unsigned __int128 u128;

#define ORC_GRID_MAX ((1 << 21) - 1) /* 21-bit model-bbox grid */
#define ORC_SUB 256                  /* READING: 8 sub-pixel bits for rasterisation */
#define ORC_NONE 0xFFFFFFFFu         /* triangle id of an uncovered texel */
#define ORC_R2_CAP ((int64_t)1 << 50)
#define ORC_WEIGHT_CAP (((uint64_t)1 << 35) - 1)
#define ORC_AREA_FRAC 8               /* fractional bits of the per-texel area weight */

enum { ORC_OK = 0, ORC_EINVAL = 1, ORC_EUNSUP = 4 };

/* ------------------------------------------------------------------------- */
/* Quantisation of vertex positions to the 21-bit model-bbox grid.            */
/* The paper uploads the geometry once (Section 4, Geometry Manager); the      */
/* quantised grid is the exact integer form in which positions enter the atlas.*/
/* READING: one uniform scale for all axes, S = (2^21-1)/max extent, so that   */
/* spheres stay spheres; round half up via floor(x + 0.5) in double.          */
/* ------------------------------------------------------------------------- */
int orc_quant_params(const float *pos, int64_t n_pos, float mn_out[3], double *scale_out)
{
    if (n_pos <= 0) return ORC_EINVAL;
    float mn[3], mx[3];
    for (int a = 0; a < 3; ++a) { mn[a] = pos[a]; mx[a] = pos[a]; }
    for (int64_t i = 0; i < n_pos; ++i)
        for (int a = 0; a < 3; ++a) {
            float v = pos[3 * i + a];
            if (!isfinite(v)) return ORC_EINVAL;
            if (v < mn[a]) mn[a] = v;
            if (v > mx[a]) mx[a] = v;
        }
    double ext = 0.0;
    for (int a = 0; a < 3; ++a) {
        double e = (double)mx[a] - (double)mn[a];
        if (e > ext) ext = e;
    }
    if (!(ext > 0.0)) return ORC_EINVAL;
    for (int a = 0; a < 3; ++a) mn_out[a] = mn[a];
    *scale_out = (double)ORC_GRID_MAX / ext;
    return ORC_OK;
}

static int32_t quantize_coord(float p, float mn, double S)
{
    double t = ((double)p - (double)mn) * S + 0.5;
    double f = floor(t);
    if (f < 0.0) f = 0.0;
    if (f > (double)ORC_GRID_MAX) f = (double)ORC_GRID_MAX;
    return (int32_t)f;
}

int orc_quantize(const float *pos, int64_t n_pos, const float mn[3], double S, int32_t *q)
{
    for (int64_t i = 0; i < n_pos; ++i)
        for (int a = 0; a < 3; ++a) q[3 * i + a] = quantize_coord(pos[3 * i + a], mn[a], S);
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* UV-space rasterisation (Section 4.3.1: the mesh is drawn with its texture   */
/* coordinates as vertex positions, so every fragment is one texel of the      */
/* layer).  READING: UVs are snapped to 1/256 texel, X = rint(u * 256 * W)      */
/* (exact in double, ties to even); the texel centre of (i, j) is              */
/* (256 i + 128, 256 j + 128); edge functions are exact int64; a texel on an   */
/* edge belongs to the triangle that owns the edge (owner: direction d with    */
/* d.y < 0, or d.y == 0 and d.x < 0, for counter-clockwise triangles); when    */
/* several triangles cover a texel (UV overlap) the smallest triangle id wins. */
/* ------------------------------------------------------------------------- */
static int64_t edge_fn(int64_t ax, int64_t ay, int64_t bx, int64_t by, int64_t px, int64_t py)
{
    return (bx - ax) * (py - ay) - (by - ay) * (px - ax);
}

static int owner(int64_t dx, int64_t dy) { return dy < 0 || (dy == 0 && dx < 0); }

static int inside_edge(int64_t w, int64_t dx, int64_t dy) { return w > 0 || (w == 0 && owner(dx, dy)); }

static int64_t floordiv(int64_t a, int64_t b) /* b > 0 */
{
    int64_t q = a / b;
    if ((a % b != 0) && (a < 0)) q -= 1;
    return q;
}

static int snap_uv(float u, int32_t extent, int64_t *X)
{
    if (!isfinite(u) || u < -1.0f || u > 2.0f) return ORC_EINVAL; /* documented UV range */
    *X = llrint((double)u * (double)(256 * (int64_t)extent));
    return ORC_OK;
}

typedef struct {
    int64_t X[3], Y[3];  /* snapped UV, counter-clockwise after normalisation */
    int32_t q[3][3];     /* quantised positions of the same corners */
    int64_t A;           /* twice the signed UV area, > 0 after normalisation */
} orc_tri;

/* Loads triangle t, returns 0 if its UV area is zero (it covers nothing). */
static int load_tri(const float *pos, const float *uv, const uint32_t *tri_pos, const uint32_t *tri_uv,
                    int64_t t, const float mn[3], double S, int32_t W, int32_t H, orc_tri *o, int *err)
{
    for (int k = 0; k < 3; ++k) {
        uint32_t iu = tri_uv[3 * t + k], ip = tri_pos[3 * t + k];
        if (snap_uv(uv[2 * (int64_t)iu], W, &o->X[k]) || snap_uv(uv[2 * (int64_t)iu + 1], H, &o->Y[k])) {
            *err = ORC_EINVAL;
            return 0;
        }
        for (int a = 0; a < 3; ++a) o->q[k][a] = quantize_coord(pos[3 * (int64_t)ip + a], mn[a], S);
    }
    o->A = edge_fn(o->X[0], o->Y[0], o->X[1], o->Y[1], o->X[2], o->Y[2]);
    if (o->A == 0) return 0;
    if (o->A < 0) { /* make the triangle counter-clockwise: swap corners 1 and 2 */
        int64_t tx = o->X[1], ty = o->Y[1];
        o->X[1] = o->X[2]; o->Y[1] = o->Y[2]; o->X[2] = tx; o->Y[2] = ty;
        for (int a = 0; a < 3; ++a) { int32_t tq = o->q[1][a]; o->q[1][a] = o->q[2][a]; o->q[2][a] = tq; }
        o->A = -o->A;
    }
    return 1;
}

/* Edge weights at point (px, py); w[k] belongs to the edge opposite corner k. */
static int covers(const orc_tri *o, int64_t px, int64_t py, int64_t w[3])
{
    w[0] = edge_fn(o->X[1], o->Y[1], o->X[2], o->Y[2], px, py);
    w[1] = edge_fn(o->X[2], o->Y[2], o->X[0], o->Y[0], px, py);
    w[2] = edge_fn(o->X[0], o->Y[0], o->X[1], o->Y[1], px, py);
    return inside_edge(w[0], o->X[2] - o->X[1], o->Y[2] - o->Y[1]) &&
           inside_edge(w[1], o->X[0] - o->X[2], o->Y[0] - o->Y[2]) &&
           inside_edge(w[2], o->X[1] - o->X[0], o->Y[1] - o->Y[0]);
}

/*
 * Atlas: for every texel of rows [y0, y1) of a W x H texture, the id of the covering
 * triangle (smallest id if several) and its 3D position interpolated at the texel centre
 * with exact rational barycentrics w_k / A, rounded half up:
 *     q = floor((2 * sum_k w_k q_k + A) / (2 A))          (READING: exact, half up)
 * Uncovered texels get tri = 0xFFFFFFFF and position (INT32_MIN, 0, 0).
 * Output planes hold (y1 - y0) rows of W texels each.
 */
int orc_atlas(const float *pos, int64_t n_pos, const float *uv, int64_t n_uv, const uint32_t *tri_pos,
              const uint32_t *tri_uv, int64_t n_tri, const float mn[3], double S, int32_t W, int32_t H,
              int32_t y0, int32_t y1, int32_t *px, int32_t *py, int32_t *pz, uint32_t *tri)
{
    (void)n_pos; (void)n_uv;
    if (W <= 0 || H <= 0 || y0 < 0 || y1 > H || y0 > y1) return ORC_EINVAL;
    int64_t n = (int64_t)(y1 - y0) * W;
    for (int64_t i = 0; i < n; ++i) { tri[i] = ORC_NONE; px[i] = INT32_MIN; py[i] = 0; pz[i] = 0; }
    for (int64_t t = 0; t < n_tri; ++t) {
        orc_tri o;
        int err = 0;
        if (!load_tri(pos, uv, tri_pos, tri_uv, t, mn, S, W, H, &o, &err)) {
            if (err) return err;
            continue;
        }
        int64_t xmin = o.X[0], xmax = o.X[0], ymin = o.Y[0], ymax = o.Y[0];
        for (int k = 1; k < 3; ++k) {
            if (o.X[k] < xmin) xmin = o.X[k];
            if (o.X[k] > xmax) xmax = o.X[k];
            if (o.Y[k] < ymin) ymin = o.Y[k];
            if (o.Y[k] > ymax) ymax = o.Y[k];
        }
        /* texel centres 256 i + 128 inside [xmin, xmax] */
        int64_t i0 = -floordiv(-(xmin - 128), 256), i1 = floordiv(xmax - 128, 256);
        int64_t j0 = -floordiv(-(ymin - 128), 256), j1 = floordiv(ymax - 128, 256);
        if (i0 < 0) i0 = 0;
        if (i1 > W - 1) i1 = W - 1;
        if (j0 < y0) j0 = y0;
        if (j1 > y1 - 1) j1 = y1 - 1;
        for (int64_t j = j0; j <= j1; ++j)
            for (int64_t i = i0; i <= i1; ++i) {
                int64_t w[3];
                if (!covers(&o, 256 * i + 128, 256 * j + 128, w)) continue;
                int64_t idx = (j - y0) * W + i;
                if (tri[idx] != ORC_NONE) continue; /* triangles run in id order: first = smallest */
                tri[idx] = (uint32_t)t;
                int32_t *dst[3] = {px, py, pz};
                for (int a = 0; a < 3; ++a) {
                    i128 N = (i128)w[0] * o.q[0][a] + (i128)w[1] * o.q[1][a] + (i128)w[2] * o.q[2][a];
                    i128 num = 2 * N + o.A, den = 2 * (i128)o.A;
                    dst[a][idx] = (int32_t)(num / den); /* num >= 0, so truncation is floor */
                }
            }
    }
    return ORC_OK;
}

/* Integer square root floor(sqrt(n)) by bisection on x with x*x <= n. */
static uint64_t isqrt_u128(u128 n)
{
    uint64_t lo = 0, hi = (uint64_t)1 << 63; /* sqrt(2^128) = 2^64 > any answer here */
    if (n < 2) return (uint64_t)n;
    while (hi - lo > 1) {
        uint64_t mid = lo + (hi - lo) / 2;
        if ((u128)mid * mid <= n) lo = mid; else hi = mid;
    }
    return lo;
}

/*
 * Per-triangle area weight (Table 1 reports the area one texel stands for).
 * READING: a texel owned by triangle t stands for (3D area of t) / (UV area of t in
 * texels), in grid^2 units with 8 fractional bits:
 *     n = (q1 - q0) x (q2 - q0),  A3 = floor(sqrt(|n|^2)),  A_uv2 = |A| (sub-pixel^2)
 *     w = min(floor(A3 * 2^(16+8) / A_uv2), 2^35 - 1),  w = 0 if A_uv2 = 0.
 */
int orc_area_weights(const float *pos, const float *uv, const uint32_t *tri_pos, const uint32_t *tri_uv,
                     int64_t n_tri, const float mn[3], double S, int32_t W, int32_t H, uint64_t *w_out)
{
    for (int64_t t = 0; t < n_tri; ++t) {
        orc_tri o;
        int err = 0;
        int ok = load_tri(pos, uv, tri_pos, tri_uv, t, mn, S, W, H, &o, &err);
        if (err) return err;
        if (!ok) { w_out[t] = 0; continue; }
        int64_t d1[3], d2[3];
        for (int a = 0; a < 3; ++a) { d1[a] = (int64_t)o.q[1][a] - o.q[0][a]; d2[a] = (int64_t)o.q[2][a] - o.q[0][a]; }
        int64_t nx = d1[1] * d2[2] - d1[2] * d2[1];
        int64_t ny = d1[2] * d2[0] - d1[0] * d2[2];
        int64_t nz = d1[0] * d2[1] - d1[1] * d2[0];
        u128 nn = (u128)((i128)nx * nx) + (u128)((i128)ny * ny) + (u128)((i128)nz * nz);
        uint64_t a3 = isqrt_u128(nn);
        u128 w = ((u128)a3 << (16 + ORC_AREA_FRAC)) / (u128)o.A;
        w_out[t] = w > ORC_WEIGHT_CAP ? ORC_WEIGHT_CAP : (uint64_t)w;
    }
    return ORC_OK;
}

/* Coverage bitmap: bit (y*W + x) of a linear array of 32-bit words is 1 iff covered. */
int orc_cover_bits(int32_t W, int32_t H, const uint32_t *tri, uint32_t *bits)
{
    int64_t n = (int64_t)W * H;
    memset(bits, 0, (size_t)((n + 31) / 32) * 4);
    for (int64_t l = 0; l < n; ++l)
        if (tri[l] != ORC_NONE) bits[l >> 5] |= 1u << (l & 31);
    return ORC_OK;
}

/*
 * Tile boxes: for each T x T tile (row-major over ceil(W/T) x ceil(H/T) tiles), 8 int32:
 * min x, min y, min z, covered-texel count, max x, max y, max z, 0.  An empty tile holds
 * INT32_MAX mins, INT32_MIN maxes and count 0.
 */
int orc_tile_aabb(int32_t W, int32_t H, int32_t T, const int32_t *px, const int32_t *py, const int32_t *pz,
                  const uint32_t *tri, int32_t *box)
{
    int32_t ntx = (W + T - 1) / T, nty = (H + T - 1) / T;
    for (int32_t ty = 0; ty < nty; ++ty)
        for (int32_t tx = 0; tx < ntx; ++tx) {
            int32_t *b = box + 8 * ((int64_t)ty * ntx + tx);
            b[0] = b[1] = b[2] = INT32_MAX;
            b[4] = b[5] = b[6] = INT32_MIN;
            b[3] = 0; b[7] = 0;
            for (int32_t y = ty * T; y < ty * T + T && y < H; ++y)
                for (int32_t x = tx * T; x < tx * T + T && x < W; ++x) {
                    int64_t l = (int64_t)y * W + x;
                    if (tri[l] == ORC_NONE) continue;
                    int32_t v[3] = {px[l], py[l], pz[l]};
                    for (int a = 0; a < 3; ++a) {
                        if (v[a] < b[a]) b[a] = v[a];
                        if (v[a] > b[4 + a]) b[4 + a] = v[a];
                    }
                    b[3] += 1;
                }
        }
    return ORC_OK;
}

/* Super-tile boxes: the union of the boxes of G x G tiles (same 8-int32 record). */
int orc_super_aabb(int32_t ntx, int32_t nty, int32_t G, const int32_t *box, int32_t *sbox)
{
    int32_t nsx = (ntx + G - 1) / G, nsy = (nty + G - 1) / G;
    for (int32_t sy = 0; sy < nsy; ++sy)
        for (int32_t sx = 0; sx < nsx; ++sx) {
            int32_t *s = sbox + 8 * ((int64_t)sy * nsx + sx);
            s[0] = s[1] = s[2] = INT32_MAX;
            s[4] = s[5] = s[6] = INT32_MIN;
            s[3] = 0; s[7] = 0;
            for (int32_t ty = sy * G; ty < sy * G + G && ty < nty; ++ty)
                for (int32_t tx = sx * G; tx < sx * G + G && tx < ntx; ++tx) {
                    const int32_t *b = box + 8 * ((int64_t)ty * ntx + tx);
                    for (int a = 0; a < 3; ++a) {
                        if (b[a] < s[a]) s[a] = b[a];
                        if (b[4 + a] > s[4 + a]) s[4 + a] = b[4 + a];
                    }
                    s[3] += b[3];
                }
        }
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Sphere brush.  The paper's tool is a circle under the cursor (Section 4.3); */
/* the 3D sphere is its object-space counterpart.  READING: a texel is        */
/* selected iff it is covered and its squared grid distance to the centre is  */
/* <= r2 (inclusive), computed in int64; strokes run in order and a later     */
/* stroke overwrites an earlier one (the selected value is stored, Section    */
/* 4.3.1).                                                                     */
/* ------------------------------------------------------------------------- */
typedef struct {
    int32_t cx, cy, cz, pad;
    int64_t r2;
    uint32_t label, flags;
} orc_sphere; /* 32 bytes */

/* Stroke from a world-space centre and radius: centre quantised like a vertex but not
 * clamped (rejected outside [-2^22, 2^22 + 2^21]); r2 = floor((r S)^2), capped at 2^50
 * (every in-grid squared distance is below 3 * 2^46, so the cap changes no selection). */
int orc_sphere_stroke(const float mn[3], double S, const double c[3], double r, uint32_t label, orc_sphere *out)
{
    if (!(r >= 0.0) || !isfinite(r)) return ORC_EINVAL;
    int32_t q[3];
    for (int a = 0; a < 3; ++a) {
        if (!isfinite(c[a])) return ORC_EINVAL;
        double f = floor((c[a] - (double)mn[a]) * S + 0.5);
        if (f < -(double)(1 << 22) || f > (double)((1 << 22) + (1 << 21))) return ORC_EINVAL;
        q[a] = (int32_t)f;
    }
    double t = r * S;
    double t2 = floor(t * t);
    int64_t r2 = t2 >= (double)ORC_R2_CAP ? ORC_R2_CAP : (int64_t)t2;
    out->cx = q[0]; out->cy = q[1]; out->cz = q[2]; out->pad = 0;
    out->r2 = r2; out->label = label; out->flags = 0;
    return ORC_OK;
}

static void store_label(void *layer, int dtype_bytes, int64_t l, uint32_t v)
{
    if (dtype_bytes == 1) ((uint8_t *)layer)[l] = (uint8_t)v;
    else ((uint16_t *)layer)[l] = (uint16_t)v;
}

static uint32_t load_label(const void *layer, int dtype_bytes, int64_t l)
{
    return dtype_bytes == 1 ? ((const uint8_t *)layer)[l] : ((const uint16_t *)layer)[l];
}

int orc_select_sphere(int64_t n_texels, const int32_t *px, const int32_t *py, const int32_t *pz,
                      const uint32_t *tri, void *layer, int dtype_bytes, const orc_sphere *strokes, int32_t n,
                      uint64_t *hits)
{
    if (dtype_bytes != 1 && dtype_bytes != 2) return ORC_EINVAL;
    for (int32_t k = 0; k < n; ++k) {
        const orc_sphere *s = &strokes[k];
        if (s->r2 < 0 || s->label >= (1u << (8 * dtype_bytes)) || s->flags != 0) return ORC_EINVAL;
        uint64_t h = 0;
        for (int64_t l = 0; l < n_texels; ++l) {
            if (tri[l] == ORC_NONE) continue;
            int64_t dx = (int64_t)px[l] - s->cx, dy = (int64_t)py[l] - s->cy, dz = (int64_t)pz[l] - s->cz;
            int64_t d2 = dx * dx + dy * dy + dz * dz;
            if (d2 <= s->r2) {
                store_label(layer, dtype_bytes, l, s->label);
                ++h;
            }
        }
        if (hits) hits[k] = h;
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Texture Padding Algorithm (Section 4.3.2, Fig. 4): after an edit, texels of  */
/* the outline mask that lie within the kernel radius of the edited area get   */
/* the edited value, so that sampling across island borders finds it.         */
/* READING: the outline mask holds the uncovered texels within `thickness` of  */
/* a covered texel; distances are measured with the square kernel (|dx| <= k   */
/* and |dy| <= k); the edited area is the set of texels the stroke selected.   */
/* Sphere strokes ask for padding in their flags: radius = flags & 15,         */
/* thickness = (flags >> 4) & 15, both at most 8, other bits zero.            */
/* ------------------------------------------------------------------------- */
static int sphere_hits_texel(const int32_t *px, const int32_t *py, const int32_t *pz, const uint32_t *tri,
                             int64_t l, const orc_sphere *s)
{
    if (tri[l] == ORC_NONE) return 0;
    int64_t dx = (int64_t)px[l] - s->cx, dy = (int64_t)py[l] - s->cy, dz = (int64_t)pz[l] - s->cz;
    return dx * dx + dy * dy + dz * dz <= s->r2;
}

int orc_select_sphere_2d(int32_t W, int32_t H, const int32_t *px, const int32_t *py, const int32_t *pz,
                         const uint32_t *tri, void *layer, int dtype_bytes, const orc_sphere *strokes, int32_t n,
                         uint64_t *hits, uint64_t *padded)
{
    if (dtype_bytes != 1 && dtype_bytes != 2) return ORC_EINVAL;
    for (int32_t k = 0; k < n; ++k) {
        const orc_sphere *s = &strokes[k];
        uint32_t rad = s->flags & 15u, thick = (s->flags >> 4) & 15u;
        if ((s->flags & ~0xFFu) || rad > 8 || thick > 8) return ORC_EINVAL;
        orc_sphere plain = *s;
        plain.flags = 0;
        int rc = orc_select_sphere((int64_t)W * H, px, py, pz, tri, layer, dtype_bytes, &plain, 1, hits ? hits + k : NULL);
        if (rc) return rc;
        uint64_t np = 0;
        if (rad > 0) {
            int32_t reach = (int32_t)(rad > thick ? rad : thick);
            for (int32_t y = 0; y < H; ++y)
                for (int32_t x = 0; x < W; ++x) {
                    int64_t l = (int64_t)y * W + x;
                    if (tri[l] != ORC_NONE) continue;
                    int outline = 0, near = 0;
                    for (int32_t dy = -reach; dy <= reach; ++dy)
                        for (int32_t dx = -reach; dx <= reach; ++dx) {
                            int32_t yy = y + dy, xx = x + dx;
                            if (yy < 0 || yy >= H || xx < 0 || xx >= W) continue;
                            int64_t m = (int64_t)yy * W + xx;
                            if (tri[m] == ORC_NONE) continue;
                            int32_t ax = dx < 0 ? -dx : dx, ay = dy < 0 ? -dy : dy;
                            if (ax <= (int32_t)thick && ay <= (int32_t)thick) outline = 1;
                            if (ax <= (int32_t)rad && ay <= (int32_t)rad && sphere_hits_texel(px, py, pz, tri, m, s)) near = 1;
                        }
                    if (outline && near) {
                        store_label(layer, dtype_bytes, l, s->label);
                        ++np;
                    }
                }
        }
        if (padded) padded[k] = np;
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Camera and depth texture (Section 4.3.1, depth test of Fig. 3a).           */
/* READING: the camera matrix M maps a grid position (q, 1) straight to clip  */
/* space, M = VP * Dequant with Dequant(q) = bbox_min + q / S, composed in     */
/* double and rounded to float.  Clip coordinates are evaluated in FP32 in the */
/* fixed order ((m0 x + m1 y) + m2 z) + m3 with no fused multiply-add; NDC     */
/* depth lies in [0, 1]; screen x = (x/w * 0.5 + 0.5) * W_s, row 0 at the      */
/* bottom; pixels use the same sub-pixel snap, edge and owner rules as the     */
/* atlas; a triangle is dropped if a corner has w <= 0, NDC z outside [0, 1]   */
/* or lies more than 2^20 pixels off screen; the depth of a pixel is the       */
/* minimum over triangles of the barycentric interpolation of corner NDC z,    */
/* evaluated in double and rounded to float; +inf where nothing is drawn.      */
/* ------------------------------------------------------------------------- */
int orc_camera_mq(const double vp[16], const float mn[3], double S, float m_out[16])
{
    for (int i = 0; i < 4; ++i) {
        for (int j = 0; j < 3; ++j) m_out[4 * i + j] = (float)(vp[4 * i + j] / S);
        double t = ((vp[4 * i + 0] * (double)mn[0] + vp[4 * i + 1] * (double)mn[1]) + vp[4 * i + 2] * (double)mn[2]) +
                   vp[4 * i + 3];
        m_out[4 * i + 3] = (float)t;
    }
    for (int i = 0; i < 16; ++i)
        if (!isfinite(m_out[i])) return ORC_EINVAL;
    return ORC_OK;
}

static void clip_of(const float m[16], int32_t qx, int32_t qy, int32_t qz, float c[4])
{
    float x = (float)qx, y = (float)qy, z = (float)qz;
    for (int r = 0; r < 4; ++r) c[r] = ((m[4 * r + 0] * x + m[4 * r + 1] * y) + m[4 * r + 2] * z) + m[4 * r + 3];
}

static float screen_of(float ndc, int32_t extent) { return (ndc * 0.5f + 0.5f) * (float)extent; }

#define ORC_GUARD_SUB ((int64_t)1 << 28) /* 2^20 pixels in sub-pixel units */

int orc_depth(const float *pos, const uint32_t *tri_pos, int64_t n_tri, const float mn[3], double S,
              const float m[16], int32_t Ws, int32_t Hs, float *depth)
{
    if (Ws <= 0 || Hs <= 0) return ORC_EINVAL;
    for (int64_t i = 0; i < (int64_t)Ws * Hs; ++i) depth[i] = INFINITY;
    for (int64_t t = 0; t < n_tri; ++t) {
        int64_t X[3], Y[3];
        float Z[3];
        int ok = 1;
        for (int k = 0; k < 3 && ok; ++k) {
            uint32_t ip = tri_pos[3 * t + k];
            float c[4];
            clip_of(m, quantize_coord(pos[3 * (int64_t)ip + 0], mn[0], S), quantize_coord(pos[3 * (int64_t)ip + 1], mn[1], S),
                    quantize_coord(pos[3 * (int64_t)ip + 2], mn[2], S), c);
            if (!(c[3] > 0.0f)) { ok = 0; break; }
            float zn = c[2] / c[3];
            if (!(zn >= 0.0f && zn <= 1.0f)) { ok = 0; break; }
            float xs = screen_of(c[0] / c[3], Ws) * 256.0f, ys = screen_of(c[1] / c[3], Hs) * 256.0f;
            if (!(fabsf(xs) <= (float)ORC_GUARD_SUB && fabsf(ys) <= (float)ORC_GUARD_SUB)) { ok = 0; break; }
            X[k] = llrintf(xs); Y[k] = llrintf(ys); Z[k] = zn;
        }
        if (!ok) continue;
        int64_t A = edge_fn(X[0], Y[0], X[1], Y[1], X[2], Y[2]);
        if (A == 0) continue;
        if (A < 0) {
            int64_t tx = X[1], ty = Y[1]; float tz = Z[1];
            X[1] = X[2]; Y[1] = Y[2]; Z[1] = Z[2]; X[2] = tx; Y[2] = ty; Z[2] = tz;
            A = -A;
        }
        orc_tri o;
        memset(&o, 0, sizeof o);
        for (int k = 0; k < 3; ++k) { o.X[k] = X[k]; o.Y[k] = Y[k]; }
        o.A = A;
        int64_t xmin = X[0], xmax = X[0], ymin = Y[0], ymax = Y[0];
        for (int k = 1; k < 3; ++k) {
            if (X[k] < xmin) xmin = X[k];
            if (X[k] > xmax) xmax = X[k];
            if (Y[k] < ymin) ymin = Y[k];
            if (Y[k] > ymax) ymax = Y[k];
        }
        int64_t i0 = -floordiv(-(xmin - 128), 256), i1 = floordiv(xmax - 128, 256);
        int64_t j0 = -floordiv(-(ymin - 128), 256), j1 = floordiv(ymax - 128, 256);
        if (i0 < 0) i0 = 0;
        if (i1 > Ws - 1) i1 = Ws - 1;
        if (j0 < 0) j0 = 0;
        if (j1 > Hs - 1) j1 = Hs - 1;
        for (int64_t j = j0; j <= j1; ++j)
            for (int64_t i = i0; i <= i1; ++i) {
                int64_t w[3];
                if (!covers(&o, 256 * i + 128, 256 * j + 128, w)) continue;
                double num = ((double)w[0] * (double)Z[0] + (double)w[1] * (double)Z[1]) + (double)w[2] * (double)Z[2];
                float z = (float)(num / (double)A);
                z = z + 0.0f; /* no negative zero in the map */
                int64_t p = j * Ws + i;
                if (z < depth[p]) depth[p] = z;
            }
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Lasso selection: the paper's TEA (Section 4.3.1, Fig. 3) -- depth test     */
/* with a small bias, projection of the texel to the screen, and a test       */
/* against the tool's shape -- with the shape given as a polygon in screen    */
/* pixels.  READING: per covered texel, clip = M (q, 1) as for the depth map;  */
/* drop if w <= 0, NDC z outside [0, 1] or the point is outside the viewport; */
/* inside by the even-odd rule, an edge (a, b) toggling when                   */
/*   (a.y > y) != (b.y > y)  and  x < (b.x - a.x) * (y - a.y) / (b.y - a.y) + a.x */
/* in FP32 in that order; visible iff z <= D[floor(y)][floor(x)] + bias.       */
/* A texel is ambiguous (its label may legitimately differ between two exact   */
/* FP32 evaluations) if its screen point lies within 1e-4 px of an edge or    */
/* its depth margin |z - (D + bias)| is below 1e-6; both measured in double.   */
/* ------------------------------------------------------------------------- */
static double seg_dist(double px, double py, double ax, double ay, double bx, double by)
{
    double vx = bx - ax, vy = by - ay, wx = px - ax, wy = py - ay;
    double L = vx * vx + vy * vy, t = 0.0;
    if (L > 0.0) {
        t = (wx * vx + wy * vy) / L;
        if (t < 0.0) t = 0.0;
        if (t > 1.0) t = 1.0;
    }
    double dx = wx - t * vx, dy = wy - t * vy;
    return sqrt(dx * dx + dy * dy);
}

typedef struct {
    const int32_t *px, *py, *pz;
    const uint32_t *tri;
    const float *m;
    int32_t Ws, Hs;
    const float *depth;
    const float *poly;
    int32_t nv;
    float bias;
} lasso_ctx;

/* The lasso test of texel l: returns 1 if selected; *amb (if given) = ambiguous. */
static int lasso_eval(const lasso_ctx *t, int64_t l, int *amb)
{
    if (amb) *amb = 0;
    if (t->tri[l] == ORC_NONE) return 0;
    float c[4];
    clip_of(t->m, t->px[l], t->py[l], t->pz[l], c);
    if (!(c[3] > 0.0f)) return 0;
    float zn = c[2] / c[3];
    if (!(zn >= 0.0f && zn <= 1.0f)) return 0;
    float xs = screen_of(c[0] / c[3], t->Ws), ys = screen_of(c[1] / c[3], t->Hs);
    if (!(xs >= 0.0f && xs < (float)t->Ws && ys >= 0.0f && ys < (float)t->Hs)) return 0;
    const float *poly = t->poly;
    int32_t nv = t->nv;
    int inside = 0;
    for (int32_t e = 0; e < nv; ++e) {
        float ax = poly[2 * e], ay = poly[2 * e + 1];
        float bx = poly[2 * ((e + 1) % nv)], by = poly[2 * ((e + 1) % nv) + 1];
        if ((ay > ys) != (by > ys)) {
            float xi = (bx - ax) * (ys - ay) / (by - ay) + ax;
            if (xs < xi) inside = !inside;
        }
    }
    int32_t ix = (int32_t)xs, iy = (int32_t)ys; /* xs, ys >= 0: truncation is floor */
    float dref = t->depth[(int64_t)iy * t->Ws + ix];
    float lim = dref + t->bias;
    int visible = zn <= lim;
    if (amb) {
        double me = INFINITY;
        for (int32_t e = 0; e < nv; ++e) {
            double d = seg_dist(xs, ys, poly[2 * e], poly[2 * e + 1], poly[2 * ((e + 1) % nv)],
                                poly[2 * ((e + 1) % nv) + 1]);
            if (d < me) me = d;
        }
        double md = fabs((double)zn - ((double)dref + (double)t->bias));
        *amb = me < 1e-4 || md < 1e-6;
    }
    return inside && visible;
}

int orc_select_lasso(int64_t n_texels, const int32_t *px, const int32_t *py, const int32_t *pz,
                     const uint32_t *tri, void *layer, int dtype_bytes, const float m[16], int32_t Ws, int32_t Hs,
                     const float *depth, const float *poly, int32_t nv, uint32_t label, float bias, uint64_t *hits,
                     uint8_t *ambiguous)
{
    if (dtype_bytes != 1 && dtype_bytes != 2) return ORC_EINVAL;
    if (nv < 3 || nv > 64) return ORC_EUNSUP;
    if (label >= (1u << (8 * dtype_bytes))) return ORC_EINVAL;
    lasso_ctx t = {px, py, pz, tri, m, Ws, Hs, depth, poly, nv, bias};
    uint64_t h = 0;
    for (int64_t l = 0; l < n_texels; ++l) {
        int amb = 0;
        if (lasso_eval(&t, l, ambiguous ? &amb : NULL)) {
            store_label(layer, dtype_bytes, l, label);
            ++h;
        }
        if (ambiguous) ambiguous[l] = (uint8_t)amb;
    }
    if (hits) *hits = h;
    return ORC_OK;
}

/* Texture padding (Section 4.3.2) of one edit whose selection is `sel` (0/1 per texel, whole
 * texture W x H), as for sphere strokes: uncovered texels within `thick` of a covered texel and
 * within `rad` of a selected texel (square kernels) get `label`.  A padded texel is ambiguous
 * (amb, in place) if a texel within the kernel radius is.  Returns the number of padded texels. */
static uint64_t pad_selection(int32_t W, int32_t H, const uint32_t *tri, const uint8_t *sel, uint8_t *amb,
                              uint32_t rad, uint32_t thick, void *layer, int dtype_bytes, uint32_t label)
{
    uint64_t np = 0;
    if (rad == 0) return 0;
    int32_t reach = (int32_t)(rad > thick ? rad : thick);
    for (int32_t y = 0; y < H; ++y)
        for (int32_t x = 0; x < W; ++x) {
            int64_t l = (int64_t)y * W + x;
            if (tri[l] != ORC_NONE) continue;
            int outline = 0, near = 0, near_amb = 0;
            for (int32_t dy = -reach; dy <= reach; ++dy)
                for (int32_t dx = -reach; dx <= reach; ++dx) {
                    int32_t yy = y + dy, xx = x + dx;
                    if (yy < 0 || yy >= H || xx < 0 || xx >= W) continue;
                    int64_t q = (int64_t)yy * W + xx;
                    if (tri[q] == ORC_NONE) continue;
                    int32_t ax = dx < 0 ? -dx : dx, ay = dy < 0 ? -dy : dy;
                    if (ax <= (int32_t)thick && ay <= (int32_t)thick) outline = 1;
                    if (ax <= (int32_t)rad && ay <= (int32_t)rad) {
                        if (sel[q]) near = 1;
                        if (amb[q]) near_amb = 1;
                    }
                }
            if (outline && near) {
                store_label(layer, dtype_bytes, l, label);
                ++np;
            }
            if (outline && near_amb) amb[l] = 1;
        }
    return np;
}

/* A lasso with texture padding (flags = radius | thickness << 4, both at most 8): the selection of
 * orc_select_lasso, then pad_selection.  Whole texture (W x H) only. */
int orc_select_lasso_2d(int32_t W, int32_t H, const int32_t *px, const int32_t *py, const int32_t *pz,
                        const uint32_t *tri, void *layer, int dtype_bytes, const float m[16], int32_t Ws, int32_t Hs,
                        const float *depth, const float *poly, int32_t nv, uint32_t label, float bias, uint32_t flags,
                        uint64_t *hits, uint64_t *padded, uint8_t *ambiguous)
{
    if (dtype_bytes != 1 && dtype_bytes != 2) return ORC_EINVAL;
    if (nv < 3 || nv > 64) return ORC_EUNSUP;
    if (label >= (1u << (8 * dtype_bytes))) return ORC_EINVAL;
    uint32_t rad = flags & 15u, thick = (flags >> 4) & 15u;
    if ((flags & ~0xFFu) || rad > 8 || thick > 8) return ORC_EINVAL;
    lasso_ctx t = {px, py, pz, tri, m, Ws, Hs, depth, poly, nv, bias};
    int64_t n = (int64_t)W * H;
    uint8_t *sel = (uint8_t *)calloc((size_t)n, 1), *amb = (uint8_t *)calloc((size_t)n, 1);
    if (!sel || !amb) {
        free(sel);
        free(amb);
        return ORC_EINVAL;
    }
    uint64_t h = 0;
    for (int64_t l = 0; l < n; ++l) {
        int a = 0;
        sel[l] = (uint8_t)lasso_eval(&t, l, &a);
        amb[l] = (uint8_t)a;
        if (sel[l]) {
            store_label(layer, dtype_bytes, l, label);
            ++h;
        }
    }
    uint64_t np = pad_selection(W, H, tri, sel, amb, rad, thick, layer, dtype_bytes, label);
    if (ambiguous) memcpy(ambiguous, amb, (size_t)n);
    free(sel);
    free(amb);
    if (hits) *hits = h;
    if (padded) *padded = np;
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* The paper's editing tool (Section 4.3.1, Fig. 3).  The tool window is the   */
/* tw x th pixel area centred on the tool position (px, py); projective        */
/* texturing maps it onto the tool's shape texture (scale and translate        */
/* factors S_f, T_f), coordinates outside it are discarded (Fig. 3 b), and the */
/* shape texture masks the rest (Fig. 3 c); the depth test with a small bias   */
/* comes first (Fig. 3 a).  READING:                                           */
/*  - the screen point (xs, ys) of a covered texel is computed as for lassos;  */
/*  - with a shape texture of W_m x H_m texels (row 0 at the bottom):          */
/*      fu = (xs - x0) * su,  fv = (ys - y0) * sv   (FP32, in that order)       */
/*    with x0 = float(px - tw/2), su = float(W_m / tw), y0, sv likewise        */
/*    (computed in double, rounded once); the texel is in the tool iff         */
/*    0 <= fu < W_m, 0 <= fv < H_m and shape[floor(fv)][floor(fu)] != 0;       */
/*  - without a shape texture the shape is the circle (ellipse) inscribed in   */
/*    the window: ex = (xs - px) * kx, ey = (ys - py) * ky with kx =           */
/*    float(2 / tw), ky = float(2 / th), inside iff ex*ex + ey*ey <= 1 (FP32,  */
/*    products then the sum);                                                  */
/*  - visible iff z <= D[floor(ys)][floor(xs)] + bias, as for lassos.          */
/* Ambiguous texels (double): within 1e-4 px of the circle or of a shape-cell  */
/* boundary line, or depth margin below 1e-6.                                  */
/* ------------------------------------------------------------------------- */
typedef struct {
    const int32_t *px, *py, *pz;
    const uint32_t *tri;
    const float *m;
    int32_t Ws, Hs;
    const float *depth;
    float tpx, tpy, tw, th, x0, y0, su, sv, kx, ky, bias;
    const uint8_t *shape;
    int32_t shape_w, shape_h;
} tool_ctx;

/* The tool test of texel l: returns 1 if selected; *amb (if given) = ambiguous. */
static int tool_eval(const tool_ctx *t, int64_t l, int *amb)
{
    if (amb) *amb = 0;
    if (t->tri[l] == ORC_NONE) return 0;
    float c[4];
    clip_of(t->m, t->px[l], t->py[l], t->pz[l], c);
    if (!(c[3] > 0.0f)) return 0;
    float zn = c[2] / c[3];
    if (!(zn >= 0.0f && zn <= 1.0f)) return 0;
    float xs = screen_of(c[0] / c[3], t->Ws), ys = screen_of(c[1] / c[3], t->Hs);
    if (!(xs >= 0.0f && xs < (float)t->Ws && ys >= 0.0f && ys < (float)t->Hs)) return 0;
    int32_t ix = (int32_t)xs, iy = (int32_t)ys; /* xs, ys >= 0: truncation is floor */
    float dref = t->depth[(int64_t)iy * t->Ws + ix];
    int visible = zn <= dref + t->bias;
    int inside = 0;
    double near_edge = INFINITY; /* px distance to the shape's boundary, for the ambiguity flag */
    if (t->shape) {
        float fu = (xs - t->x0) * t->su, fv = (ys - t->y0) * t->sv;
        if (fu >= 0.0f && fu < (float)t->shape_w && fv >= 0.0f && fv < (float)t->shape_h)
            inside = t->shape[(int64_t)(int32_t)fv * t->shape_w + (int32_t)fu] != 0;
        if (amb) {
            double du = ((double)xs - t->x0) * ((double)t->shape_w / t->tw);
            double dv = ((double)ys - t->y0) * ((double)t->shape_h / t->th);
            if (du > -1.0 && du < t->shape_w + 1.0 && dv > -1.0 && dv < t->shape_h + 1.0) {
                double eu = fabs(du - floor(du + 0.5)) * (t->tw / (double)t->shape_w);
                double ev = fabs(dv - floor(dv + 0.5)) * (t->th / (double)t->shape_h);
                near_edge = eu < ev ? eu : ev;
            }
        }
    } else {
        float ex = (xs - t->tpx) * t->kx, ey = (ys - t->tpy) * t->ky;
        float ex2 = ex * ex, ey2 = ey * ey;
        inside = ex2 + ey2 <= 1.0f;
        if (amb) {
            double dx = ((double)xs - t->tpx) * (2.0 / t->tw), dy = ((double)ys - t->tpy) * (2.0 / t->th);
            double rmin = 0.5 * (t->tw < t->th ? t->tw : t->th);
            near_edge = fabs(sqrt(dx * dx + dy * dy) - 1.0) * rmin;
        }
    }
    if (amb) {
        double md = fabs((double)zn - ((double)dref + (double)t->bias));
        *amb = near_edge < 1e-4 || md < 1e-6;
    }
    return inside && visible;
}

static int tool_setup(tool_ctx *t, const int32_t *px, const int32_t *py, const int32_t *pz, const uint32_t *tri,
                      const float m[16], int32_t Ws, int32_t Hs, const float *depth, float tpx, float tpy, float tw,
                      float th, const uint8_t *shape, int32_t shape_w, int32_t shape_h, float bias)
{
    if (!(tw > 0.0f) || !(th > 0.0f)) return ORC_EINVAL;
    if (shape && (shape_w < 1 || shape_h < 1)) return ORC_EINVAL;
    t->px = px; t->py = py; t->pz = pz; t->tri = tri; t->m = m;
    t->Ws = Ws; t->Hs = Hs; t->depth = depth;
    t->tpx = tpx; t->tpy = tpy; t->tw = tw; t->th = th; t->bias = bias;
    t->shape = shape; t->shape_w = shape_w; t->shape_h = shape_h;
    t->x0 = (float)((double)tpx - 0.5 * (double)tw);
    t->y0 = (float)((double)tpy - 0.5 * (double)th);
    t->su = shape ? (float)((double)shape_w / (double)tw) : 0.0f;
    t->sv = shape ? (float)((double)shape_h / (double)th) : 0.0f;
    t->kx = (float)(2.0 / (double)tw);
    t->ky = (float)(2.0 / (double)th);
    return ORC_OK;
}

int orc_select_tool(int64_t n_texels, const int32_t *px, const int32_t *py, const int32_t *pz, const uint32_t *tri,
                    void *layer, int dtype_bytes, const float m[16], int32_t Ws, int32_t Hs, const float *depth,
                    float tpx, float tpy, float tw, float th, const uint8_t *shape, int32_t shape_w,
                    int32_t shape_h, uint32_t label, float bias, uint64_t *hits, uint8_t *ambiguous)
{
    if (dtype_bytes != 1 && dtype_bytes != 2) return ORC_EINVAL;
    if (label >= (1u << (8 * dtype_bytes))) return ORC_EINVAL;
    tool_ctx t;
    int rc = tool_setup(&t, px, py, pz, tri, m, Ws, Hs, depth, tpx, tpy, tw, th, shape, shape_w, shape_h, bias);
    if (rc) return rc;
    uint64_t h = 0;
    for (int64_t l = 0; l < n_texels; ++l) {
        int amb = 0;
        if (tool_eval(&t, l, ambiguous ? &amb : NULL)) {
            store_label(layer, dtype_bytes, l, label);
            ++h;
        }
        if (ambiguous) ambiguous[l] = (uint8_t)amb;
    }
    if (hits) *hits = h;
    return ORC_OK;
}

/* The tool with texture padding (Section 4.3.2, read as for sphere strokes): flags = radius |
 * thickness << 4 (both at most 8).  A padded texel is ambiguous if a texel within the kernel
 * radius is.  Whole texture (W x H) only. */
int orc_select_tool_2d(int32_t W, int32_t H, const int32_t *px, const int32_t *py, const int32_t *pz,
                       const uint32_t *tri, void *layer, int dtype_bytes, const float m[16], int32_t Ws, int32_t Hs,
                       const float *depth, float tpx, float tpy, float tw, float th, const uint8_t *shape,
                       int32_t shape_w, int32_t shape_h, uint32_t label, float bias, uint32_t flags, uint64_t *hits,
                       uint64_t *padded, uint8_t *ambiguous)
{
    if (dtype_bytes != 1 && dtype_bytes != 2) return ORC_EINVAL;
    if (label >= (1u << (8 * dtype_bytes))) return ORC_EINVAL;
    uint32_t rad = flags & 15u, thick = (flags >> 4) & 15u;
    if ((flags & ~0xFFu) || rad > 8 || thick > 8) return ORC_EINVAL;
    tool_ctx t;
    int rc = tool_setup(&t, px, py, pz, tri, m, Ws, Hs, depth, tpx, tpy, tw, th, shape, shape_w, shape_h, bias);
    if (rc) return rc;
    int64_t n = (int64_t)W * H;
    uint8_t *sel = (uint8_t *)calloc((size_t)n, 1), *amb = (uint8_t *)calloc((size_t)n, 1);
    if (!sel || !amb) {
        free(sel);
        free(amb);
        return ORC_EINVAL;
    }
    uint64_t h = 0, np = 0;
    for (int64_t l = 0; l < n; ++l) {
        int a = 0;
        sel[l] = (uint8_t)tool_eval(&t, l, &a);
        amb[l] = (uint8_t)a;
        if (sel[l]) {
            store_label(layer, dtype_bytes, l, label);
            ++h;
        }
    }
    if (rad > 0) {
        int32_t reach = (int32_t)(rad > thick ? rad : thick);
        for (int32_t y = 0; y < H; ++y)
            for (int32_t x = 0; x < W; ++x) {
                int64_t l = (int64_t)y * W + x;
                if (tri[l] != ORC_NONE) continue;
                int outline = 0, near = 0, near_amb = 0;
                for (int32_t dy = -reach; dy <= reach; ++dy)
                    for (int32_t dx = -reach; dx <= reach; ++dx) {
                        int32_t yy = y + dy, xx = x + dx;
                        if (yy < 0 || yy >= H || xx < 0 || xx >= W) continue;
                        int64_t q = (int64_t)yy * W + xx;
                        if (tri[q] == ORC_NONE) continue;
                        int32_t ax = dx < 0 ? -dx : dx, ay = dy < 0 ? -dy : dy;
                        if (ax <= (int32_t)thick && ay <= (int32_t)thick) outline = 1;
                        if (ax <= (int32_t)rad && ay <= (int32_t)rad) {
                            if (sel[q]) near = 1;
                            if (amb[q]) near_amb = 1;
                        }
                    }
                if (outline && near) {
                    store_label(layer, dtype_bytes, l, label);
                    ++np;
                }
                if (outline && near_amb) amb[l] = 1;
            }
    }
    if (ambiguous) memcpy(ambiguous, amb, (size_t)n);
    free(sel);
    free(amb);
    if (hits) *hits = h;
    if (padded) *padded = np;
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Overlay of two layers.  Layer systems combine layers with arithmetic,      */
/* logic, geometric and topological operations (Section 3.4.2); the paper's   */
/* architecture claims the same capability.  READING: bitwise operators on the */
/* label values, with optional complement of either operand and of the result */
/* (within the label width); MASK keeps a where b is non-zero; uncovered       */
/* texels become 0.                                                           */
/* ------------------------------------------------------------------------- */
enum { ORC_AND = 0, ORC_OR = 1, ORC_XOR = 2, ORC_MASK = 3 };
enum { ORC_NOT_A = 1, ORC_NOT_B = 2, ORC_NOT_OUT = 4 };

int orc_overlay(int64_t n_texels, const uint32_t *tri, const void *a, const void *b, void *out, int dtype_bytes,
                int op, uint32_t flags)
{
    if (dtype_bytes != 1 && dtype_bytes != 2) return ORC_EINVAL;
    if (op < 0 || op > 3 || (flags & ~7u)) return ORC_EINVAL;
    uint32_t full = dtype_bytes == 1 ? 0xFFu : 0xFFFFu;
    for (int64_t l = 0; l < n_texels; ++l) {
        uint32_t r = 0;
        if (tri[l] != ORC_NONE) {
            uint32_t x = load_label(a, dtype_bytes, l), y = load_label(b, dtype_bytes, l);
            if (flags & ORC_NOT_A) x = ~x & full;
            if (flags & ORC_NOT_B) y = ~y & full;
            switch (op) {
            case ORC_AND: r = x & y; break;
            case ORC_OR: r = x | y; break;
            case ORC_XOR: r = x ^ y; break;
            default: r = y != 0 ? x : 0; break;
            }
            if (flags & ORC_NOT_OUT) r = ~r & full;
        }
        store_label(out, dtype_bytes, l, r);
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Per-label surface area (Table 1: area one texel stands for).  For every    */
/* covered texel whose label l < n_labels: count[l] += 1 and                   */
/* area[l] += weight of its triangle (fixed point, 8 fractional bits of grid^2). */
/* ------------------------------------------------------------------------- */
int orc_label_area(int64_t n_texels, const void *layer, int dtype_bytes, const uint32_t *tri, const uint64_t *w_tri,
                   uint32_t n_labels, uint64_t *count, uint64_t *area)
{
    if (dtype_bytes != 1 && dtype_bytes != 2) return ORC_EINVAL;
    for (uint32_t i = 0; i < n_labels; ++i) { count[i] = 0; area[i] = 0; }
    for (int64_t l = 0; l < n_texels; ++l) {
        if (tri[l] == ORC_NONE) continue;
        uint32_t lab = load_label(layer, dtype_bytes, l);
        if (lab >= n_labels) continue;
        count[lab] += 1;
        area[lab] += w_tri[tri[l]];
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Numeric layers (Section 4.2): a data texture holding one number per texel  */
/* -- an integer of 8, 16 or 32 bits or a float of 16 or 32 bits -- and a     */
/* mask texture holding one boolean per texel (the texel holds valid data).   */
/* Here the mask is one byte per texel (0 or 1).  Type codes: low nibble =    */
/* bytes, high nibble = kind (1 unsigned, 2 signed, 3 IEEE float).            */
/* READING (the paper names the types, not their arithmetic):                 */
/*  - integers add, subtract and multiply modulo 2^bits (two's complement),   */
/*    compare by their signed or unsigned value; division is floats only;     */
/*  - float32 operations are IEEE single, round to nearest even;              */
/*  - float16 operands are widened to float32 (exact), the operation is done  */
/*    once in float32 and the result rounded to float16 (nearest even); with  */
/*    24 >= 2*11 + 2 significand bits this equals the correctly rounded        */
/*    float16 operation for + - * /;                                          */
/*  - a result is valid where both operands are valid and the texel is        */
/*    covered; elsewhere data = 0 and mask = 0;                                 */
/*  - MIN / MAX of floats: a < b ? a : b and a > b ? a : b.                    */
/* ------------------------------------------------------------------------- */
enum { ORC_NUM_U8 = 0x11, ORC_NUM_U16 = 0x12, ORC_NUM_U32 = 0x14, ORC_NUM_I8 = 0x21, ORC_NUM_I16 = 0x22,
       ORC_NUM_I32 = 0x24, ORC_NUM_F16 = 0x32, ORC_NUM_F32 = 0x34 };
enum { ORC_AR_ADD = 0, ORC_AR_SUB = 1, ORC_AR_MUL = 2, ORC_AR_DIV = 3, ORC_AR_MIN = 4, ORC_AR_MAX = 5 };
enum { ORC_CMP_LT = 0, ORC_CMP_LE = 1, ORC_CMP_GT = 2, ORC_CMP_GE = 3, ORC_CMP_EQ = 4, ORC_CMP_NE = 5 };

static int num_type_ok(int type)
{
    switch (type) {
    case ORC_NUM_U8: case ORC_NUM_U16: case ORC_NUM_U32: case ORC_NUM_I8: case ORC_NUM_I16: case ORC_NUM_I32:
    case ORC_NUM_F16: case ORC_NUM_F32: return 1;
    default: return 0;
    }
}

static int num_bytes(int type) { return type & 15; }
static int num_kind(int type) { return type >> 4; }

/* IEEE 754 binary16 -> binary32, exact: sign, 5 exponent bits (bias 15), 10 fraction bits. */
float orc_half_to_float(uint16_t h)
{
    uint32_t sign = (uint32_t)(h >> 15) & 1u, e = (uint32_t)(h >> 10) & 31u, f = (uint32_t)h & 1023u;
    float mag;
    if (e == 0) mag = ldexpf((float)f, -24);                    /* zero or subnormal: f * 2^-24 */
    else if (e == 31) mag = f ? NAN : INFINITY;
    else mag = ldexpf((float)(1024u + f), (int)e - 25);         /* (1 + f/1024) * 2^(e-15) */
    return sign ? -mag : mag;
}

/* binary32 -> binary16, round to nearest, ties to even, overflow to infinity, NaN kept quiet.
 * Works on the exact value: |x| = M * 2^E with integer M; the half result is a multiple of
 * 2^-24 (subnormal spacing) or of 2^(e-10) for a normal exponent e. */
uint16_t orc_float_to_half(float x)
{
    uint32_t b;
    memcpy(&b, &x, 4);
    uint16_t sign = (uint16_t)((b >> 16) & 0x8000u);
    if (isnan(x)) return (uint16_t)(sign | 0x7E00u);
    double a = fabs((double)x);
    if (isinf(x) || a >= 65520.0) return (uint16_t)(sign | 0x7C00u); /* 65520 = halfway above 65504 */
    if (a == 0.0) return sign;
    /* spacing of half values around a: 2^-24 below 2^-14, else 2^(floor(log2 a) - 10) */
    int e2;
    frexp(a, &e2); /* a = m * 2^e2, m in [0.5, 1): floor(log2 a) = e2 - 1 */
    int ulp_exp = (e2 - 1) - 10;
    if (ulp_exp < -24) ulp_exp = -24;
    double q = ldexp(a, -ulp_exp); /* exact: a has 24 significant bits and q < 2^12 */
    double r = floor(q), frac = q - r;
    if (frac > 0.5 || (frac == 0.5 && fmod(r, 2.0) != 0.0)) r += 1.0;
    double v = ldexp(r, ulp_exp); /* the rounded magnitude, exact in double */
    if (v >= 65520.0) return (uint16_t)(sign | 0x7C00u);
    /* encode v */
    if (v < ldexp(1.0, -14)) return (uint16_t)(sign | (uint16_t)ldexp(v, 24));
    int ev;
    double mv = frexp(v, &ev); /* v = mv * 2^ev, mv in [0.5, 1) */
    uint32_t frac10 = (uint32_t)(ldexp(mv, 11) - 1024.0);
    uint32_t ebits = (uint32_t)(ev - 1 + 15);
    return (uint16_t)(sign | (uint16_t)(ebits << 10) | (uint16_t)frac10);
}

void orc_half_to_float_n(const uint16_t *h, int64_t n, float *out)
{
    for (int64_t i = 0; i < n; ++i) out[i] = orc_half_to_float(h[i]);
}

void orc_float_to_half_n(const float *x, int64_t n, uint16_t *out)
{
    for (int64_t i = 0; i < n; ++i) out[i] = orc_float_to_half(x[i]);
}

static uint32_t num_load_bits(const void *data, int type, int64_t l)
{
    switch (num_bytes(type)) {
    case 1: return ((const uint8_t *)data)[l];
    case 2: return ((const uint16_t *)data)[l];
    default: return ((const uint32_t *)data)[l];
    }
}

static void num_store_bits(void *data, int type, int64_t l, uint32_t v)
{
    switch (num_bytes(type)) {
    case 1: ((uint8_t *)data)[l] = (uint8_t)v; break;
    case 2: ((uint16_t *)data)[l] = (uint16_t)v; break;
    default: ((uint32_t *)data)[l] = v; break;
    }
}

/* Integer value of the bits of an integer type (sign-extended for signed types). */
static int64_t num_int(int type, uint32_t bits)
{
    switch (type) {
    case ORC_NUM_I8: return (int8_t)(uint8_t)bits;
    case ORC_NUM_I16: return (int16_t)(uint16_t)bits;
    case ORC_NUM_I32: return (int32_t)bits;
    default: return (int64_t)bits;
    }
}

/* Float value of the bits of a float type. */
static float num_float(int type, uint32_t bits)
{
    if (type == ORC_NUM_F16) return orc_half_to_float((uint16_t)bits);
    float f;
    memcpy(&f, &bits, 4);
    return f;
}

static uint32_t num_from_float(int type, float f)
{
    if (type == ORC_NUM_F16) return orc_float_to_half(f);
    uint32_t b;
    memcpy(&b, &f, 4);
    return b;
}

static uint32_t width_mask(int type) { return num_bytes(type) == 4 ? 0xFFFFFFFFu : (1u << (8 * num_bytes(type))) - 1u; }

/* One arithmetic operation on two values of `type` (bits in, bits out). */
static uint32_t num_apply(int type, int op, uint32_t xa, uint32_t xb)
{
    if (num_kind(type) == 3) {
        float a = num_float(type, xa), b = num_float(type, xb), r;
        switch (op) {
        case ORC_AR_ADD: r = a + b; break;
        case ORC_AR_SUB: r = a - b; break;
        case ORC_AR_MUL: r = a * b; break;
        case ORC_AR_DIV: r = a / b; break;
        case ORC_AR_MIN: r = a < b ? a : b; break;
        default: r = a > b ? a : b; break;
        }
        return num_from_float(type, r);
    }
    int64_t a = num_int(type, xa), b = num_int(type, xb);
    uint64_t r;
    switch (op) {
    case ORC_AR_ADD: r = (uint64_t)a + (uint64_t)b; break;
    case ORC_AR_SUB: r = (uint64_t)a - (uint64_t)b; break;
    case ORC_AR_MUL: r = (uint64_t)a * (uint64_t)b; break;
    case ORC_AR_MIN: r = (uint64_t)(a < b ? a : b); break;
    default: r = (uint64_t)(a > b ? a : b); break;
    }
    return (uint32_t)r & width_mask(type);
}

/* Arithmetic overlay of two numeric layers, or of a layer and a scalar (b == NULL: every texel
 * of b holds b_scalar and is valid).  out / out_mask may alias a or b. */
int orc_num_arith(int64_t n_texels, const uint32_t *tri, int type, const void *a, const uint8_t *ma, const void *b,
                  const uint8_t *mb, uint32_t b_scalar, void *out, uint8_t *mout, int op)
{
    if (!num_type_ok(type) || op < ORC_AR_ADD || op > ORC_AR_MAX) return ORC_EINVAL;
    if (op == ORC_AR_DIV && num_kind(type) != 3) return ORC_EUNSUP;
    if (!b && (b_scalar & ~width_mask(type))) return ORC_EINVAL;
    for (int64_t l = 0; l < n_texels; ++l) {
        int valid = tri[l] != ORC_NONE && ma[l] && (b ? mb[l] != 0 : 1);
        uint32_t r = 0;
        if (valid) r = num_apply(type, op, num_load_bits(a, type, l), b ? num_load_bits(b, type, l) : b_scalar);
        num_store_bits(out, type, l, r);
        mout[l] = (uint8_t)valid;
    }
    return ORC_OK;
}

/* Selection by value: covered texels whose mask is set and whose value v satisfies
 * v <cmp> threshold get `label` in a label layer; no other texel changes.  Integers compare
 * by value, floats as IEEE floats (a NaN satisfies only NE). */
int orc_num_select(int64_t n_texels, const uint32_t *tri, int type, const void *data, const uint8_t *mask, int cmp,
                   uint32_t threshold, void *layer, int dtype_bytes, uint32_t label, uint64_t *hits)
{
    if (!num_type_ok(type) || cmp < ORC_CMP_LT || cmp > ORC_CMP_NE) return ORC_EINVAL;
    if (dtype_bytes != 1 && dtype_bytes != 2) return ORC_EINVAL;
    if (label >= (1u << (8 * dtype_bytes)) || (threshold & ~width_mask(type))) return ORC_EINVAL;
    uint64_t h = 0;
    for (int64_t l = 0; l < n_texels; ++l) {
        if (tri[l] == ORC_NONE || !mask[l]) continue;
        uint32_t bits = num_load_bits(data, type, l);
        int sel;
        if (num_kind(type) == 3) {
            float v = num_float(type, bits), t = num_float(type, threshold);
            switch (cmp) {
            case ORC_CMP_LT: sel = v < t; break;
            case ORC_CMP_LE: sel = v <= t; break;
            case ORC_CMP_GT: sel = v > t; break;
            case ORC_CMP_GE: sel = v >= t; break;
            case ORC_CMP_EQ: sel = v == t; break;
            default: sel = v != t; break;
            }
        } else {
            int64_t v = num_int(type, bits), t = num_int(type, threshold);
            switch (cmp) {
            case ORC_CMP_LT: sel = v < t; break;
            case ORC_CMP_LE: sel = v <= t; break;
            case ORC_CMP_GT: sel = v > t; break;
            case ORC_CMP_GE: sel = v >= t; break;
            case ORC_CMP_EQ: sel = v == t; break;
            default: sel = v != t; break;
            }
        }
        if (sel) {
            store_label(layer, dtype_bytes, l, label);
            ++h;
        }
    }
    if (hits) *hits = h;
    return ORC_OK;
}

/* Zonal statistics of a numeric layer over the zones of a label layer (the quantitative side of
 * Section 4.2 measured with the area weights of Table 1).  For every covered texel whose mask is
 * set, whose value v is not NaN, and whose zone label z < n_labels (zones == NULL: z = 0):
 *   count[z] += 1, area[z] += w (its triangle's area weight),
 *   vmin[z] = min, vmax[z] = max of v (as double; -0 counts as +0),
 *   sum[z] += v, wsum[z] += (double)w * v   (double, in texel order).
 * Empty zones: count = area = 0, vmin = +inf, vmax = -inf, sums 0. */
int orc_num_stats(int64_t n_texels, const uint32_t *tri, const uint64_t *w_tri, int type, const void *data,
                  const uint8_t *mask, const void *zones, int zone_bytes, uint32_t n_labels, uint64_t *count,
                  uint64_t *area, double *vmin, double *vmax, double *sum, double *wsum)
{
    if (!num_type_ok(type) || n_labels < 1) return ORC_EINVAL;
    if (zones && zone_bytes != 1 && zone_bytes != 2) return ORC_EINVAL;
    if (!zones && n_labels != 1) return ORC_EINVAL;
    for (uint32_t i = 0; i < n_labels; ++i) {
        count[i] = 0; area[i] = 0;
        vmin[i] = INFINITY; vmax[i] = -INFINITY;
        sum[i] = 0.0; wsum[i] = 0.0;
    }
    for (int64_t l = 0; l < n_texels; ++l) {
        if (tri[l] == ORC_NONE || !mask[l]) continue;
        uint32_t z = zones ? load_label(zones, zone_bytes, l) : 0u;
        if (z >= n_labels) continue;
        uint32_t bits = num_load_bits(data, type, l);
        double v = num_kind(type) == 3 ? (double)num_float(type, bits) : (double)num_int(type, bits);
        if (isnan(v)) continue;
        if (v == 0.0) v = 0.0;
        uint64_t w = w_tri[tri[l]];
        count[z] += 1;
        area[z] += w;
        if (v < vmin[z]) vmin[z] = v;
        if (v > vmax[z]) vmax[z] = v;
        sum[z] += v;
        wsum[z] += (double)w * v;
    }
    return ORC_OK;
}
