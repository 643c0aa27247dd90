// batch.cu -- batched edits: many models, each with a queue of sphere and lasso strokes, edited
// by two cull launches and one persistent apply launch (capturable in a CUDA graph).
//
// The paper edits one layer of one model per operation (Section 4.3.1).  A server holding many
// models batches their queued strokes instead: the result must equal applying each model's
// strokes one by one, in queue order, so
//   k_batch_pairs  gives every tile of every model a 64-bit mask of the model's queued strokes
//                  (queue order = bit order) whose conservative box test can reach the tile, and
//                  of those a `sure` mask (spheres containing the tile, lassos inside whose polygon
//                  it lies): a CTA per (super-tile, stroke) unit, a thread per tile, the bits ORed
//                  into per-tile masks, so one super-tile's strokes are tested in parallel;
//   k_batch_compact turns every tile with a non-empty mask into a work item (model, tile, masks);
//   k_batch_apply  takes (item, part) units from a work queue (one atomic per unit and CTA); a
//                  thread loads its four texels' positions once and evaluates the masked strokes
//                  from the newest down: the first stroke that selects a texel is the last one
//                  sequential application would have written there, so the texel is final and
//                  the thread stops once its four texels are final (or no stroke is left); each
//                  label word is written once.  Texture padding (Section 4.3.2) writes only
//                  uncovered texels, so for those the masked padded strokes are evaluated the
//                  same way (newest first, on the neighbours' positions), and a padded stroke's
//                  cull counts a tile whose 3 x 3 neighbourhood it may reach.
// Each texel belongs to one unit and one thread, so no two threads write a texel, and the label a
// texel receives is that of the newest stroke selecting it: the result is bit-identical to
// sequential single-stroke calls.
//
// The host uploads compact descriptors (models, strokes, each lasso's camera and polygon);
// k_batch_prep clears the tile masks and builds the lassos' culling boxes and y-band edge lists on
// the device, one warp per lasso.  Workspace layout and launch shape depend only on the limits (capacities) and the config,
// and the kernels read the batch's counts from the workspace header, so the launch is independent
// of the batch's contents: it can be captured once in a CUDA graph and replayed after each upload.
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
    int64_t tile0;    // first flattened tile of this model (index into the tile masks)
};

struct BStroke {
    int32_t kind;     // LCL_STROKE_SPHERE or LCL_STROKE_LASSO
    int32_t lasso;    // index into the lasso array
    SphereArg sphere;
};

struct BLasso {  // built on the device by k_batch_prep
    LassoArg arg;
    const float *depth;
    int32_t pad_r, pad_t;  // texture padding: kernel radius and outline thickness (0: none)
};

struct BLassoIn {  // what the host uploads per lasso
    float m[16];
    int32_t w_s, h_s;
    const float *depth;
    float poly[2 * LCL_MAX_LASSO_VERTICES];
    int32_t nv;
    uint32_t label;
    float bias;
    uint32_t flags;  // texture padding: radius = bits 0-3, thickness = bits 4-7
};

struct BItem {
    uint32_t model, tile;
    unsigned long long mask;  // strokes that can write a texel of the tile
    unsigned long long sure;  // of those: spheres containing the tile's box (every covered texel
                              // selected) and unpadded lassos inside whose polygon the tile lies
};

// Capacities of a workspace's arrays (its limits), for the kernels' index checks.
struct BCaps {
    int32_t models, strokes, lassos, pad;
    int64_t supers, tiles;
};

// Can the stroke's descriptors be read: its index within the strokes and, for a lasso, the lasso's
// within the lassos (the debug build's checks; always true otherwise).
__device__ __forceinline__ bool stroke_in_bounds(const BStroke *strokes, int64_t si, const BCaps &caps) {
    if (!LCL_IN(si, caps.strokes)) return false;
    return strokes[si].kind == LCL_STROKE_SPHERE || LCL_IN(strokes[si].lasso, caps.lassos);
}

// Workspace header (first 256 bytes), uploaded with the descriptors; the counters are reset by
// k_batch_prep at every launch.
struct BHdr {
    int32_t n_models, n_strokes, n_lassos, n_supers;
    unsigned int n_items;          // written by k_batch_compact
    unsigned int n_tiles;          // tiles of the batch's models (the tile masks in use)
    unsigned long long next_unit;  // work queue of k_batch_apply
};

// Workspace: [hdr | models | strokes | lasso inputs | super-tile -> model] is uploaded (the
// staging holds its image); [lassos | items | tile masks] is written by the kernels.
struct BLayout {
    size_t hdr, models, strokes, lasso_in, super_model, upload, lassos, items, tmask, total;
};

BLayout b_layout(const lcl_batch_limits &lim) {
    BLayout L;
    L.hdr = 0;
    L.models = align256(sizeof(BHdr));
    L.strokes = L.models + align256((size_t)std::max(lim.models, 1) * sizeof(BModel));
    L.lasso_in = L.strokes + align256((size_t)std::max(lim.strokes, 1) * sizeof(BStroke));
    L.super_model = L.lasso_in + align256((size_t)std::max(lim.lassos, 1) * sizeof(BLassoIn));
    L.upload = L.super_model + align256((size_t)std::max<int64_t>(lim.supers, 1) * 4);
    L.lassos = L.upload;
    L.items = L.lassos + align256((size_t)std::max(lim.lassos, 1) * sizeof(BLasso));
    L.tmask = L.items + align256((size_t)std::max<int64_t>(lim.tiles, 1) * sizeof(BItem));
    L.total = L.tmask + align256((size_t)std::max<int64_t>(lim.tiles, 1) * sizeof(ulonglong2));
    return L;
}

__device__ __forceinline__ bool stroke_may_touch(const BStroke &st, const BLasso *lassos, int4 lo, int4 hi) {
    if (lo.w == 0) return false;
    if (st.kind == LCL_STROKE_SPHERE) return box_dist2(lo, hi, st.sphere) <= st.sphere.r2;
    return box_may_touch(lassos[st.lasso].arg, lo, hi, lassos[st.lasso].depth);
}

__device__ __forceinline__ bool stroke_pads(const BStroke &st, const BLasso *lassos) {
    return st.kind == LCL_STROKE_SPHERE ? st.sphere.pad_r > 0 : lassos[st.lasso].pad_r > 0;
}

// Box (bx, by) of a grid of nx x ny boxes (8 int32 each): can the stroke write a texel in it?  With
// texture padding a texel may be written because a neighbour within 8 texels (at most one tile,
// and so one super-tile, away) is selected, so then any box of the 3 x 3 neighbourhood counts.
__device__ __forceinline__ bool stroke_may_reach(const BStroke &st, const BLasso *lassos, const int32_t *boxes,
                                                 int32_t nx, int32_t ny, int32_t bx, int32_t by) {
    const bool pad = stroke_pads(st, lassos);
    const int32_t r = pad ? 1 : 0;
    for (int32_t y = max(by - r, 0); y <= min(by + r, ny - 1); ++y)
        for (int32_t x = max(bx - r, 0); x <= min(bx + r, nx - 1); ++x) {
            if (!LCL_IN((int64_t)y * nx + x, (int64_t)nx * ny)) continue;
            const int4 *b = reinterpret_cast<const int4 *>(boxes + 8 * ((int64_t)y * nx + x));
            if (stroke_may_touch(st, lassos, b[0], b[1])) return true;
        }
    return false;
}

constexpr int kPrepWarps = kThreads / 32;  // lassos per CTA of k_batch_prep
static_assert(kBands == 32, "k_batch_prep gives each y-band one lane");

// Resets the work counters and the tile masks and builds every lasso's argument, one warp per
// lasso: lane 0 the
// head (bounding boxes, band mapping), then lane b counts and lists the edges of band b (the
// same predicate, in the same edge order, as the host builder).
__global__ void __launch_bounds__(kThreads) k_batch_prep(BHdr *hdr, const BLassoIn *__restrict__ in,
                                                         BLasso *__restrict__ out, ulonglong2 *__restrict__ tmask,
                                                         BCaps caps) {
    pdl_allow_next();
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        hdr->n_items = 0;
        hdr->next_unit = 0;
    }
    const int64_t n_tiles = hdr->n_tiles;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n_tiles; t += (int64_t)gridDim.x * blockDim.x)
        if (LCL_IN(t, caps.tiles)) tmask[t] = make_ulonglong2(0ull, 0ull);
    const int lane = threadIdx.x & 31;
    const int j = blockIdx.x * kPrepWarps + (int)(threadIdx.x / 32);
    if (j >= hdr->n_lassos) return;  // uniform over the warp
    if (!LCL_IN(j, caps.lassos)) return;
    (void)caps;
    const BLassoIn &L = in[j];
    LassoArg &p = out[j].arg;
    if (lane == 0) {
        lasso_arg_head(p, L.m, L.w_s, L.h_s, L.poly, L.nv, L.label, L.bias);
        out[j].depth = L.depth;
        out[j].pad_r = (int32_t)(L.flags & 15u);
        out[j].pad_t = (int32_t)((L.flags >> 4) & 15u);
    }
    __syncwarp();
    const double bh = lasso_band_height(p);
    const int nv = p.nv;
    int c = 0;
    for (int e = 0; e < nv; ++e) c += lasso_band_has(p, lane, e, bh) ? 1 : 0;
    int incl = c;
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    int k = incl - c;
    p.band_off[lane] = (uint16_t)k;
    if (lane == 31) p.band_off[kBands] = (uint16_t)incl;
    for (int e = 0; e < nv; ++e)
        if (lasso_band_has(p, lane, e, bh)) p.band_edge[k++] = (uint8_t)e;
}

// Masks of one (super-tile, stroke) unit: unit u is super-tile u / 64 of the batch and stroke u % 64
// of its model, so the tile tests of one super-tile and all its strokes run in parallel (a thread
// per tile, a CTA per unit) rather than one after another in one thread.  A stroke whose test can
// reach the super-tile tests each of its 256 tiles and ORs its bit into the tile's mask (and, for an
// exact class, into `sure`).
__global__ void __launch_bounds__(kThreads) k_batch_pairs(const BHdr *__restrict__ hdr,
                                                          const BModel *__restrict__ models,
                                                          const BStroke *__restrict__ strokes,
                                                          const BLasso *__restrict__ lassos,
                                                          const uint32_t *__restrict__ super_model,
                                                          ulonglong2 *__restrict__ tmask, BCaps caps) {
    pdl_wait();  // the tile masks are cleared and the lassos built
    pdl_allow_next();
    __shared__ int s_reach;
    const int64_t n_units = (int64_t)hdr->n_supers * 64;
    for (int64_t u = blockIdx.x; u < n_units; u += gridDim.x) {  // uniform over the CTA
        const int32_t g = (int32_t)(u >> 6), k = (int32_t)(u & 63);
        if (!LCL_IN(g, caps.supers)) break;
        const uint32_t mi = super_model[g];
        if (!LCL_IN(mi, caps.models)) continue;
        const BModel &M = models[mi];
        if (k >= M.ns) continue;
        if (!stroke_in_bounds(strokes, (int64_t)M.s0 + k, caps)) continue;
        const AtlasDev &a = M.a;
        const int32_t sidx = g - M.super0;
        if (!LCL_IN(sidx, (int64_t)a.supers_x * a.supers_y)) continue;
        const int32_t sx = sidx % a.supers_x, sy = sidx / a.supers_x;
        const BStroke &st = strokes[M.s0 + k];
        __syncthreads();  // s_reach of the previous unit has been read
        if (threadIdx.x == 0) s_reach = stroke_may_reach(st, lassos, a.super_box, a.supers_x, a.supers_y, sx, sy);
        __syncthreads();
        if (!s_reach) continue;
        const int32_t tx = sx * LCL_SUPER + (threadIdx.x % LCL_SUPER);
        const int32_t ty = sy * LCL_SUPER + (threadIdx.x / LCL_SUPER);
        if (tx >= a.tiles_x || ty >= a.tiles_y) continue;
        const int64_t tile = (int64_t)ty * a.tiles_x + tx;
        bool hit = false, sure = false;
        if (!stroke_pads(st, lassos) && LCL_IN(tile, (int64_t)a.tiles_x * a.tiles_y)) {
            // unpadded: the tile's own box decides, with its exact class
            const int4 *b = reinterpret_cast<const int4 *>(a.tile_box + 8 * tile);
            const int4 lo = b[0], hi = b[1];
            if (lo.w == 0) continue;
            if (st.kind == LCL_STROKE_SPHERE) {
                hit = box_dist2(lo, hi, st.sphere) <= st.sphere.r2;
                sure = hit && box_far2(lo, hi, st.sphere) <= st.sphere.r2;
            } else {
                const BLasso &L = lassos[st.lasso];
                float4 sb;
                if (box_may_touch(L.arg, lo, hi, L.depth, &sb)) {
                    const int cls = lasso_tile_class8<1>(L.arg, L.arg.vx, L.arg.vy, sb);
                    hit = cls != kTileOut;
                    sure = cls == kTileIn;
                }
            }
        } else {
            hit = stroke_may_reach(st, lassos, a.tile_box, a.tiles_x, a.tiles_y, tx, ty);
        }
        if (hit && LCL_IN(M.tile0 + tile, caps.tiles)) {
            atomicOr(&tmask[M.tile0 + tile].x, 1ull << k);
            if (sure) atomicOr(&tmask[M.tile0 + tile].y, 1ull << k);
        }
    }
}

// Work items: every tile whose mask is not empty becomes (model, tile, mask, sure); a CTA per
// super-tile, a thread per tile.
__global__ void __launch_bounds__(kThreads) k_batch_compact(const BHdr *__restrict__ hdr,
                                                            const BModel *__restrict__ models,
                                                            const uint32_t *__restrict__ super_model,
                                                            const ulonglong2 *__restrict__ tmask, BItem *items,
                                                            unsigned int *n_items, BCaps caps) {
    pdl_wait();  // the masks are complete
    pdl_allow_next();
    const int32_t n_supers = hdr->n_supers;
    for (int32_t g = blockIdx.x; g < n_supers; g += gridDim.x) {
        if (!LCL_IN(g, caps.supers)) break;  // uniform over the CTA
        const uint32_t mi = super_model[g];
        if (!LCL_IN(mi, caps.models)) continue;
        const BModel &M = models[mi];
        const AtlasDev &a = M.a;
        const int32_t sidx = g - M.super0;
        if (!LCL_IN(sidx, (int64_t)a.supers_x * a.supers_y)) continue;
        const int32_t sx = sidx % a.supers_x, sy = sidx / a.supers_x;
        const int32_t tx = sx * LCL_SUPER + (threadIdx.x % LCL_SUPER);
        const int32_t ty = sy * LCL_SUPER + (threadIdx.x / LCL_SUPER);
        ulonglong2 m = make_ulonglong2(0ull, 0ull);
        const int64_t tile = (int64_t)ty * a.tiles_x + tx;
        if (tx < a.tiles_x && ty < a.tiles_y && LCL_IN(M.tile0 + tile, caps.tiles)) m = tmask[M.tile0 + tile];
        const bool cand = m.x != 0ull;
        const uint32_t bal = __ballot_sync(0xffffffffu, cand);
        if (bal) {
            const int lane = threadIdx.x & 31;
            uint32_t base = 0;
            if (lane == __ffs(bal) - 1) base = atomicAdd(n_items, (unsigned)__popc(bal));
            base = __shfl_sync(0xffffffffu, base, __ffs(bal) - 1);
            const uint32_t slot = base + __popc(bal & ((1u << lane) - 1));
            if (cand && LCL_IN(slot, caps.tiles)) {
                BItem it;
                it.model = mi;
                it.tile = (uint32_t)tile;
                it.mask = m.x;
                it.sure = m.y;
                items[slot] = it;
            }
        }
    }
}

// Does stroke `st` select the covered texel n?
__device__ __forceinline__ bool stroke_selects(const AtlasDev &a, const BStroke &st, const BLasso *__restrict__ lassos,
                                               int64_t n, int32_t qx) {
    if (st.kind == LCL_STROKE_SPHERE) {
        const int64_t dx = (int64_t)qx - st.sphere.cx, dy = (int64_t)__ldg(a.py + n) - st.sphere.cy;
        const int64_t dz = (int64_t)__ldg(a.pz + n) - st.sphere.cz;
        return dx * dx + dy * dy + dz * dz <= st.sphere.r2;
    }
    const BLasso &ls = lassos[st.lasso];
    return lasso_hit(ls.arg, ls.arg, ls.depth, qx, __ldg(a.py + n), __ldg(a.pz + n));
}

// Texture padding of the uncovered texels `unc` of the quad at l: for each, the masked padded strokes
// from the newest down; the first whose outline (a covered texel within its thickness) and kernel
// (a texel it selects within its radius) both hold gives the label.  Returns the texels written.
__device__ __noinline__ uint32_t pad_texels(const AtlasDev &a, int64_t l, uint32_t unc, unsigned long long mask, int32_t s0,
                               const BStroke *__restrict__ strokes, const BLasso *__restrict__ lassos,
                               uint32_t lab[4], const BCaps &caps) {
    const int32_t x0 = (int32_t)(l % a.w), y0 = (int32_t)(l / a.w);
    uint32_t written = 0u;
#pragma unroll 1
    for (int k = 0; k < 4; ++k) {
        if (!(unc & (1u << k))) continue;
        for (unsigned long long m = mask; m; ) {
            const int si = 63 - __clzll((long long)m);  // newest stroke left
            m &= ~(1ull << si);
            if (!stroke_in_bounds(strokes, (int64_t)s0 + si, caps)) continue;
            const BStroke &st = strokes[s0 + si];
            const int32_t pr = st.kind == LCL_STROKE_SPHERE ? st.sphere.pad_r : lassos[st.lasso].pad_r;
            if (pr == 0) continue;
            const int32_t pt = st.kind == LCL_STROKE_SPHERE ? st.sphere.pad_t : lassos[st.lasso].pad_t;
            const int32_t reach = max(pr, pt);
            bool outline = false, near = false;
            for (int32_t dy = -reach; dy <= reach && !(outline && near); ++dy) {
                const int32_t yy = y0 + dy;
                if (yy < 0 || yy >= a.h) continue;
                for (int32_t dx = -reach; dx <= reach; ++dx) {
                    const int32_t xx = x0 + k + dx;
                    if (xx < 0 || xx >= a.w) continue;
                    const int64_t n = (int64_t)yy * a.w + xx;
                    if (!LCL_IN(n, (int64_t)a.w * a.h)) continue;
                    const int32_t qx = __ldg(a.px + n);
                    if (qx == INT32_MIN) continue;
                    const int32_t ax = abs(dx), ay = abs(dy);
                    if (ax <= pt && ay <= pt) outline = true;
                    if (ax <= pr && ay <= pr && !near) near = stroke_selects(a, st, lassos, n, qx);
                }
            }
            if (outline && near) {
                lab[k] = st.kind == LCL_STROKE_SPHERE ? st.sphere.label : lassos[st.lasso].arg.label;
                written |= 1u << k;
                break;
            }
        }
    }
    return written;
}

// Quads [q0, q1) of a work item's tile (quad = 4 consecutive texels of a tile row, row-major in
// the tile), one per thread per pass.
template <typename L>
__device__ __forceinline__ void apply_part(const BModel &M, const BItem &it, int32_t q0, int32_t q1,
                                           const BStroke *__restrict__ strokes, const BLasso *__restrict__ lassos,
                                           const BCaps &caps) {
    const AtlasDev &a = M.a;
    L *layer = static_cast<L *>(M.layer);
    if (!LCL_IN(it.tile, (int64_t)a.tiles_x * a.tiles_y)) return;
    int32_t tx, ty;
    tile_xy(a, it.tile, tx, ty);
    const int32_t qpr = a.T / 4;
    for (int32_t qd = q0 + (int32_t)threadIdx.x; qd < q1; qd += (int32_t)blockDim.x) {
        const int32_t x = tx * a.T + 4 * (qd & (qpr - 1)), y = ty * a.T + (qd >> (__ffs(qpr) - 1));
        if (x >= a.w || y >= a.h) continue;
        const int64_t l = (int64_t)y * a.w + x;
        if (!LCL_IN(l + 3, (int64_t)a.w * a.h)) continue;
        const int4 X = __ldg(reinterpret_cast<const int4 *>(a.px + l));
        const int4 Y = __ldg(reinterpret_cast<const int4 *>(a.py + l));
        const int4 Z = __ldg(reinterpret_cast<const int4 *>(a.pz + l));
        const int32_t xs[4] = {X.x, X.y, X.z, X.w}, ys[4] = {Y.x, Y.y, Y.z, Y.w}, zs[4] = {Z.x, Z.y, Z.z, Z.w};
        // uncovered texels (x = INT32_MIN) are never selected: they start final
        uint32_t open = 0u;
#pragma unroll
        for (int k = 0; k < 4; ++k) open |= (xs[k] != INT32_MIN ? 1u : 0u) << k;
        uint32_t lab[4] = {0u, 0u, 0u, 0u}, hit = 0u;
        for (unsigned long long m = it.mask; m && open; ) {
            const int si = 63 - __clzll((long long)m);  // newest stroke left
            m &= ~(1ull << si);
            if (!stroke_in_bounds(strokes, (int64_t)M.s0 + si, caps)) continue;
            const BStroke &st = strokes[M.s0 + si];
            uint32_t sel = 0u;
            const bool sure = (it.sure >> si) & 1ull;
            if (st.kind == LCL_STROKE_SPHERE) {
                if (sure) {
                    sel = open;  // the sphere contains the tile's box: every covered texel is selected
                } else {
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const int64_t dx = (int64_t)xs[k] - st.sphere.cx, dy = (int64_t)ys[k] - st.sphere.cy;
                        const int64_t dz = (int64_t)zs[k] - st.sphere.cz;
                        sel |= (dx * dx + dy * dy + dz * dz <= st.sphere.r2 ? 1u : 0u) << k;
                    }
                    sel &= open;
                }
                if (sel) {
#pragma unroll
                    for (int k = 0; k < 4; ++k)
                        if (sel & (1u << k)) lab[k] = st.sphere.label;
                }
            } else {
                const BLasso &ls = lassos[st.lasso];
#pragma unroll 1
                for (int k = 0; k < 4; ++k) {  // selects, not a runtime index into the arrays
                    if (!(open & (1u << k))) continue;
                    const int32_t qx = k == 0 ? X.x : k == 1 ? X.y : k == 2 ? X.z : X.w;
                    const int32_t qy = k == 0 ? Y.x : k == 1 ? Y.y : k == 2 ? Y.z : Y.w;
                    const int32_t qz = k == 0 ? Z.x : k == 1 ? Z.y : k == 2 ? Z.z : Z.w;
                    if (sure ? lasso_hit<true>(ls.arg, ls.arg, ls.depth, qx, qy, qz)
                             : lasso_hit<false>(ls.arg, ls.arg, ls.depth, qx, qy, qz))
                        sel |= 1u << k;
                }
                const uint32_t label = ls.arg.label;
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    if (sel & (1u << k)) lab[k] = label;
            }
            hit |= sel;
            open &= ~sel;
        }
        // texture padding (Section 4.3.2) of the quad's uncovered texels: the newest padded stroke
        // that selects a texel within its kernel radius, with a covered texel within its outline
        // thickness, writes its label there
        uint32_t unc = 0u;
#pragma unroll
        for (int k = 0; k < 4; ++k) unc |= (xs[k] == INT32_MIN ? 1u : 0u) << k;
        if (unc) {
            const uint32_t ph = pad_texels(a, l, unc, it.mask, M.s0, strokes, lassos, lab, caps);
            hit |= ph;
        }
        if (hit) store_labels<L>(layer, l, hit, lab);
    }
}

__global__ void __launch_bounds__(256, 3) k_batch_apply(const BHdr *__restrict__ hdr, const BModel *__restrict__ models,
                                                     const BStroke *__restrict__ strokes,
                                                     const BLasso *__restrict__ lassos,
                                                     const BItem *__restrict__ items, unsigned long long *next_unit,
                                                     int32_t split, BCaps caps) {
    pdl_wait();
    pdl_allow_next();
    __shared__ unsigned long long s_unit;
    const unsigned long long n_units = (unsigned long long)hdr->n_items * (unsigned)split;
    for (;;) {
        if (threadIdx.x == 0) s_unit = atomicAdd(next_unit, 1ull);
        __syncthreads();
        const unsigned long long u = s_unit;
        __syncthreads();
        if (u >= n_units) break;  // uniform over the CTA
        if (!LCL_IN(u / (unsigned)split, caps.tiles)) continue;
        const BItem it = items[u / (unsigned)split];
        const int32_t part = (int32_t)(u % (unsigned)split);
        if (!LCL_IN(it.model, caps.models)) continue;
        const BModel &M = models[it.model];
        const int32_t nq = M.a.T * (M.a.T / 4), per = nq / split;  // nq is a power of 2 >= 16
        if (M.dtype_bytes == 1)
            apply_part<uint8_t>(M, it, part * per, (part + 1) * per, strokes, lassos, caps);
        else
            apply_part<uint16_t>(M, it, part * per, (part + 1) * per, strokes, lassos, caps);
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
        // a band of a texture's rows cannot pad (padding reads up to 8 rows beyond the band)
        const bool band = a->tex_height > 0 && a->height != a->tex_height;
        for (int32_t k = 0; k < m.n_strokes; ++k) {
            const lcl_batch_stroke &s = strokes[m.first_stroke + k];
            if (s.kind == LCL_STROKE_SPHERE) {
                const lcl_sphere &sp = s.sphere;
                const int32_t lo = -(1 << 22), hi = (1 << 22) + (1 << 21);
                if (sp.r2 < 0 || sp.label > lab_max || sp.cx < lo || sp.cx > hi || sp.cy < lo || sp.cy > hi ||
                    sp.cz < lo || sp.cz > hi || (sp.flags & ~0xFFu) || (sp.flags & 15u) > 8 ||
                    ((sp.flags >> 4) & 15u) > 8)
                    return fail(LCL_ERR_INVALID_ARG, "batch sphere stroke out of range");
                if (band && (sp.flags & 15u))
                    return fail(LCL_ERR_UNSUPPORTED, "texture padding needs the whole texture, not a band of its rows");
            } else if (s.kind == LCL_STROKE_LASSO) {
                if (s.lasso < 0 || s.lasso >= n_lassos) return fail(LCL_ERR_INVALID_ARG, "batch lasso index");
                if (lassos[s.lasso].label > lab_max) return fail(LCL_ERR_INVALID_ARG, "batch lasso label too wide");
                if (band && (lassos[s.lasso].flags & 15u))
                    return fail(LCL_ERR_UNSUPPORTED, "texture padding needs the whole texture, not a band of its rows");
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
        if ((L.flags & ~0xFFu) || (L.flags & 15u) > 8 || ((L.flags >> 4) & 15u) > 8)
            return fail(LCL_ERR_INVALID_ARG, "batch lasso flags: padding radius and thickness at most 8");
    }
    if (ns > INT32_MAX || nt > UINT32_MAX) return fail(LCL_ERR_UNSUPPORTED, "batch too large");
    *n_supers = ns;
    *n_tiles = nt;
    return LCL_OK;
}

bool limits_ok(const lcl_batch_limits *lim) {
    return lim && lim->models >= 0 && lim->strokes >= 0 && lim->lassos >= 0 && lim->supers >= 0 &&
           lim->supers <= INT32_MAX && lim->tiles >= 0 && lim->tiles <= (int64_t)UINT32_MAX;
}

bool config_ok(const lcl_batch_config &c) {
    return (c.threads == 64 || c.threads == 128 || c.threads == 256) && c.ctas_per_sm >= 0 && c.ctas_per_sm <= 32 &&
           (c.split == 1 || c.split == 2 || c.split == 4 || c.split == 8);
}

lcl_batch_config default_config() {
    lcl_batch_config c;
    std::memset(&c, 0, sizeof(c));
    c.threads = 256;
    c.ctas_per_sm = 0;
    c.split = 1;
    return c;
}

struct BPtrs {
    BHdr *hdr;
    const BModel *models;
    const BStroke *strokes;
    const BLassoIn *lasso_in;
    BLasso *lassos;
    const uint32_t *super_model;
    BItem *items;
    ulonglong2 *tmask;
};

BPtrs b_ptrs(const BLayout &L, void *ws) {
    char *base = static_cast<char *>(ws);
    BPtrs p;
    p.hdr = reinterpret_cast<BHdr *>(base + L.hdr);
    p.models = reinterpret_cast<const BModel *>(base + L.models);
    p.strokes = reinterpret_cast<const BStroke *>(base + L.strokes);
    p.lasso_in = reinterpret_cast<const BLassoIn *>(base + L.lasso_in);
    p.lassos = reinterpret_cast<BLasso *>(base + L.lassos);
    p.super_model = reinterpret_cast<const uint32_t *>(base + L.super_model);
    p.items = reinterpret_cast<BItem *>(base + L.items);
    p.tmask = reinterpret_cast<ulonglong2 *>(base + L.tmask);
    return p;
}

cudaError_t launch_kernels(const BPtrs &p, const lcl_batch_limits &lim, const lcl_batch_config &c, cudaStream_t st) {
    BCaps caps;
    caps.models = lim.models;
    caps.strokes = lim.strokes;
    caps.lassos = lim.lassos;
    caps.pad = 0;
    caps.supers = lim.supers;
    caps.tiles = lim.tiles;
    // enough CTAs for the lassos (a warp each) and for clearing the tile masks
    const int pg = (int)std::max<int64_t>((std::max(lim.lassos, 1) + kPrepWarps - 1) / kPrepWarps,
                                          std::min<int64_t>((lim.tiles + kThreads - 1) / kThreads, 4 * sm_count()));
    k_batch_prep<<<pg, kThreads, 0, st>>>(p.hdr, p.lasso_in, p.lassos, p.tmask, caps);
    cudaError_t e = cudaSuccess;
    if (lim.supers > 0) {
        const int ug = (int)std::min<int64_t>(lim.supers * 64, resident_grid(k_batch_pairs));
        e = launch_pdl(k_batch_pairs, dim3(ug), st, (const BHdr *)p.hdr, p.models, p.strokes, p.lassos, p.super_model,
                       p.tmask, caps);
        const int cg = (int)std::min<int64_t>(lim.supers, resident_grid(k_batch_compact));
        if (e == cudaSuccess)
            e = launch_pdl(k_batch_compact, dim3(cg), st, (const BHdr *)p.hdr, p.models, p.super_model,
                           (const ulonglong2 *)p.tmask, p.items, &p.hdr->n_items, caps);
        if (e == cudaSuccess) {
            const int fit = resident_per_sm(k_batch_apply, c.threads);
            const int per_sm = c.ctas_per_sm > 0 ? std::min(c.ctas_per_sm, fit) : fit;
            e = launch_pdl_shape(k_batch_apply, dim3(per_sm * sm_count()), dim3(c.threads), st, (const BHdr *)p.hdr,
                                 p.models, p.strokes, p.lassos, (const BItem *)p.items, &p.hdr->next_unit,
                                 (int32_t)c.split, caps);
        }
    }
    count_launches(lim.supers > 0 ? 4 : 1);
    if (e == cudaSuccess) e = cudaGetLastError();
    return e;
}

}  // namespace

lcl_status batch_limits_of(const lcl_batch_model *models, int32_t n_models, int32_t n_strokes, int32_t n_lassos,
                           lcl_batch_limits *out) {
    if (!out || n_models < 0 || n_strokes < 0 || n_lassos < 0 || (n_models && !models))
        return fail(LCL_ERR_INVALID_ARG, "batch limits: bad counts or NULL");
    int64_t ns = 0, nt = 0;
    for (int32_t i = 0; i < n_models; ++i) {
        const lcl_atlas *a = models[i].atlas;
        if (!a || a->tiles_x <= 0 || a->tiles_y <= 0) return fail(LCL_ERR_INVALID_ARG, "batch model without atlas");
        ns += (int64_t)a->supers_x * a->supers_y;
        nt += (int64_t)a->tiles_x * a->tiles_y;
    }
    std::memset(out, 0, sizeof(*out));
    out->models = n_models;
    out->strokes = n_strokes;
    out->lassos = n_lassos;
    out->supers = ns;
    out->tiles = nt;
    if (!limits_ok(out)) return fail(LCL_ERR_UNSUPPORTED, "batch too large");
    return LCL_OK;
}

size_t batch_ws_bytes(const lcl_batch_limits *lim) { return limits_ok(lim) ? b_layout(*lim).total : 0; }

size_t batch_host_bytes(const lcl_batch_limits *lim) { return limits_ok(lim) ? b_layout(*lim).upload : 0; }

namespace {
__global__ void k_copy16(uint4 *__restrict__ dst, const uint4 *__restrict__ src, int64_t n16) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n16; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = src[i];
}
}  // namespace

cudaError_t copy_by_kernel(void *dst, const void *src, size_t n, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    const int64_t n16 = (int64_t)(n / 16);
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((n16 + kThreads - 1) / kThreads, 2 * sm_count()));
    k_copy16<<<grid, kThreads, 0, st>>>(static_cast<uint4 *>(dst), static_cast<const uint4 *>(src), n16);
    count_launches(1);
    return cudaGetLastError();
}

// staging_dev: the device address of host_staging (pinned, mapped) or NULL; with it the descriptors
// go to the workspace by a copy kernel instead of the copy engines.
lcl_status batch_upload_impl(const lcl_batch_limits *lim, const lcl_batch_model *models, int32_t n_models,
                             const lcl_batch_stroke *strokes, int32_t n_strokes, const lcl_batch_lasso *lassos,
                             int32_t n_lassos, void *ws, size_t ws_bytes, void *host_staging, size_t host_bytes,
                             cudaStream_t st, const void *staging_dev) {
    if (!limits_ok(lim)) return fail(LCL_ERR_INVALID_ARG, "batch limits out of range");
    if (!ws || !host_staging) return fail(LCL_ERR_INVALID_ARG, "batch workspace or staging is NULL");
    int64_t n_supers = 0, n_tiles = 0;
    lcl_status s = check_batch(models, n_models, strokes, n_strokes, lassos, n_lassos, &n_supers, &n_tiles);
    if (s != LCL_OK) return s;
    if (n_models > lim->models || n_strokes > lim->strokes || n_lassos > lim->lassos || n_supers > lim->supers ||
        n_tiles > lim->tiles)
        return fail(LCL_ERR_INVALID_ARG, "batch exceeds the workspace limits");
    const BLayout L = b_layout(*lim);
    if (ws_bytes < L.total) return fail(LCL_ERR_OUT_OF_MEMORY, "batch workspace smaller than lcl_batch_workspace_bytes");
    if (host_bytes < L.upload) return fail(LCL_ERR_OUT_OF_MEMORY, "batch staging smaller than lcl_batch_staging_bytes");
    char *img = static_cast<char *>(host_staging);  // image of the uploaded part of the workspace
    const size_t head = L.models + (size_t)n_models * sizeof(BModel);  // header + models
    std::memset(img, 0, head);
    BHdr hdr;
    std::memset(&hdr, 0, sizeof(hdr));
    hdr.n_models = n_models;
    hdr.n_strokes = n_strokes;
    hdr.n_lassos = n_lassos;
    hdr.n_supers = (int32_t)n_supers;
    hdr.n_tiles = (uint32_t)n_tiles;
    std::memcpy(img + L.hdr, &hdr, sizeof(hdr));
    BModel *bm = reinterpret_cast<BModel *>(img + L.models);
    uint32_t *super_model = reinterpret_cast<uint32_t *>(img + L.super_model);
    int32_t super0 = 0;
    int64_t tile0 = 0;
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
        d.tile0 = tile0;
        bm[i] = d;
        tile0 += (int64_t)m.atlas->tiles_x * m.atlas->tiles_y;
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
        d.sphere.pad_r = (int32_t)(strokes[k].sphere.flags & 15u);
        d.sphere.pad_t = (int32_t)((strokes[k].sphere.flags >> 4) & 15u);
        bs[k] = d;
    }
    BLassoIn *bl = reinterpret_cast<BLassoIn *>(img + L.lasso_in);
    for (int32_t j = 0; j < n_lassos; ++j) {
        BLassoIn &d = bl[j];
        std::memcpy(d.m, lassos[j].camera.m, sizeof(d.m));
        d.w_s = lassos[j].camera.width;
        d.h_s = lassos[j].camera.height;
        d.depth = lassos[j].depth;
        std::memcpy(d.poly, lassos[j].poly_xy, sizeof(float) * 2 * (size_t)lassos[j].n_vertices);
        d.nv = lassos[j].n_vertices;
        d.label = lassos[j].label;
        d.bias = lassos[j].bias;
        d.flags = lassos[j].flags;
    }
    // the used front of each region (the kernels read no further; the limits may be far larger)
    const size_t part[4][2] = {{0, head},
                               {L.strokes, (size_t)n_strokes * sizeof(BStroke)},
                               {L.lasso_in, (size_t)n_lassos * sizeof(BLassoIn)},
                               {L.super_model, (size_t)n_supers * 4}};
    char *dst = static_cast<char *>(ws);
    for (const auto &pc : part) {
        if (pc[1] == 0) continue;
        // by kernel: whole 16-byte words (regions are 256-byte aligned and sized, so rounding up stays
        // inside the region in both images)
        const cudaError_t e = staging_dev ? copy_by_kernel(dst + pc[0], static_cast<const char *>(staging_dev) + pc[0],
                                                           (pc[1] + 15) & ~size_t(15), st)
                                          : cudaMemcpyAsync(dst + pc[0], img + pc[0], pc[1], cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return cuda_fail(e, "batch descriptor upload");
    }
    return LCL_OK;
}

lcl_status batch_launch_impl(const lcl_batch_limits *lim, const lcl_batch_config *cfg, void *ws, size_t ws_bytes,
                             cudaStream_t st) {
    if (!limits_ok(lim)) return fail(LCL_ERR_INVALID_ARG, "batch limits out of range");
    const lcl_batch_config c = cfg ? *cfg : default_config();
    if (!config_ok(c)) return fail(LCL_ERR_INVALID_ARG, "batch config: threads 64/128/256, split 1/2/4/8, ctas_per_sm 0..32");
    const BLayout L = b_layout(*lim);
    if (!ws || ws_bytes < L.total) return fail(LCL_ERR_INVALID_ARG, "batch workspace NULL or smaller than the limits need");
    const cudaError_t e = launch_kernels(b_ptrs(L, ws), *lim, c, st);
    if (e != cudaSuccess) return cuda_fail(e, "batch launch");
    return LCL_OK;
}

lcl_status batch_tune_impl(const lcl_batch_limits *lim, void *ws, size_t ws_bytes, int32_t reps, cudaStream_t st,
                           lcl_batch_config *best, float *best_ms) {
    if (!best || reps < 1 || reps > 100) return fail(LCL_ERR_INVALID_ARG, "batch tune: best is NULL or reps not in 1..100");
    if (!limits_ok(lim)) return fail(LCL_ERR_INVALID_ARG, "batch limits out of range");
    const BLayout L = b_layout(*lim);
    if (!ws || ws_bytes < L.total) return fail(LCL_ERR_INVALID_ARG, "batch workspace NULL or smaller than the limits need");
    const BPtrs p = b_ptrs(L, ws);
    const int fit256 = resident_per_sm(k_batch_apply, 256);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float t_best = INFINITY;
    lcl_batch_config c_best = default_config();
    const int threads[3] = {64, 128, 256}, splits[4] = {1, 2, 4, 8};
    for (int ti = 0; ti < 3 && e == cudaSuccess; ++ti)
        for (int si = 0; si < 4 && e == cudaSuccess; ++si)
            for (int half = 0; half < 2 && e == cudaSuccess; ++half) {
                lcl_batch_config c = default_config();
                c.threads = threads[ti];
                c.split = splits[si];
                const int fit = resident_per_sm(k_batch_apply, c.threads);
                c.ctas_per_sm = half ? std::max(1, fit / 2) : 0;
                if (half && c.ctas_per_sm >= fit) continue;
                (void)fit256;
                e = launch_kernels(p, *lim, c, st);  // warm-up
                if (e == cudaSuccess) e = cudaEventRecord(e0, st);
                for (int r = 0; r < reps && e == cudaSuccess; ++r) e = launch_kernels(p, *lim, c, st);
                if (e == cudaSuccess) e = cudaEventRecord(e1, st);
                if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                float ms = 0.0f;
                if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
                if (e == cudaSuccess && ms / reps < t_best) {
                    t_best = ms / reps;
                    c_best = c;
                }
            }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess) return cuda_fail(e, "batch tune");
    *best = c_best;
    if (best_ms) *best_ms = t_best;
    return LCL_OK;
}

}  // namespace lcl
