// select.cu -- per-texel selection edits: the sphere brush and the screen-space lasso
// (arXiv 2501.14807, Section 4.3.1, Fig. 3: depth test, projection of the tool, shape mask,
// then the selected value is stored in the texels that survive).
//
// Culling: a stroke is tested against the box of every super-tile (16 x 16 tiles); where the
// super-tile's box can touch the stroke, each of its tiles' boxes is tested, one per thread, and
// the candidate tiles are appended to a list with one atomic per warp (ballot + popc).  Both
// tests are conservative, so culling never changes a result.
//
// Apply: a resident grid (as many CTAs as fit on the SMs) walks the candidate list; each thread
// owns four consecutive texels of a tile row: three 16-byte loads of the position planes, the
// per-texel test, and one 4-byte (uint8) or 8-byte (uint16) label word written only if a texel in
// it was hit (read first only if some of its texels were not).  The loads of the thread's next
// work item are issued before the current one is tested, so two items are in flight per thread.
// Measured on GB300 (1000 strokes on a 16384^2 atlas): culling the next stroke before the wait
// (below) rather than after the apply loop saves ~0.65 us per stroke; culling two strokes ahead
// over four lists so that a grid could also read its counter, list and first work item before
// its wait cost ~2.2 us per stroke; reading the candidate list two items ahead, or a padding
// branch that raises the kernel above 40 registers (5 instead of 6 CTAs per SM), cost 1.3-1.6 ms
// per 1000 strokes, hence the separate template instances.
//
// Sphere strokes take one launch each: the kernel that applies stroke k also culls stroke k + 1,
// and every launch is a programmatic dependent launch, so the next grid is scheduled while the
// current one drains and waits (griddepcontrol.wait) only for its completion.  Stroke k's
// candidates go to list k mod 3, and the cull of stroke k + 1 runs before the wait, in the
// shadow of stroke k - 1's tail: list (k + 1) mod 3 was last read by stroke k - 2, which has
// completed, because grid k is only launched once every CTA of grid k - 1 has passed its own
// wait.  Strokes of one call run in stream order, so a later stroke overwrites an earlier one.  Lassos take a cull and an apply launch (two culls with texture padding).  Hit counts are per-warp popcounts
// reduced per CTA into one 64-bit atomic.
#include <algorithm>
#include <cmath>

#include "select_common.cuh"

namespace lcl {
namespace {

// Zeroes n counters and the first n_hits of `hits` (nullable).
__global__ void k_sel_init(uint32_t *counters, int32_t n, unsigned long long *hits, int32_t n_hits) {
    pdl_wait();  // launched as a dependent: the previous grid no longer reads the counters
    pdl_allow_next();
    const int32_t end = max(n, hits ? n_hits : 0);
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < end; i += gridDim.x * blockDim.x) {
        if (i < n && LCL_IN(i, n)) counters[i] = 0;
        if (hits && i < n_hits) hits[i] = 0;
    }
}

// Culls stroke s against super-tile `sidx`, appending its candidate tiles.  Uniform per CTA.
// With texture padding (PAD) a texel may be written because a neighbour within 8 texels was
// selected, so a tile (super-tile) is then a candidate if any box of its 3 x 3 neighbourhood is
// in reach.  PAD is a template parameter so that the common case carries no registers for it.
// Tiles inside the sphere go to the back of the list (counter `inside_counter`) when whole-row
// handling applies (`rows`: tile side >= 32 and width a multiple of 32), else to the front with
// kInsideTile set.
template <bool PAD>
__device__ __forceinline__ void cull_super_sphere(const AtlasDev &a, const SphereArg &s, int32_t sidx,
                                                  uint32_t *counter, uint32_t *list, uint32_t *inside_counter,
                                                  bool rows) {
    const int32_t sx = sidx % a.supers_x, sy = sidx / a.supers_x;
    bool in_reach;
    if (PAD) {
        in_reach = near_box_3x3(a.super_box, a.supers_x, a.supers_y, sx, sy, s);
    } else if (LCL_IN(sidx, (int64_t)a.supers_x * a.supers_y)) {
        const int4 *sb = reinterpret_cast<const int4 *>(a.super_box + 8 * (int64_t)sidx);
        const int4 slo = sb[0], shi = sb[1];
        in_reach = slo.w > 0 && box_dist2(slo, shi, s) <= s.r2;
    } else {
        in_reach = false;
    }
    if (!in_reach) return;  // uniform over the CTA
    const int32_t tx = sx * LCL_SUPER + (threadIdx.x % LCL_SUPER);
    const int32_t ty = sy * LCL_SUPER + (threadIdx.x / LCL_SUPER);
    bool cand = false, inside = false;
    const int64_t n_tiles = (int64_t)a.tiles_x * a.tiles_y;
    if (tx < a.tiles_x && ty < a.tiles_y) {
        if (PAD) {
            cand = near_box_3x3(a.tile_box, a.tiles_x, a.tiles_y, tx, ty, s);
        } else if (LCL_IN((int64_t)ty * a.tiles_x + tx, n_tiles)) {
            const int4 *tb = reinterpret_cast<const int4 *>(a.tile_box + 8 * ((int64_t)ty * a.tiles_x + tx));
            const int4 lo = tb[0], hi = tb[1];
            cand = lo.w > 0 && box_dist2(lo, hi, s) <= s.r2;
            // the sphere contains the tile's box: every covered texel of the tile is selected
            inside = cand && box_far2(lo, hi, s) <= s.r2;
        }
    }
    const uint32_t tile = (uint32_t)(ty * a.tiles_x + tx);
    append_candidate(cand && !(inside && rows), tile | (inside ? kInsideTile : 0u), counter, list, n_tiles);
    if (!PAD) append_candidate_back(inside && rows, tile, inside_counter, list, n_tiles);
}

// Culls the first stroke of a call.
__global__ void __launch_bounds__(kThreads) k_sphere_cull(AtlasDev a, SphereArg s, uint32_t *counter,
                                                          uint32_t *list, uint32_t *inside_counter) {
    pdl_wait();
    const int32_t n_super = a.supers_x * a.supers_y;
    const bool rows = a.T >= 32 && (a.w & 31) == 0;
    for (int32_t sidx = blockIdx.x; sidx < n_super; sidx += gridDim.x) {
        if (s.pad_r > 0)
            cull_super_sphere<true>(a, s, sidx, counter, list, inside_counter, rows);
        else
            cull_super_sphere<false>(a, s, sidx, counter, list, inside_counter, rows);
    }
    pdl_allow_next();
}

// One work item = one tile, or a 256-quad chunk of a larger tile; this thread's quad of it.
struct Item {
    int64_t l;     // linear index of the quad's first texel, -1 if the thread has no quad here
    int32_t sure;  // the quad's tile lies inside the sphere: its covered texels (bit k: texel k), else -1
    int4 X, Y, Z;  // positions (loaded only when sure is -1)
};

__device__ __forceinline__ Item load_item(const AtlasDev &a, const uint32_t *__restrict__ list, uint32_t item,
                                          int cpt_log2, int32_t qpr, int32_t nq) {
    Item it;
    it.l = -1;
    it.sure = -1;
    if (!LCL_IN(item >> cpt_log2, (int64_t)a.tiles_x * a.tiles_y)) return it;
    const uint32_t entry = __ldg(list + (item >> cpt_log2));
    const uint32_t tile = entry & ~kInsideTile;
    const int32_t qd = (int32_t)((item & ((1u << cpt_log2) - 1)) * kThreads + threadIdx.x);
    int32_t tx, ty;
    tile_xy(a, tile, tx, ty);
    const int32_t x = tx * a.T + 4 * (qd & (qpr - 1)), y = ty * a.T + (qd >> (__ffs(qpr) - 1));
    if (qd < nq && x < a.w && y < a.h && LCL_IN((int64_t)y * a.w + x + 3, (int64_t)a.w * a.h)) {
        it.l = (int64_t)y * a.w + x;
        if (entry & kInsideTile) {  // inside the sphere: the coverage bits decide, no positions needed
            if (LCL_IN(it.l >> 5, ((int64_t)a.w * a.h + 31) >> 5))
                it.sure = (int32_t)((__ldg(a.cover + (it.l >> 5)) >> (it.l & 31)) & 0xFu);
            else
                it.sure = 0;
        } else {
            it.X = __ldg(reinterpret_cast<const int4 *>(a.px + it.l));
            it.Y = __ldg(reinterpret_cast<const int4 *>(a.py + it.l));
            it.Z = __ldg(reinterpret_cast<const int4 *>(a.pz + it.l));
        }
    }
    return it;
}

// Hit mask of a quad.  Uncovered texels hold x = INT32_MIN, y = z = 0: their squared distance
// exceeds 2^61, above every accepted r2 (<= 2^50), so they never test as hit.
__device__ __forceinline__ uint32_t sphere_mask(const Item &it, const SphereArg &s) {
    if (it.sure >= 0) return (uint32_t)it.sure;
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

// Texture padding (Section 4.3.2) of the uncovered texels of a quad: a texel is written if a
// covered texel lies within the outline thickness (square kernel) and a texel the stroke selects
// lies within the kernel radius.  Neighbours are read from the position planes.
__device__ uint32_t pad_mask(const AtlasDev &a, const Item &it, const SphereArg &s) {
    const int32_t xs[4] = {it.X.x, it.X.y, it.X.z, it.X.w};
    const int32_t x0 = (int32_t)(it.l % a.w), y0 = (int32_t)(it.l / a.w);
    const int32_t reach = max(s.pad_r, s.pad_t);
    uint32_t m = 0;
    for (int k = 0; k < 4; ++k) {
        if (xs[k] != INT32_MIN) continue;
        bool outline = false, near = false;
        for (int32_t dy = -reach; dy <= reach; ++dy) {
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
                if (ax <= s.pad_t && ay <= s.pad_t) outline = true;
                if (ax <= s.pad_r && ay <= s.pad_r && !near) {
                    const int64_t ddx = (int64_t)qx - s.cx, ddy = (int64_t)__ldg(a.py + n) - s.cy;
                    const int64_t ddz = (int64_t)__ldg(a.pz + n) - s.cz;
                    near = ddx * ddx + ddy * ddy + ddz * ddz <= s.r2;
                }
            }
        }
        if (outline && near) m |= 1u << k;
    }
    return m;
}

// Applies stroke `s` from its candidate list and culls stroke `nxt` (if has_next) into the other list.
// PAD: `s` pads the texture; NEXT_PAD: `nxt` does.  NUM: a numeric layer, whose mask bits (vm) are
// set (or cleared) for every texel written.
// Lists: candidate tiles the sphere's surface may cross at the front (`counter` entries), tiles
// inside the sphere at the back (`inside_counter` entries, whole-row layouts only): a warp takes one
// such tile, each lane one 32-texel row segment, whose coverage word says which texels get the label.
template <typename L, bool PAD, bool NEXT_PAD, bool NUM>
__global__ void __launch_bounds__(kThreads, 6) k_sphere_step(AtlasDev a, L *__restrict__ layer, SphereArg s,
                                                          const uint32_t *__restrict__ counter,
                                                          const uint32_t *__restrict__ inside_counter,
                                                          const uint32_t *__restrict__ list,
                                                          unsigned long long *hits, int has_next, SphereArg nxt,
                                                          uint32_t *next_counter, uint32_t *next_inside_counter,
                                                          uint32_t *next_list, ValMask vm) {
    const bool rows = a.T >= 32 && (a.w & 31) == 0;  // uniform
    // Cull of the next stroke: reads only the atlas boxes; its list is free (see the top of the file).
    if (has_next) {
        const int32_t n_super = a.supers_x * a.supers_y;
        for (int32_t sidx = blockIdx.x; sidx < n_super; sidx += gridDim.x)
            cull_super_sphere<NEXT_PAD>(a, nxt, sidx, next_counter, next_list, next_inside_counter, rows);
    }
    pdl_wait();
    pdl_allow_next();  // after the wait: grid k + 1 starts once every CTA of this grid got here
    const int32_t qpr = a.T / 4, nq = a.T * qpr;
    const int cpt_log2 = nq > kThreads ? 31 - __clz(nq / kThreads) : 0;
    const uint32_t n_items = *counter << cpt_log2;
    const bool grouped = a.T >= 32 && (a.w & 31) == 0;  // uniform: see valid_update_warp
    const int64_t n_tex = (int64_t)a.w * a.h;
    (void)n_tex;
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
        if (NUM) {
            uint32_t wm = 0;
            if (cur.l >= 0) {
                const uint32_t m = sphere_mask(cur, s);
                wm = PAD ? (m | pad_mask(a, cur, s)) : m;
                if (wm && LCL_IN(cur.l + 3, n_tex)) store_hits<L>(layer, cur.l, wm, s.label);
                cnt += __popc(m);
            }
            if (grouped) valid_update_warp<true>(vm, cur.l, wm, n_tex);
            else valid_update_warp<false>(vm, cur.l, wm, n_tex);
        } else if (cur.l >= 0) {
            const uint32_t m = sphere_mask(cur, s);
            if (PAD) {
                const uint32_t p = pad_mask(a, cur, s);
                if ((m | p) && LCL_IN(cur.l + 3, n_tex)) store_hits<L>(layer, cur.l, m | p, s.label);
                cnt += __popc(m);
            } else if (m) {
                if (LCL_IN(cur.l + 3, n_tex)) store_hits<L>(layer, cur.l, m, s.label);
                cnt += __popc(m);
            }
        }
        cur = next;
    }
    // tiles inside the sphere: one warp per tile, one lane per 32-texel row segment
    const uint32_t n_in = *inside_counter;
    if (n_in) {  // uniform
        const int64_t cap = (int64_t)a.tiles_x * a.tiles_y;
        const int32_t wpr = a.T >> 5, words = a.T * wpr;  // row segments per tile row and per tile
        const uint32_t warps = gridDim.x * (kThreads / 32);
        // from the last CTA down: when the grid has CTAs to spare, the tiles above go to the first
        // CTAs and these to others, so that neither waits for the other
        for (uint32_t b = (gridDim.x - 1 - blockIdx.x) * (kThreads / 32) + (threadIdx.x >> 5); b < n_in; b += warps) {
            if (!LCL_IN(cap - 1 - (int64_t)b, cap)) break;
            const uint32_t tile = __ldg(list + (cap - 1 - (int64_t)b));
            int32_t tx, ty;
            tile_xy(a, tile, tx, ty);
            for (int32_t wi = threadIdx.x & 31; wi < words; wi += 32) {
                const int32_t x = tx * a.T + 32 * (wi % wpr), y = ty * a.T + wi / wpr;
                if (x >= a.w || y >= a.h) continue;   // x < w implies x + 31 < w (w a multiple of 32)
                const int64_t l = (int64_t)y * a.w + x;
                if (!LCL_IN(l + 31, n_tex)) continue;
                const uint32_t cov = __ldg(a.cover + (l >> 5));
                if (!cov) continue;
                store_word32<L>(layer, l, cov, s.label);
                if (NUM) {  // the row segment's mask word belongs to this lane alone
                    uint32_t *mp = vm.bits + (l >> 5);
                    *mp = vm.set ? (*mp | cov) : (*mp & ~cov);
                }
                cnt += __popc(cov);
            }
        }
    }
    add_hits(hits, cnt);
}

// ---- grouped sphere strokes ----------------------------------------------------------------
//
// A run of up to kGroup consecutive unpadded strokes on a label layer is applied by one cull and one
// apply launch instead of one launch per stroke.  Applying strokes one by one leaves each texel with
// the label of the newest stroke that selects it (older labels are overwritten), so the apply walks a
// texel's strokes from the newest down and writes it once; every stroke is still evaluated for its
// hit count, which does not depend on the order.  Items are (tile, mask, sure): `mask` holds the
// group's strokes whose sphere reaches the tile's box (bit k = stroke k of the group), `sure` those
// of them whose sphere contains the box, so that every covered texel of the tile is selected.  Tiles
// whose strokes are all sure need no positions: with whole-row layouts they go to the back of the
// lists and a warp writes them from the coverage bits, one lane per 32-texel row segment.

constexpr int kGroup = 32;

struct GroupArg {
    int32_t n;     // strokes in the group (<= kGroup)
    int32_t rows;  // whole-row handling of all-sure tiles (tile side >= 32, width a multiple of 32)
    SphereArg s[kGroup];
};

// The three lists hold an item's tile, mask and sure at the same index; front items from index 0
// (count counters[0]), all-sure items from the last index down (count counters[1]).
__device__ __forceinline__ void append_item(bool front, bool back, uint32_t tile, uint32_t mask, uint32_t sure,
                                            uint32_t *counters, uint32_t *tiles, uint32_t *masks, uint32_t *sures,
                                            int64_t cap) {
    const int lane = threadIdx.x & 31;
    const uint32_t fm = __ballot_sync(0xffffffffu, front), bm = __ballot_sync(0xffffffffu, back);
    uint32_t fb = 0, bb = 0;
    if (fm && lane == __ffs(fm) - 1) fb = atomicAdd(counters, (uint32_t)__popc(fm));
    if (bm && lane == __ffs(bm) - 1) bb = atomicAdd(counters + 1, (uint32_t)__popc(bm));
    if (fm) fb = __shfl_sync(0xffffffffu, fb, __ffs(fm) - 1);
    if (bm) bb = __shfl_sync(0xffffffffu, bb, __ffs(bm) - 1);
    int64_t slot = -1;
    if (front) slot = fb + __popc(fm & ((1u << lane) - 1));
    if (back) slot = cap - 1 - (int64_t)(bb + __popc(bm & ((1u << lane) - 1)));
    if ((front || back) && LCL_IN(slot, cap)) {
        tiles[slot] = tile;
        masks[slot] = mask;
        sures[slot] = sure;
    }
}

// ahead = 1 (every group but a call's first): the lists this cull writes were last read by the apply
// two groups back, which had completed before the previous apply started, so the cull runs while the
// previous group's apply is still writing the layer, and waits for it only at its end (the next
// apply starts after this grid completes, hence after the previous apply).  The first group's cull
// waits at once: its counters are being cleared by the grid before it.
__global__ void __launch_bounds__(kThreads) k_group_cull(AtlasDev a, const __grid_constant__ GroupArg g,
                                                         uint32_t *counters, uint32_t *tiles, uint32_t *masks,
                                                         uint32_t *sures, int ahead) {
    if (!ahead) pdl_wait();
    __shared__ uint32_t s_mask;
    const int32_t n_super = a.supers_x * a.supers_y;
    const int64_t n_tiles = (int64_t)a.tiles_x * a.tiles_y;
    for (int32_t sidx = blockIdx.x; sidx < n_super; sidx += gridDim.x) {
        if (threadIdx.x == 0) s_mask = 0u;
        __syncthreads();
        if ((int)threadIdx.x < g.n && LCL_IN(sidx, (int64_t)n_super)) {  // one thread per stroke
            const int4 *sb = reinterpret_cast<const int4 *>(a.super_box + 8 * (int64_t)sidx);
            const int4 slo = sb[0], shi = sb[1];
            const SphereArg &sp = g.s[threadIdx.x];
            if (slo.w > 0 && box_dist2(slo, shi, sp) <= sp.r2) atomicOr(&s_mask, 1u << threadIdx.x);
        }
        __syncthreads();
        const uint32_t smask = s_mask;
        __syncthreads();
        if (!smask) continue;  // uniform over the CTA
        const int32_t sx = sidx % a.supers_x, sy = sidx / a.supers_x;
        const int32_t tx = sx * LCL_SUPER + (threadIdx.x % LCL_SUPER);
        const int32_t ty = sy * LCL_SUPER + (threadIdx.x / LCL_SUPER);
        const int64_t tile = (int64_t)ty * a.tiles_x + tx;
        uint32_t mask = 0u, sure = 0u;
        if (tx < a.tiles_x && ty < a.tiles_y && LCL_IN(tile, n_tiles)) {
            const int4 *tb = reinterpret_cast<const int4 *>(a.tile_box + 8 * tile);
            const int4 lo = tb[0], hi = tb[1];
            if (lo.w > 0) {
                for (uint32_t m = smask; m; m &= m - 1) {
                    const int k = __ffs(m) - 1;
                    const SphereArg &sp = g.s[k];
                    if (box_dist2(lo, hi, sp) > sp.r2) continue;
                    mask |= 1u << k;
                    if (box_far2(lo, hi, sp) <= sp.r2) sure |= 1u << k;
                }
            }
        }
        const bool back = g.rows && mask != 0u && mask == sure;
        append_item(mask != 0u && !back, back, (uint32_t)tile, mask, sure, counters, tiles, masks, sures, n_tiles);
    }
    if (ahead) pdl_wait();
    pdl_allow_next();
}

// A front item's list entry, loaded two items ahead; tile = kNone: none.
struct GEnt {
    uint32_t tile, mask, sure;
};

__device__ __forceinline__ GEnt load_gent(const AtlasDev &a, const uint32_t *__restrict__ tiles,
                                          const uint32_t *__restrict__ masks, const uint32_t *__restrict__ sures,
                                          uint32_t item, uint32_t n_items, int cpt_log2) {
    GEnt e;
    e.tile = kNone;
    e.mask = e.sure = 0u;
    const uint32_t idx = item >> cpt_log2;
    if (item < n_items && LCL_IN(idx, (int64_t)a.tiles_x * a.tiles_y)) {
        e.tile = __ldg(tiles + idx);
        e.mask = __ldg(masks + idx);
        e.sure = __ldg(sures + idx);
    }
    return e;
}

// A front item's quad for this thread, loaded one item ahead: the entry's masks and the raw data --
// positions when some stroke of the item is not sure, else the coverage word -- with nothing that
// waits for them (the coverage bits are taken out when the item is processed).
struct GItem {
    int64_t l;  // -1: no quad for this thread (the masks are still the item's)
    uint32_t mask, sure, cw;
    int4 X, Y, Z;
};

__device__ __forceinline__ GItem load_gquad(const AtlasDev &a, const GEnt &e, uint32_t item, int cpt_log2,
                                            int32_t qpr, int32_t nq) {
    GItem it;
    it.l = -1;
    it.mask = e.mask;
    it.sure = e.sure;
    it.cw = 0u;
    it.X = it.Y = it.Z = make_int4(INT32_MIN, 0, 0, 0);
    if (e.tile == kNone) return it;
    const int32_t qd = (int32_t)((item & ((1u << cpt_log2) - 1)) * kThreads + threadIdx.x);
    int32_t tx, ty;
    tile_xy(a, e.tile, tx, ty);
    const int32_t x = tx * a.T + 4 * (qd & (qpr - 1)), y = ty * a.T + (qd >> (__ffs(qpr) - 1));
    const int64_t n_tex = (int64_t)a.w * a.h;
    (void)n_tex;
    if (qd < nq && x < a.w && y < a.h && LCL_IN((int64_t)y * a.w + x + 3, n_tex)) {
        it.l = (int64_t)y * a.w + x;
        if (it.mask & ~it.sure) {  // uniform over the item
            it.X = __ldg(reinterpret_cast<const int4 *>(a.px + it.l));
            it.Y = __ldg(reinterpret_cast<const int4 *>(a.py + it.l));
            it.Z = __ldg(reinterpret_cast<const int4 *>(a.pz + it.l));
        } else if (LCL_IN(it.l >> 5, (n_tex + 31) >> 5)) {
            it.cw = __ldg(a.cover + (it.l >> 5));
        }
    }
    return it;
}

// The quad's coverage bits (bit k: texel k) from its raw data.
__device__ __forceinline__ uint32_t gquad_cov(const GItem &it) {
    if (it.l < 0) return 0u;
    if (it.mask & ~it.sure)
        return (it.X.x != INT32_MIN ? 1u : 0u) | (it.X.y != INT32_MIN ? 2u : 0u) | (it.X.z != INT32_MIN ? 4u : 0u) |
               (it.X.w != INT32_MIN ? 8u : 0u);
    return (it.cw >> (it.l & 31)) & 0xFu;
}

template <typename L>
__global__ void __launch_bounds__(kThreads, 5) k_group_apply(AtlasDev a, L *__restrict__ layer,
                                                             const __grid_constant__ GroupArg g,
                                                             const uint32_t *__restrict__ counters,
                                                             const uint32_t *__restrict__ tiles,
                                                             const uint32_t *__restrict__ masks,
                                                             const uint32_t *__restrict__ sures,
                                                             unsigned long long *hits) {
    __shared__ unsigned long long s_hits[kGroup];
    if (threadIdx.x < kGroup) s_hits[threadIdx.x] = 0ull;
    __syncthreads();
    pdl_wait();
    pdl_allow_next();
    const int lane = threadIdx.x & 31;
    const int64_t n_tex = (int64_t)a.w * a.h;
    (void)n_tex;
    // front items: a CTA per tile (or 256-quad chunk of one), a thread per quad
    const int32_t qpr = a.T / 4, nq = a.T * qpr;
    const int cpt_log2 = nq > kThreads ? 31 - __clz(nq / kThreads) : 0;
    const uint32_t n_items = counters[0] << cpt_log2;
    // entries two items ahead, quads one item ahead: the position loads of the next item are issued
    // as soon as this item starts, from an entry that arrived during the previous one
    uint32_t item = blockIdx.x;
    GItem cur = load_gquad(a, load_gent(a, tiles, masks, sures, item, n_items, cpt_log2), item, cpt_log2, qpr, nq);
    GEnt e1 = load_gent(a, tiles, masks, sures, item + gridDim.x, n_items, cpt_log2);
    for (; item < n_items; item += gridDim.x) {
        const uint32_t after = item + gridDim.x;
        const GEnt e2 = load_gent(a, tiles, masks, sures, after + gridDim.x, n_items, cpt_log2);
        const GItem next = load_gquad(a, e1, after, cpt_log2, qpr, nq);
        e1 = e2;
        const int32_t xs[4] = {cur.X.x, cur.X.y, cur.X.z, cur.X.w}, ys[4] = {cur.Y.x, cur.Y.y, cur.Y.z, cur.Y.w},
                      zs[4] = {cur.Z.x, cur.Z.y, cur.Z.z, cur.Z.w};
        const uint32_t cov = gquad_cov(cur);
        const int ks = cur.sure ? 31 - __clz(cur.sure) : -1;  // the newest stroke containing the tile
        uint32_t open = cov;
        uint32_t lab[4] = {0u, 0u, 0u, 0u};
        // strokes whose surface crosses the tile, newest first (uniform over the CTA): each is tested
        // per texel for its hit count; only those newer than stroke ks can give a texel its label
        for (uint32_t m = cur.mask & ~cur.sure; m;) {
            const int k = 31 - __clz(m);
            m &= ~(1u << k);
            if (!hits && k < ks) break;  // no counts wanted: stroke ks labels every open texel
            const SphereArg &sp = g.s[k];
            uint32_t sel = 0u;
            if (cur.l >= 0) {
                // The stroke reaches the tile's box (r <= 2^25 and the box inside [0, 2^21)^3), so for a
                // covered texel every coordinate difference lies within +-(2^25 + 2^21) and its square
                // is one 32 x 32 -> 64-bit product.  Uncovered texels (x = INT32_MIN) wrap around in
                // the unsigned difference; the coverage bits drop them.
                const uint32_t cx = (uint32_t)sp.cx, cy = (uint32_t)sp.cy, cz = (uint32_t)sp.cz;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int32_t dx = (int32_t)((uint32_t)xs[q] - cx), dy = (int32_t)((uint32_t)ys[q] - cy),
                                  dz = (int32_t)((uint32_t)zs[q] - cz);
                    const int64_t d2 = (int64_t)dx * dx + (int64_t)dy * dy + (int64_t)dz * dz;
                    sel |= (d2 <= sp.r2 ? 1u : 0u) << q;
                }
                sel &= cov;
            }
            if (hits) {
                const uint32_t c = __reduce_add_sync(0xffffffffu, (uint32_t)__popc(sel));
                if (lane == 0 && c) atomicAdd(&s_hits[k], (unsigned long long)c);
            }
            if (k > ks) {
                const uint32_t nw = sel & open;
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (nw & (1u << q)) lab[q] = sp.label;
                open &= ~sel;
            }
        }
        if (ks >= 0) {  // strokes containing the tile select every covered texel
            const uint32_t label = g.s[ks].label;
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (open & (1u << q)) lab[q] = label;
            open = 0u;
            if (hits) {
                const uint32_t c = __reduce_add_sync(0xffffffffu, (uint32_t)__popc(cov));
                if (lane == 0 && c)
                    for (uint32_t m = cur.sure; m; m &= m - 1) atomicAdd(&s_hits[__ffs(m) - 1], (unsigned long long)c);
            }
        }
        const uint32_t written = cov & ~open;
        if (written && LCL_IN(cur.l + 3, n_tex)) store_labels<L>(layer, cur.l, written, lab);
        cur = next;
    }
    // all-sure items (whole-row layouts): a warp per tile from the far end of the grid, one lane per
    // 32-texel row segment; the newest stroke's label goes to every covered texel
    const uint32_t n_back = counters[1];
    if (n_back) {  // uniform
        const int64_t cap = (int64_t)a.tiles_x * a.tiles_y;
        const int32_t wpr = a.T >> 5, words = a.T * wpr;
        const uint32_t warps = gridDim.x * (kThreads / 32);
        // the next tile's entry is loaded one tile ahead
        auto entry = [&](uint32_t bb, uint32_t &t, uint32_t &m) {
            t = kNone;
            m = 0u;
            if (bb < n_back && LCL_IN(cap - 1 - (int64_t)bb, cap)) {
                t = __ldg(tiles + (cap - 1 - (int64_t)bb));
                m = __ldg(masks + (cap - 1 - (int64_t)bb));
            }
        };
        uint32_t b = (gridDim.x - 1 - blockIdx.x) * (kThreads / 32) + (threadIdx.x >> 5);
        uint32_t next_tile, next_mask;
        entry(b, next_tile, next_mask);
        for (; b < n_back; b += warps) {
            const uint32_t tile = next_tile, mask = next_mask;
            entry(b + warps, next_tile, next_mask);
            if (!mask || tile == kNone) continue;  // uniform over the warp
            const uint32_t label = g.s[31 - __clz(mask)].label;
            int32_t tx, ty;
            tile_xy(a, tile, tx, ty);
            uint32_t c = 0u;
            for (int32_t wi = lane; wi < words; wi += 32) {
                const int32_t x = tx * a.T + 32 * (wi % wpr), y = ty * a.T + wi / wpr;
                if (x >= a.w || y >= a.h) continue;  // x < w implies x + 31 < w (w a multiple of 32)
                const int64_t l = (int64_t)y * a.w + x;
                if (!LCL_IN(l + 31, n_tex)) continue;
                const uint32_t cov = __ldg(a.cover + (l >> 5));
                if (!cov) continue;
                store_word32<L>(layer, l, cov, label);
                c += __popc(cov);
            }
            if (hits) {
                c = __reduce_add_sync(0xffffffffu, c);
                if (lane == 0 && c)
                    for (uint32_t m = mask; m; m &= m - 1) atomicAdd(&s_hits[__ffs(m) - 1], (unsigned long long)c);
            }
        }
    }
    if (hits) {
        __syncthreads();
        if ((int)threadIdx.x < g.n && s_hits[threadIdx.x]) atomicAdd(hits + threadIdx.x, s_hits[threadIdx.x]);
    }
}

// ---- lasso ---------------------------------------------------------------------------

// Super-tiles a lasso (or tool window) can touch: 8 lanes per super-tile (box_may_touch8 without
// the depth map), appended to `list` (counter `counter`).
__global__ void __launch_bounds__(kThreads) k_lasso_supers(AtlasDev a, const __grid_constant__ LassoArg p,
                                                           uint32_t *counter, uint32_t *list) {
    const int64_t n_super = (int64_t)a.supers_x * a.supers_y;
    const int64_t sidx = (int64_t)blockIdx.x * (kThreads / 8) + threadIdx.x / 8;
    bool cand = false;
    if (sidx < n_super) {  // uniform over each group of 8 lanes
        const int4 *sb = reinterpret_cast<const int4 *>(a.super_box + 8 * sidx);
        const int4 slo = sb[0], shi = sb[1];
        cand = slo.w > 0 && box_may_touch8(p, slo, shi, nullptr);
    }
    pdl_wait();  // the counter was reset by the previous grid
    pdl_allow_next();
    append_candidate(cand && (threadIdx.x & 7u) == 0, (uint32_t)sidx, counter, list, n_super);
}

constexpr int kCullParts = LCL_SUPER * LCL_SUPER / (kThreads / 8);  // 8 parts of 32 tiles per super-tile

// Candidate tiles of a lasso (or tool window) in the super-tiles k_lasso_supers listed: the CTAs take
// (super-tile, part) units, a part being 32 tiles tested by 8 lanes each (box_may_touch8 with the
// depth map), so the work spreads over the GPU however few super-tiles the lasso reaches.  FLAGS:
// write a 0/1 flag per tile instead of appending candidates (first pass of a padded edit; the flags
// of tiles in other super-tiles were cleared before).  CLASSIFY (lassos): tiles that
// lasso_tile_class8 finds outside the polygon are dropped, and those it finds inside are listed with
// kInsideTile set (their texels skip the edge tests).
template <bool FLAGS, bool CLASSIFY>
__global__ void __launch_bounds__(kThreads) k_lasso_cull(AtlasDev a, const __grid_constant__ LassoArg p,
                                                         const float *__restrict__ depth,
                                                         const uint32_t *__restrict__ super_count,
                                                         const uint32_t *__restrict__ supers, uint32_t *counter,
                                                         uint32_t *list) {
    __shared__ float svx[LCL_MAX_LASSO_VERTICES + 1], svy[LCL_MAX_LASSO_VERTICES + 1];
    if (CLASSIFY) {
        for (int e = threadIdx.x; e <= p.nv; e += blockDim.x) {
            svx[e] = p.vx[e];
            svy[e] = p.vy[e];
        }
        __syncthreads();
    }
    pdl_wait();  // the candidate super-tiles are complete
    pdl_allow_next();
    const int64_t n_tiles = (int64_t)a.tiles_x * a.tiles_y, n_super = (int64_t)a.supers_x * a.supers_y;
    (void)n_super;
    const uint32_t n_units = *super_count * kCullParts;
    for (uint32_t u = blockIdx.x; u < n_units; u += gridDim.x) {  // uniform over the CTA
        if (!LCL_IN(u / kCullParts, n_super)) break;
        const uint32_t sidx = supers[u / kCullParts];
        const int32_t sx = (int32_t)(sidx % a.supers_x), sy = (int32_t)(sidx / a.supers_x);
        const int32_t local = (int32_t)(u % kCullParts) * (kThreads / 8) + (int32_t)(threadIdx.x / 8);
        const int32_t tx = sx * LCL_SUPER + local % LCL_SUPER, ty = sy * LCL_SUPER + local / LCL_SUPER;
        const bool in_grid = tx < a.tiles_x && ty < a.tiles_y;  // uniform over each group of 8 lanes
        bool cand = false;
        int cls = kTileTest;
        // the group's 8 lanes take the same branch (in_grid and the index check are per tile)
        if (in_grid && LCL_IN((int64_t)ty * a.tiles_x + tx, n_tiles)) {
            const int4 *tb = reinterpret_cast<const int4 *>(a.tile_box + 8 * ((int64_t)ty * a.tiles_x + tx));
            const int4 lo = tb[0], hi = tb[1];
            if (lo.w > 0) {  // uniform over the group (one tile)
                if (CLASSIFY) cand = box_may_touch8<true>(p, lo, hi, depth, nullptr, svx, svy, &cls);
                else cand = box_may_touch8(p, lo, hi, depth);
            }
        }
        const uint32_t tile = (uint32_t)(ty * a.tiles_x + tx);
        if (FLAGS) {
            if (in_grid && (threadIdx.x & 7u) == 0 && LCL_IN(tile, n_tiles)) list[tile] = cand ? 1u : 0u;
        } else {
            append_candidate(cand && (threadIdx.x & 7u) == 0, tile | (cls == kTileIn ? kInsideTile : 0u), counter,
                             list, n_tiles);
        }
    }
}

// Second pass of a padded edit: with texture padding a texel may be written because a neighbour
// within 8 texels (at most one tile away) was selected, so a tile is a candidate if any tile of
// its 3 x 3 neighbourhood is flagged.
__global__ void __launch_bounds__(kThreads) k_dilate_candidates(AtlasDev a, const uint32_t *__restrict__ flags,
                                                                uint32_t *counter, uint32_t *list) {
    const int64_t t = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    const int64_t n_tiles = (int64_t)a.tiles_x * a.tiles_y;
    bool cand = false;
    if (t < n_tiles) {
        const int32_t tx = (int32_t)(t % a.tiles_x), ty = (int32_t)(t / a.tiles_x);
        for (int32_t y = max(ty - 1, 0); y <= min(ty + 1, a.tiles_y - 1) && !cand; ++y)
            for (int32_t x = max(tx - 1, 0); x <= min(tx + 1, a.tiles_x - 1); ++x)
                if (LCL_IN((int64_t)y * a.tiles_x + x, n_tiles) && flags[(int64_t)y * a.tiles_x + x]) cand = true;
    }
    append_candidate(cand, (uint32_t)t, counter, list, n_tiles);
}


// Texture padding of the uncovered texels of a quad for a lasso edit (Section 4.3.2, as for
// spheres): written if a covered texel lies within the outline thickness and a texel the lasso
// selects within the kernel radius (square kernels).
__device__ uint32_t lasso_pad_mask(const AtlasDev &a, int64_t l, int4 X, const LassoArg &p, const LassoShared &sh,
                                   const float *__restrict__ depth, int32_t pad_r, int32_t pad_t) {
    const int32_t x0 = (int32_t)(l % a.w), y0 = (int32_t)(l / a.w);
    const int32_t reach = max(pad_r, pad_t);
    uint32_t m = 0;
#pragma unroll 1
    for (int k = 0; k < 4; ++k) {
        const int32_t xk = k == 0 ? X.x : k == 1 ? X.y : k == 2 ? X.z : X.w;  // a select, not a local array
        if (xk != INT32_MIN) continue;
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
                if (ax <= pad_t && ay <= pad_t) outline = true;
                if (ax <= pad_r && ay <= pad_r && !near) near = lasso_hit(p, sh, depth, qx, __ldg(a.py + n), __ldg(a.pz + n));
            }
        }
        if (outline && near) m |= 1u << k;
    }
    return m;
}

// A lasso's candidate-list entry: tile index, kInsideTile set when every texel of the tile that
// projects lies inside the polygon (lasso_tile_class8).  Padded edits list plain tile indices.
template <typename L, bool NUM, bool PAD>
__global__ void __launch_bounds__(kThreads) k_lasso_apply(AtlasDev a, L *__restrict__ layer,
                                                          const __grid_constant__ LassoArg p,
                                                          const float *__restrict__ depth,
                                                          const uint32_t *__restrict__ counter,
                                                          const uint32_t *__restrict__ list,
                                                          unsigned long long *hits, ValMask vm, int32_t pad_r,
                                                          int32_t pad_t) {
    __shared__ LassoShared sh;
    stage_lasso(sh, p);
    __syncthreads();
    pdl_wait();  // the candidate tiles are complete
    pdl_allow_next();
    const uint32_t n = *counter;
    const int32_t qpr = a.T / 4, nq = a.T * qpr;
    uint32_t cnt = 0;
    const int64_t n_tex = (int64_t)a.w * a.h;
    for (uint32_t i = blockIdx.x; i < n; i += gridDim.x) {
        if (!LCL_IN(i, (int64_t)a.tiles_x * a.tiles_y)) break;
        const uint32_t entry = list[i];
        const bool inside = (entry & kInsideTile) != 0u;  // uniform over the CTA
        const uint32_t tile = entry & ~kInsideTile;
        int32_t tx, ty;
        tile_xy(a, tile, tx, ty);
        for (int32_t qd = threadIdx.x; qd < nq; qd += kThreads) {
            const int32_t x = tx * a.T + 4 * (qd & (qpr - 1)), y = ty * a.T + (qd >> (__ffs(qpr) - 1));
            if (x >= a.w || y >= a.h) continue;
            const int64_t l = (int64_t)y * a.w + x;
            if (!LCL_IN(l + 3, n_tex)) continue;
            const int4 X = __ldg(reinterpret_cast<const int4 *>(a.px + l));
            const int4 Y = __ldg(reinterpret_cast<const int4 *>(a.py + l));
            const int4 Z = __ldg(reinterpret_cast<const int4 *>(a.pz + l));
            const uint32_t m = inside ? lasso_quad<true>(p, sh, depth, X, Y, Z) : lasso_quad<false>(p, sh, depth, X, Y, Z);
            const uint32_t pm = PAD ? lasso_pad_mask(a, l, X, p, sh, depth, pad_r, pad_t) : 0u;
            if (m | pm) {
                store_hits<L>(layer, l, m | pm, p.label);
                if (NUM) valid_update_atomic(vm, l, m | pm, n_tex);
                cnt += __popc(m);
            }
        }
    }
    add_hits(hits, cnt);
}

// ---- the paper's editing tool -------------------------------------------------------------

// Texture padding of the uncovered texels of a quad for a tool edit (Section 4.3.2, as for
// spheres): written if a covered texel lies within the outline thickness and a texel the tool
// selects within the kernel radius (square kernels).
template <bool MASK>
__device__ __forceinline__ uint32_t tool_pad_mask(const AtlasDev &a, int64_t l, int4 X, const LassoArg &p, const ToolArg &t,
                                  const float *__restrict__ depth) {
    const int32_t x0 = (int32_t)(l % a.w), y0 = (int32_t)(l / a.w);
    const int32_t reach = max(t.pad_r, t.pad_t);
    uint32_t m = 0;
#pragma unroll 1
    for (int k = 0; k < 4; ++k) {
        const int32_t xk = k == 0 ? X.x : k == 1 ? X.y : k == 2 ? X.z : X.w;  // a select, not a local array
        if (xk != INT32_MIN) continue;
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
                if (ax <= t.pad_t && ay <= t.pad_t) outline = true;
                if (ax <= t.pad_r && ay <= t.pad_r && !near)
                    near = tool_hit<MASK>(p, t, depth, qx, __ldg(a.py + n), __ldg(a.pz + n));
            }
        }
        if (outline && near) m |= 1u << k;
    }
    return m;
}

template <typename L, bool MASK, bool PAD, bool NUM>
__global__ void __launch_bounds__(kThreads, 4) k_tool_apply(AtlasDev a, L *__restrict__ layer,
                                                         const __grid_constant__ LassoArg p, ToolArg t,
                                                         const float *__restrict__ depth,
                                                         const uint32_t *__restrict__ counter,
                                                         const uint32_t *__restrict__ list,
                                                         unsigned long long *hits, ValMask vm) {
    const uint32_t n = *counter;
    const int32_t qpr = a.T / 4, nq = a.T * qpr;
    uint32_t cnt = 0;
    const int64_t n_tex = (int64_t)a.w * a.h;
    for (uint32_t i = blockIdx.x; i < n; i += gridDim.x) {
        if (!LCL_IN(i, (int64_t)a.tiles_x * a.tiles_y)) break;
        const uint32_t tile = list[i] & ~kInsideTile;  // the tool's cull lists plain tiles
        int32_t tx, ty;
        tile_xy(a, tile, tx, ty);
        for (int32_t qd = threadIdx.x; qd < nq; qd += kThreads) {
            const int32_t x = tx * a.T + 4 * (qd & (qpr - 1)), y = ty * a.T + (qd >> (__ffs(qpr) - 1));
            if (x >= a.w || y >= a.h) continue;
            const int64_t l = (int64_t)y * a.w + x;
            if (!LCL_IN(l + 3, n_tex)) continue;
            const int4 X = __ldg(reinterpret_cast<const int4 *>(a.px + l));
            const int4 Y = __ldg(reinterpret_cast<const int4 *>(a.py + l));
            const int4 Z = __ldg(reinterpret_cast<const int4 *>(a.pz + l));
            uint32_t m = 0;
            m |= tool_hit<MASK>(p, t, depth, X.x, Y.x, Z.x) ? 1u : 0u;
            m |= tool_hit<MASK>(p, t, depth, X.y, Y.y, Z.y) ? 2u : 0u;
            m |= tool_hit<MASK>(p, t, depth, X.z, Y.z, Z.z) ? 4u : 0u;
            m |= tool_hit<MASK>(p, t, depth, X.w, Y.w, Z.w) ? 8u : 0u;
            const uint32_t pm = PAD ? tool_pad_mask<MASK>(a, l, X, p, t, depth) : 0u;
            if (m | pm) {
                store_hits<L>(layer, l, m | pm, p.label);
                if (NUM) valid_update_atomic(vm, l, m | pm, n_tex);
                cnt += __popc(m);
            }
        }
    }
    add_hits(hits, cnt);
}

struct SelWs {
    uint32_t *counters, *list, *list2, *list3;  // three candidate lists: sphere stroke k uses list k mod 3
    uint32_t *list4, *list5, *list6;            // calls of two or more strokes: a second item set for groups
};

SelWs sel_ws(const lcl_atlas *a, int32_t n, void *ws) {
    SelWs w;
    char *base = static_cast<char *>(ws);
    const size_t lb = align256((size_t)a->tiles_x * a->tiles_y * 4);
    w.counters = reinterpret_cast<uint32_t *>(base);  // n + 1 front counters, then n + 1 inside counters
    w.list = reinterpret_cast<uint32_t *>(base + align256((size_t)2 * (n + 1) * 4));
    w.list2 = reinterpret_cast<uint32_t *>(reinterpret_cast<char *>(w.list) + lb);
    w.list3 = reinterpret_cast<uint32_t *>(reinterpret_cast<char *>(w.list2) + lb);
    w.list4 = w.list5 = w.list6 = nullptr;
    if (n >= 2) {
        w.list4 = reinterpret_cast<uint32_t *>(reinterpret_cast<char *>(w.list3) + lb);
        w.list5 = reinterpret_cast<uint32_t *>(reinterpret_cast<char *>(w.list4) + lb);
        w.list6 = reinterpret_cast<uint32_t *>(reinterpret_cast<char *>(w.list5) + lb);
    }
    return w;
}

// Launches the cull of a lasso / tool into w.list (counter w.counters[0]); with padding, the flags
// go to w.list2 first.  Small atlases split each super-tile over up to 8 CTAs so that the grid
// still covers the GPU.  Returns the number of launches.
int launch_lasso_cull(const AtlasDev &a, const lcl_atlas *atlas, const LassoArg &p, const float *depth,
                      const SelWs &w, bool pad, bool classify, cudaStream_t st) {
    // counters[1] and list3 hold the candidate super-tiles (lassos and the tool use list and list2 only)
    const int n_super = atlas->supers_x * atlas->supers_y;
    const int grid = std::max(1, std::min(n_super * kCullParts, 8 * sm_count()));
    if (!pad && classify) {  // the lasso's chain: each launch a programmatic dependent of the one before
        launch_pdl(k_lasso_supers, dim3((n_super + kThreads / 8 - 1) / (kThreads / 8)), st, a, p, w.counters + 1,
                   w.list3);
        launch_pdl(k_lasso_cull<false, true>, dim3(grid), st, a, p, depth, (const uint32_t *)(w.counters + 1),
                   (const uint32_t *)w.list3, w.counters, w.list);
        return 2;
    }
    k_lasso_supers<<<(n_super + kThreads / 8 - 1) / (kThreads / 8), kThreads, 0, st>>>(a, p, w.counters + 1, w.list3);
    if (!pad) {
        if (classify)
            k_lasso_cull<false, true><<<grid, kThreads, 0, st>>>(a, p, depth, w.counters + 1, w.list3, w.counters,
                                                                 w.list);
        else
            k_lasso_cull<false, false><<<grid, kThreads, 0, st>>>(a, p, depth, w.counters + 1, w.list3, w.counters,
                                                                  w.list);
        return 2;
    }
    // padded edits: flags for every tile that may hold a selected texel (polygon-outside tiles of a
    // lasso hold none; tiles of super-tiles the lasso cannot reach keep the cleared 0), dilated to the
    // tiles padding can reach
    const int64_t tiles = (int64_t)atlas->tiles_x * atlas->tiles_y;
    cudaMemsetAsync(w.list2, 0, (size_t)tiles * 4, st);
    if (classify)
        k_lasso_cull<true, true><<<grid, kThreads, 0, st>>>(a, p, depth, w.counters + 1, w.list3, w.counters, w.list2);
    else
        k_lasso_cull<true, false><<<grid, kThreads, 0, st>>>(a, p, depth, w.counters + 1, w.list3, w.counters,
                                                             w.list2);
    k_dilate_candidates<<<(unsigned)((tiles + kThreads - 1) / kThreads), kThreads, 0, st>>>(a, w.list2, w.counters,
                                                                                        w.list);
    return 3;
}

// ---- division check ----------------------------------------------------------------------

__device__ __forceinline__ uint32_t mix32(uint32_t x) {
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}

// Compares div_rn with __fdiv_rn on operand i of four families (i % 4): random signs and mantissas
// with exponents across and beyond div_rn's window; quotients next to a rounding midpoint (a = q b
// rounded, +-1 ulp); operands at the window's edges and just outside; special values (zeros,
// subnormals, infinities, NaN, the largest and smallest normals, tiny positive and negative w).
// counts[0] += compared, counts[1] += mismatches (NaN results compare equal to NaN).  For b > 0 the
// exact decisions quot_ge0 and quot_le are compared with the same tests on __fdiv_rn's quotient.
__global__ void k_check_division(uint64_t n, uint32_t seed, unsigned long long *counts) {
    unsigned long long cmp = 0, bad = 0;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t h1 = mix32((uint32_t)i * 2u + seed), h2 = mix32((uint32_t)(i >> 32) ^ ((uint32_t)i * 2u + 1u) ^ (seed * 0x9e3779b9u));
        float a, b;
        switch (i & 3u) {
        case 0: {  // exponents 67..187 (the window is 97..157)
            const uint32_t ea = 67u + (h1 >> 25) % 121u, eb = 67u + (h2 >> 25) % 121u;
            a = __uint_as_float((h1 & 0x80000000u) | (ea << 23) | (h2 & 0x7FFFFFu));
            b = __uint_as_float((h2 & 0x80000000u) | (eb << 23) | (h1 & 0x7FFFFFu));
            break;
        }
        case 1: {  // near-midpoint quotients: a = RN(q b) and its neighbours
            const uint32_t eq = 97u + (h1 >> 26) % 30u, eb = 110u + (h2 >> 27) % 30u;
            const float q = __uint_as_float((eq << 23) | (h1 & 0x7FFFFFu));
            b = __uint_as_float((h2 & 0x80000000u) | (eb << 23) | (h2 & 0x7FFFFFu));
            a = __fmul_rn(q, b);
            a = __uint_as_float(__float_as_uint(a) + (h1 >> 30) - 1u);
            break;
        }
        case 2: {  // window edges: exponents 95..99 and 155..159, mantissas at their ends
            const uint32_t edges[10] = {95u, 96u, 97u, 98u, 99u, 155u, 156u, 157u, 158u, 159u};
            const uint32_t ma = (h1 & 1u) ? 0x7FFFFFu : (h1 & 2u) ? 0u : (h2 & 0x7FFFFFu);
            const uint32_t mb = (h2 & 1u) ? 0x7FFFFFu : (h2 & 2u) ? 0u : (h1 & 0x7FFFFFu);
            a = __uint_as_float((h1 & 0x80000000u) | (edges[(h1 >> 8) % 10u] << 23) | ma);
            b = __uint_as_float((h2 & 0x80000000u) | (edges[(h2 >> 8) % 10u] << 23) | mb);
            break;
        }
        default: {  // special values against random ones
            const float sp[12] = {0.0f, -0.0f, __uint_as_float(1u), __uint_as_float(0x807FFFFFu), INFINITY, -INFINITY,
                                  __uint_as_float(0x7FC00000u), 3.4028235e38f, 1.17549435e-38f, 1e-30f, -1e-30f,
                                  7.0f};
            const float rnd = __uint_as_float((h1 & 0x80000000u) | ((97u + (h2 >> 26) % 61u) << 23) | (h2 & 0x7FFFFFu));
            const float s = sp[(h1 >> 4) % 12u];
            a = (h2 & 1u) ? s : rnd;
            b = (h2 & 1u) ? rnd : s;
            if ((h2 & 6u) == 6u) b = sp[(h2 >> 9) % 12u];
            break;
        }
        }
        const float q = __fdiv_rn(a, b), m = div_rn(a, b);
        const bool same = __float_as_uint(q) == __float_as_uint(m) || (isnan(q) && isnan(m));
        ++cmp;
        bad += same ? 0 : 1;
        // quot_ge0 and quot_le (b > 0) against the quotient, at thresholds on it, one ulp either
        // side, 1 and a random value
        if (b > 0.0f && !isnan(q)) {
            ++cmp;
            bad += quot_ge0(a, b) == (q >= 0.0f) ? 0 : 1;
            const float ts[5] = {q, nextafterf(q, INFINITY), nextafterf(q, -INFINITY), 1.0f,
                                 __uint_as_float((h2 & 0x80000000u) | ((100u + (h1 >> 27)) << 23) | (h1 & 0x7FFFFFu))};
#pragma unroll
            for (int j = 0; j < 5; ++j) {
                ++cmp;
                bad += quot_le(a, b, ts[j]) == (q <= ts[j]) ? 0 : 1;
            }
        }
    }
    for (int o = 16; o; o >>= 1) {
        cmp += __shfl_xor_sync(0xffffffffu, cmp, o);
        bad += __shfl_xor_sync(0xffffffffu, bad, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(counts, cmp);
        if (bad) atomicAdd(counts + 1, bad);
    }
}

}  // namespace

lcl_status division_check_impl(uint64_t n, uint32_t seed, uint64_t *counts, cudaStream_t st) {
    k_check_division<<<sm_count() * 8, kThreads, 0, st>>>(n, seed, reinterpret_cast<unsigned long long *>(counts));
    count_launches(1);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "lcl_check_division launch");
    return LCL_OK;
}

size_t select_ws_bytes(const lcl_atlas *a, int32_t n) {
    return align256((size_t)2 * (n + 1) * 4) + (n >= 2 ? 6 : 3) * align256((size_t)a->tiles_x * a->tiles_y * 4);
}

// Unpadded strokes on a label layer, kGroup at a time (see k_group_apply): zeroing, then a cull and
// an apply launch per group, chained with programmatic dependent launch.
template <typename L, typename ArgOf>
lcl_status select_sphere_grouped(const lcl_atlas *atlas, const AtlasDev &a, L *layer, const SelWs &w, int32_t n,
                                 unsigned long long *h, const ArgOf &arg, cudaStream_t st) {
    const int32_t n_groups = (n + kGroup - 1) / kGroup;
    k_sel_init<<<(std::max(2 * n_groups, n) + kThreads - 1) / kThreads, kThreads, 0, st>>>(w.counters, 2 * n_groups,
                                                                                          h, n);
    static thread_local GroupArg g;  // ~1.5 KB: kept off the stack
    g.rows = (a.T >= 32 && (a.w & 31) == 0) ? 1 : 0;
    const int n_super = atlas->supers_x * atlas->supers_y;
    const int cull_grid = std::min(n_super, resident_grid(k_group_cull));
    const int apply_grid = resident_grid(k_group_apply<L>);
    cudaError_t e = cudaSuccess;
    for (int32_t gi = 0; gi < n_groups && e == cudaSuccess; ++gi) {
        const int32_t k0 = gi * kGroup;
        g.n = std::min(kGroup, n - k0);
        for (int32_t k = 0; k < g.n; ++k) g.s[k] = arg(k0 + k);
        uint32_t *const c = w.counters + 2 * gi;
        // item sets alternate between groups, so a group's cull can run while the previous apply does
        uint32_t *const t = (gi & 1) ? w.list4 : w.list, *const m = (gi & 1) ? w.list5 : w.list2,
                        *const su = (gi & 1) ? w.list6 : w.list3;
        e = launch_pdl(k_group_cull, dim3(cull_grid), st, a, g, c, t, m, su, gi > 0 ? 1 : 0);
        if (e == cudaSuccess)
            e = launch_pdl(k_group_apply<L>, dim3(apply_grid), st, a, layer, g, (const uint32_t *)c,
                           (const uint32_t *)t, (const uint32_t *)m, (const uint32_t *)su, h ? h + k0 : nullptr);
    }
    count_launches(1 + 2 * n_groups);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "lcl_select_sphere launch");
    return LCL_OK;
}

template <typename L>
using StepKernel = void (*)(AtlasDev, L *, SphereArg, const uint32_t *, const uint32_t *, const uint32_t *,
                            unsigned long long *, int, SphereArg, uint32_t *, uint32_t *, uint32_t *, ValMask);

// Sphere strokes on a label layer (NUM false) or on the data texture of a numeric layer whose mask
// bits are `mask` (NUM true; an erase stroke writes 0 and clears the bits).
template <typename L, bool NUM>
lcl_status select_sphere_run(const lcl_atlas *atlas, L *layer, uint32_t *mask, const lcl_sphere *strokes, int32_t n,
                             uint64_t *hits, void *ws, cudaStream_t st) {
    const AtlasDev a = dev_view(atlas);
    const SelWs w = sel_ws(atlas, n, ws);
    unsigned long long *h = reinterpret_cast<unsigned long long *>(hits);
    auto arg = [&](int32_t k) {
        SphereArg s;
        s.cx = strokes[k].cx;
        s.cy = strokes[k].cy;
        s.cz = strokes[k].cz;
        s.r2 = strokes[k].r2 > kR2Cap ? kR2Cap : strokes[k].r2;
        s.label = (NUM && (strokes[k].flags & LCL_ERASE)) ? 0u : strokes[k].label;
        s.pad_r = (int32_t)(strokes[k].flags & 15u);
        s.pad_t = (int32_t)((strokes[k].flags >> 4) & 15u);
        return s;
    };
    auto vmask = [&](int32_t k) {
        ValMask vm;
        vm.bits = mask;
        vm.set = (strokes[k].flags & LCL_ERASE) ? 0u : 1u;
        return vm;
    };
    if constexpr (!NUM) {
        bool padded = false;
        for (int32_t k = 0; k < n; ++k) padded = padded || (strokes[k].flags & 15u) != 0;
        if (n >= 2 && !padded) return select_sphere_grouped(atlas, a, layer, w, n, h, arg, st);
    }
    // [pad][next_pad] variants and their resident grids
    const StepKernel<L> step[2][2] = {{k_sphere_step<L, false, false, NUM>, k_sphere_step<L, false, true, NUM>},
                                      {k_sphere_step<L, true, false, NUM>, k_sphere_step<L, true, true, NUM>}};
    int grid[2][2];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) grid[i][j] = resident_grid(step[i][j]);
    uint32_t *const inside = w.counters + (n + 1);
    k_sel_init<<<(2 * (n + 1) + kThreads - 1) / kThreads, kThreads, 0, st>>>(w.counters, 2 * (n + 1), h, n);
    const int n_super = atlas->supers_x * atlas->supers_y;
    cudaError_t e = launch_pdl(k_sphere_cull, dim3(std::min(n_super, grid[0][0])), st, a, arg(0), w.counters, w.list,
                               inside);
    for (int32_t k = 0; k < n && e == cudaSuccess; ++k) {
        uint32_t *const lists[3] = {w.list, w.list2, w.list3};
        uint32_t *cur_list = lists[k % 3], *next_list = lists[(k + 1) % 3];
        const int has_next = k + 1 < n;
        const SphereArg cur = arg(k), nxt = arg(has_next ? k + 1 : k);
        const int pi = cur.pad_r > 0, pj = has_next && nxt.pad_r > 0;
        e = launch_pdl(step[pi][pj], dim3(grid[pi][pj]), st, a, layer, cur, (const uint32_t *)(w.counters + k),
                       (const uint32_t *)(inside + k), (const uint32_t *)cur_list, h ? h + k : nullptr, has_next, nxt,
                       w.counters + k + 1, inside + k + 1, next_list, vmask(k));
    }
    count_launches(2 + n);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, NUM ? "lcl_numeric_sphere launch" : "lcl_select_sphere launch");
    return LCL_OK;
}

lcl_status select_sphere_impl(const lcl_atlas *atlas, void *layer, int dtype_bytes, const lcl_sphere *strokes,
                              int32_t n, uint64_t *hits, void *ws, cudaStream_t st) {
    if (dtype_bytes == 1)
        return select_sphere_run<uint8_t, false>(atlas, static_cast<uint8_t *>(layer), nullptr, strokes, n, hits, ws,
                                                 st);
    return select_sphere_run<uint16_t, false>(atlas, static_cast<uint16_t *>(layer), nullptr, strokes, n, hits, ws, st);
}

lcl_status numeric_sphere_impl(const lcl_atlas *atlas, void *data, int data_bytes, uint32_t *mask,
                               const lcl_sphere *strokes, int32_t n, uint64_t *hits, void *ws, cudaStream_t st) {
    if (data_bytes == 1)
        return select_sphere_run<uint8_t, true>(atlas, static_cast<uint8_t *>(data), mask, strokes, n, hits, ws, st);
    if (data_bytes == 2)
        return select_sphere_run<uint16_t, true>(atlas, static_cast<uint16_t *>(data), mask, strokes, n, hits, ws, st);
    return select_sphere_run<uint32_t, true>(atlas, static_cast<uint32_t *>(data), mask, strokes, n, hits, ws, st);
}

template <typename L, bool NUM>
void launch_lasso_apply(bool pad, const AtlasDev &a, L *layer, const LassoArg &p, const float *depth,
                        const SelWs &w, unsigned long long *h, ValMask vm, int32_t pad_r, int32_t pad_t,
                        cudaStream_t st) {
    if (pad)
        k_lasso_apply<L, NUM, true><<<resident_grid(k_lasso_apply<L, NUM, true>), kThreads, 0, st>>>(
            a, layer, p, depth, w.counters, w.list, h, vm, pad_r, pad_t);
    else
        launch_pdl(k_lasso_apply<L, NUM, false>, dim3(resident_grid(k_lasso_apply<L, NUM, false>)), st, a, layer, p,
                   depth, (const uint32_t *)w.counters, (const uint32_t *)w.list, h, vm, 0, 0);
}

// Lasso on a label layer (mask NULL) or on a numeric layer (data bytes 1, 2 or 4 and its mask bits),
// with texture padding when pad_flags asks for it (radius = bits 0-3, thickness = bits 4-7).
lcl_status lasso_run(const lcl_atlas *atlas, void *layer, int bytes, uint32_t *mask, uint32_t set, const lcl_camera *cam,
                     const float *depth, const float *poly, int32_t nv, uint32_t label, float bias, uint32_t pad_flags,
                     uint64_t *hits, void *ws, cudaStream_t st) {
    const AtlasDev a = dev_view(atlas);
    const SelWs w = sel_ws(atlas, 1, ws);
    unsigned long long *h = reinterpret_cast<unsigned long long *>(hits);
    static thread_local LassoArg p;  // ~2.8 KB: kept off the stack
    fill_lasso_arg(p, cam, poly, nv, label, bias);
    const int32_t pad_r = (int32_t)(pad_flags & 15u), pad_t = (int32_t)((pad_flags >> 4) & 15u);
    const bool pad = pad_r > 0;
    if (pad)
        k_sel_init<<<1, kThreads, 0, st>>>(w.counters, 2, h, 1);
    else
        launch_pdl(k_sel_init, dim3(1), st, w.counters, 2, h, 1);
    const int n_cull = launch_lasso_cull(a, atlas, p, depth, w, pad, true, st);
    ValMask vm;
    vm.bits = mask;
    vm.set = set;
    if (!mask) {
        if (bytes == 1)
            launch_lasso_apply<uint8_t, false>(pad, a, static_cast<uint8_t *>(layer), p, depth, w, h, vm, pad_r, pad_t, st);
        else
            launch_lasso_apply<uint16_t, false>(pad, a, static_cast<uint16_t *>(layer), p, depth, w, h, vm, pad_r, pad_t,
                                                st);
    } else if (bytes == 1) {
        launch_lasso_apply<uint8_t, true>(pad, a, static_cast<uint8_t *>(layer), p, depth, w, h, vm, pad_r, pad_t, st);
    } else if (bytes == 2) {
        launch_lasso_apply<uint16_t, true>(pad, a, static_cast<uint16_t *>(layer), p, depth, w, h, vm, pad_r, pad_t, st);
    } else {
        launch_lasso_apply<uint32_t, true>(pad, a, static_cast<uint32_t *>(layer), p, depth, w, h, vm, pad_r, pad_t, st);
    }
    count_launches(2 + n_cull);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, mask ? "lcl_numeric_lasso launch" : "lcl_select_lasso launch");
    return LCL_OK;
}

lcl_status select_lasso_impl(const lcl_atlas *atlas, void *layer, int dtype_bytes, const lcl_camera *cam,
                             const float *depth, const float *poly, int32_t nv, uint32_t label, uint32_t flags,
                             float bias, uint64_t *hits, void *ws, cudaStream_t st) {
    return lasso_run(atlas, layer, dtype_bytes, nullptr, 1u, cam, depth, poly, nv, label, bias, flags & 0xFFu, hits, ws,
                     st);
}

lcl_status numeric_lasso_impl(const lcl_atlas *atlas, void *data, int data_bytes, uint32_t *mask, uint32_t value,
                              uint32_t flags, const lcl_camera *cam, const float *depth, const float *poly, int32_t nv,
                              float bias, uint64_t *hits, void *ws, cudaStream_t st) {
    const bool erase = (flags & LCL_ERASE) != 0;
    return lasso_run(atlas, data, data_bytes, mask, erase ? 0u : 1u, cam, depth, poly, nv, erase ? 0u : value, bias,
                     flags & 0xFFu, hits, ws, st);
}

template <typename L, bool NUM>
void launch_tool(int sel, const AtlasDev &a, L *layer, const LassoArg &p, const ToolArg &t, const float *depth,
                 const SelWs &w, unsigned long long *h, ValMask vm, cudaStream_t st) {
    switch (sel) {  // bit 0: shape mask, bit 1: padding
    case 0:
        k_tool_apply<L, false, false, NUM><<<resident_grid(k_tool_apply<L, false, false, NUM>), kThreads, 0, st>>>(
            a, layer, p, t, depth, w.counters, w.list, h, vm);
        break;
    case 1:
        k_tool_apply<L, true, false, NUM><<<resident_grid(k_tool_apply<L, true, false, NUM>), kThreads, 0, st>>>(
            a, layer, p, t, depth, w.counters, w.list, h, vm);
        break;
    case 2:
        k_tool_apply<L, false, true, NUM><<<resident_grid(k_tool_apply<L, false, true, NUM>), kThreads, 0, st>>>(
            a, layer, p, t, depth, w.counters, w.list, h, vm);
        break;
    default:
        k_tool_apply<L, true, true, NUM><<<resident_grid(k_tool_apply<L, true, true, NUM>), kThreads, 0, st>>>(
            a, layer, p, t, depth, w.counters, w.list, h, vm);
        break;
    }
}

// The tool on a label layer (mask NULL) or on a numeric layer.
lcl_status tool_run(const lcl_atlas *atlas, void *layer, int bytes, uint32_t *mask, uint32_t set, const lcl_camera *cam,
                    const float *depth, const lcl_tool *tool, uint32_t label, float bias, uint64_t *hits, void *ws,
                    cudaStream_t st) {
    const AtlasDev a = dev_view(atlas);
    const SelWs w = sel_ws(atlas, 1, ws);
    unsigned long long *h = reinterpret_cast<unsigned long long *>(hits);
    static thread_local LassoArg p;  // ~2.8 KB: kept off the stack
    ToolArg t;
    fill_tool_arg(t, p, cam, tool, label, bias);
    k_sel_init<<<1, kThreads, 0, st>>>(w.counters, 2, h, 1);
    const bool pad = t.pad_r > 0;
    const int n_cull = launch_lasso_cull(a, atlas, p, depth, w, pad, false, st);
    const int sel = (tool->shape != nullptr ? 1 : 0) + (pad ? 2 : 0);
    ValMask vm;
    vm.bits = mask;
    vm.set = set;
    if (!mask) {
        if (bytes == 1) launch_tool<uint8_t, false>(sel, a, static_cast<uint8_t *>(layer), p, t, depth, w, h, vm, st);
        else launch_tool<uint16_t, false>(sel, a, static_cast<uint16_t *>(layer), p, t, depth, w, h, vm, st);
    } else if (bytes == 1) {
        launch_tool<uint8_t, true>(sel, a, static_cast<uint8_t *>(layer), p, t, depth, w, h, vm, st);
    } else if (bytes == 2) {
        launch_tool<uint16_t, true>(sel, a, static_cast<uint16_t *>(layer), p, t, depth, w, h, vm, st);
    } else {
        launch_tool<uint32_t, true>(sel, a, static_cast<uint32_t *>(layer), p, t, depth, w, h, vm, st);
    }
    count_launches(2 + n_cull);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, mask ? "lcl_numeric_tool launch" : "lcl_select_tool launch");
    return LCL_OK;
}

lcl_status select_tool_impl(const lcl_atlas *atlas, void *layer, int dtype_bytes, const lcl_camera *cam,
                            const float *depth, const lcl_tool *tool, uint32_t label, float bias, uint64_t *hits,
                            void *ws, cudaStream_t st) {
    return tool_run(atlas, layer, dtype_bytes, nullptr, 1u, cam, depth, tool, label, bias, hits, ws, st);
}

lcl_status numeric_tool_impl(const lcl_atlas *atlas, void *data, int data_bytes, uint32_t *mask, uint32_t value,
                             uint32_t flags, const lcl_camera *cam, const float *depth, const lcl_tool *tool,
                             float bias, uint64_t *hits, void *ws, cudaStream_t st) {
    const bool erase = (flags & LCL_ERASE) != 0;
    return tool_run(atlas, data, data_bytes, mask, erase ? 0u : 1u, cam, depth, tool, erase ? 0u : value, bias, hits,
                    ws, st);
}

}  // namespace lcl

