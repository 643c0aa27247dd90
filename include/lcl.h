/*
 * lcl.h -- C ABI of the GPU layer-editing library (GB300, sm_103a).
 *
 * Thematic information layers are 2D textures indexed by a mesh's texture
 * coordinates (arXiv 2501.14807, Section 4.1 and 4.2).  Editing a layer maps a
 * selection made in 3D or on the screen onto the texels it covers (Section 4.3.1,
 * Fig. 3).  This library precomputes, once per model, a UV atlas that tells for
 * every texel which triangle covers it and where that texel lies on the surface,
 * then edits, overlays and measures layers with per-texel kernels.
 *
 * Conventions shared by every entry point:
 *  - All buffers are caller-owned.  "device" pointers are CUDA device memory of the
 *    current device, "host" pointers are ordinary host memory.  The library keeps no
 *    allocation between calls and allocates nothing itself.
 *  - Calls enqueue work on `stream` (a cudaStream_t; NULL is the legacy default
 *    stream) and return without waiting, except lcl_atlas_build, which waits for its
 *    stream before returning (see there).  Calls that share an atlas workspace or
 *    write the same layer must be ordered on one stream.
 *  - Host-side argument checks happen before anything is enqueued and return
 *    LCL_ERR_INVALID_ARG or LCL_ERR_UNSUPPORTED with nothing enqueued.  A failed
 *    launch returns LCL_ERR_CUDA.  lcl_last_error() gives a one-line reason for the
 *    last non-OK status on the calling thread.
 *  - Layer textures are row-major planes of width x height labels (uint8 or uint16),
 *    row 0 at v = 0.  Label 0 means "no data" (the paper's mask texture set to
 *    false, Section 4.2).
 *  - Limits: width a multiple of 4 in [4, 16384], height in [1, 16384],
 *    tile in {8, 16, 32, 64, 128}; texture coordinates in [-1, 2]; at most 2^32-2
 *    triangles.
 */
#ifndef LCL_H
#define LCL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *lcl_stream; /* same type as cudaStream_t */

typedef enum {
    LCL_OK = 0,
    LCL_ERR_INVALID_ARG = 1,
    LCL_ERR_OUT_OF_MEMORY = 2, /* a caller buffer or workspace is too small */
    LCL_ERR_CUDA = 3,
    LCL_ERR_UNSUPPORTED = 4,
    LCL_ERR_TIMEOUT = 5,
    LCL_ERR_INTERNAL = 6
} lcl_status;

typedef enum { LCL_U8 = 1, LCL_U16 = 2 } lcl_dtype;
typedef enum { LCL_AND = 0, LCL_OR = 1, LCL_XOR = 2, LCL_MASK = 3 } lcl_op;
enum { LCL_NOT_A = 1, LCL_NOT_B = 2, LCL_NOT_OUT = 4 };

#define LCL_GRID_BITS 21              /* quantised position grid: [0, 2^21 - 1] per axis */
#define LCL_SUBPIXEL_BITS 8           /* rasteriser sub-pixel precision */
#define LCL_AREA_FRAC_BITS 8          /* fractional bits of area weights */
#define LCL_NO_TRIANGLE 0xFFFFFFFFu   /* triangle plane value of an uncovered texel */
#define LCL_SUPER 16                  /* tiles per super-tile side (culling hierarchy) */
#define LCL_MAX_LASSO_VERTICES 64

/* Mesh in device memory (Section 4, Geometry Manager: geometry lives on the GPU).
 * pos: n_pos x 3 float32; uv: n_uv x 2 float32; tri_pos / tri_uv: n_tri x 3 uint32
 * indices into pos / uv (separate, so seams can duplicate texture coordinates). */
typedef struct {
    const float *pos;
    int64_t n_pos;
    const float *uv;
    int64_t n_uv;
    const uint32_t *tri_pos;
    const uint32_t *tri_uv;
    int64_t n_tri;
} lcl_mesh;

/* UV atlas of one model at one texture size.  Filled by lcl_atlas_bind (pointers into
 * one caller buffer) and lcl_atlas_build (contents, bbox_min, scale).
 *  pos_x/pos_y/pos_z: int32 planes (width x height): the 21-bit grid position of the
 *      surface point at the texel centre; an uncovered texel holds (INT32_MIN, 0, 0).
 *  tri: uint32 plane, the covering triangle (LCL_NO_TRIANGLE if none).
 *  cover: coverage bits, bit (y*width + x) of a linear uint32 array.
 *  tile_box: per tile (row-major over tiles_x x tiles_y) 8 int32: min x, min y, min z,
 *      covered count, max x, max y, max z, 0 (empty: INT32_MAX mins, INT32_MIN maxes).
 *  super_box: the same record per super-tile of LCL_SUPER x LCL_SUPER tiles.
 *  area_w: uint64 per triangle, the surface area one of its texels stands for.
 *  bbox_min, scale: the quantisation, grid = floor((p - bbox_min) * scale + 0.5).
 *  row0: first texture row held by this atlas (0, or the start of a row view or band).
 *  tex_height: rows of the whole texture this atlas is part of (height for a whole atlas; a band
 *      or row view holds rows [row0, row0 + height) of it). */
typedef struct {
    int32_t width, height, tile;
    int32_t tiles_x, tiles_y, supers_x, supers_y;
    int32_t row0;
    int64_t n_tri;
    int32_t *pos_x, *pos_y, *pos_z;
    uint32_t *tri;
    uint32_t *cover;
    int32_t *tile_box;  /* NULL in a row view */
    int32_t *super_box; /* NULL in a row view */
    uint64_t *area_w;
    float bbox_min[3];
    int32_t tex_height;
    double scale;
} lcl_atlas;

/* Sphere stroke in grid units (32 bytes): texels with (q - c)^2 <= r2 get `label`.
 * flags: texture padding (Section 4.3.2), radius = bits 0-3, outline thickness = bits 4-7, both
 * <= 8 (0 = none); LCL_ERASE (bit 8) only in lcl_numeric_sphere; other bits 0. */
typedef struct {
    int32_t cx, cy, cz, _pad;
    int64_t r2;
    uint32_t label, flags;
} lcl_sphere;

/* Camera: m maps a grid position (q, 1) to clip space (row-major 4x4, FP32),
 * m = ViewProjection * Dequantise; width x height is the depth-map / screen size. */
typedef struct {
    float m[16];
    int32_t width, height;
} lcl_camera;

/* ---- sizing and binding ------------------------------------------------- */

/* Bytes of one atlas buffer for lcl_atlas_bind (0 if the sizes are invalid). */
size_t lcl_atlas_bytes(int32_t width, int32_t height, int32_t tile, int64_t n_tri);

/* Points the atlas planes into `base` (device, at least lcl_atlas_bytes bytes, 256-byte
 * aligned).  Writes only *out; nothing is enqueued. */
lcl_status lcl_atlas_bind(void *base, size_t bytes, int32_t width, int32_t height, int32_t tile,
                          int64_t n_tri, lcl_atlas *out);

/* A view of texture rows [y0, y1) of `atlas` for lcl_overlay and lcl_label_area on a
 * band of the texture (layer pointers passed with it must point at row y0).  Requires
 * y0 * width to be a multiple of 32.  Selections reject views. */
lcl_status lcl_atlas_rows(const lcl_atlas *atlas, int32_t y0, int32_t y1, lcl_atlas *out);

/* A band atlas: rows [y0, y1) of a width x tex_height texture, with its own planes, coverage bits,
 * tile and super-tile boxes (tiles counted from row y0), in a buffer of
 * lcl_atlas_bytes(width, y1 - y0, tile, n_tri) bytes.  Texels are independent of one another
 * (Section 4.3.1 edits each texel by its own position and depth test), so one large texture can be
 * split into row bands, one per GPU: lcl_atlas_build fills a band with exactly the rows of the
 * whole atlas (texture coordinates are snapped against tex_height), every area weight included;
 * sphere, lasso and tool edits, overlays and per-label areas on a band give the rows of the whole
 * result (per-label counts and areas add up over the bands).  Texture padding reads texels up to 8
 * rows beyond a band, so padded edits on a band (height != tex_height) return LCL_ERR_UNSUPPORTED.
 * Writes only *out; nothing is enqueued. */
lcl_status lcl_atlas_bind_band(void *base, size_t bytes, int32_t width, int32_t tex_height, int32_t y0, int32_t y1,
                               int32_t tile, int64_t n_tri, lcl_atlas *out);

/* ---- atlas build -------------------------------------------------------- */

/* Device workspace bytes lcl_atlas_build needs for this mesh and texture. */
size_t lcl_atlas_workspace_bytes(const lcl_mesh *mesh, int32_t width, int32_t height);

/* Builds the atlas of `mesh`: the UV-space rasterisation of Section 4.3.1 (the mesh drawn
 * with its texture coordinates as positions, one fragment per texel), done once per model.
 *  1. bbox of all positions; scale = (2^21 - 1) / largest extent; every vertex quantised to
 *     the 21-bit grid, q = floor((p - bbox_min) * scale + 0.5) in double.
 *  2. texture coordinates snapped to 1/256 texel (round half to even); texel (i, j) is
 *     sampled at its centre; exact integer edge functions; a texel on an edge belongs to
 *     the triangle owning that edge (counter-clockwise triangles own edges running down, or
 *     left along a row); overlapping triangles: the smallest triangle id wins.
 *  3. position at the texel centre from exact barycentrics w_k / A: floor((2 sum w_k q_k + A)
 *     / (2 A)) per axis; coverage bits, tile and super-tile boxes.
 *  4. area weights (Section 5, Table 1: area one texel stands for): 3D area over UV area,
 *     floor(isqrt(|n|^2) * 2^24 / A) with n the grid-space normal, capped at 2^35 - 1.
 * mesh, atlas planes and workspace are device memory; the call waits for `stream`
 * before returning so that atlas->bbox_min and atlas->scale are valid on return.
 * Errors: LCL_ERR_INVALID_ARG for sizes, a flat or non-finite bbox, an index out of range or
 * texture coordinates outside [-1, 2] (the last three found on the device: the planes are
 * then undefined); LCL_ERR_OUT_OF_MEMORY if ws_bytes is too small. */
lcl_status lcl_atlas_build(const lcl_mesh *mesh, lcl_atlas *atlas, void *workspace, size_t ws_bytes,
                           lcl_stream stream);

/* ---- host helpers ------------------------------------------------------- */

/* Sphere stroke from a world-space centre and radius (host only): the centre is quantised
 * like a vertex but not clamped (LCL_ERR_INVALID_ARG outside [-2^22, 2^22 + 2^21]);
 * r2 = floor((radius * scale)^2), capped at 2^50 (above every in-grid squared distance). */
lcl_status lcl_quantize_sphere(const lcl_atlas *atlas, const double centre[3], double radius,
                               uint32_t label, lcl_sphere *out);

/* lcl_quantize_sphere for n strokes at once (host arrays: centres n x 3, radii n, labels n; out n).
 * Stops at the first invalid stroke and returns its error. */
lcl_status lcl_quantize_spheres(const lcl_atlas *atlas, int32_t n, const double *centres, const double *radii,
                                const uint32_t *labels, lcl_sphere *out);

/* Camera from a world view-projection `vp` (row-major, host): m = vp * Dequantise, with
 * Dequantise(q) = bbox_min + q / scale, composed in double and rounded to float. */
lcl_status lcl_camera_from_vp(const lcl_atlas *atlas, const double vp[16], int32_t width, int32_t height,
                              lcl_camera *out);

/* ---- edits -------------------------------------------------------------- */

/* Device workspace bytes for lcl_select_sphere / lcl_select_lasso with n strokes. */
size_t lcl_select_workspace_bytes(const lcl_atlas *atlas, int32_t n_strokes);

/* Sphere brush: the 3D counterpart of the paper's circular editing tool (Section 4.3).
 * For each stroke k in order, every covered texel with squared grid distance
 * (q - c)^2 <= r2 (int64) gets strokes[k].label; later strokes overwrite earlier ones; no
 * other texel changes.  Tiles whose box lies farther than r from c are skipped.
 *  layer: device, width x height labels of `dtype`, 16-byte aligned.
 *  strokes: host array of n records (copied into the launch; the array may be reused on
 *      return).  label must fit dtype; r2 >= 0 (values above 2^50 act as 2^50).
 *  hits_out: device, n uint64 (nullable): the number of texels each stroke selected.
 *  workspace: device, lcl_select_workspace_bytes(atlas, n) bytes. */
lcl_status lcl_select_sphere(const lcl_atlas *atlas, void *layer, lcl_dtype dtype, const lcl_sphere *strokes,
                             int32_t n, uint64_t *hits_out, void *workspace, size_t ws_bytes, lcl_stream stream);

#define LCL_STATIC_MAX_STROKES 4096   /* strokes per lcl_select_sphere_static call */
#define LCL_STATIC_MAX_TILES 262144   /* atlas tiles lcl_select_sphere_static supports (16384^2 at tile 32) */

/* The sphere brush without a workspace argument, for callers that cannot allocate device memory
 * when they edit: for example a plugin running inside a host application that owns the device
 * memory and its allocator, or an interactive editing loop that must not take allocator locks or
 * risk an allocation failure in the middle of a stroke.  (The paper has no counterpart: it edits
 * through the graphics pipeline, which keeps its own buffers.)
 * Same arguments, results and errors as lcl_select_sphere, whose work it does (its argument checks
 * run first), except that the scratch space (candidate counters and six tile lists, about 6 MiB)
 * is a fixed array compiled into the library, and the limits below.
 * Memory: the array belongs to the module of the library that holds it.  CUDA loads that module
 * into a context on first use, so the first call in each context (each device, or each context a
 * host application creates) loads it and allocates the ~6 MiB there; that first call can fail
 * with LCL_ERR_CUDA (out of memory).  Make it once, before the stroke loop and before any stream
 * capture; from then on the array stays until the context ends, and no call allocates or frees
 * anything.  Every call looks up the array's address in the current context (cudaGetSymbolAddress,
 * a host-side table lookup), so calls under different contexts of one device each use their own copy.
 * Limits: at most LCL_STATIC_MAX_STROKES strokes per call and atlases of at most
 * LCL_STATIC_MAX_TILES tiles; larger requests return LCL_ERR_UNSUPPORTED.
 * All calls in one context share the one array and it keeps the previous call's contents (each
 * call clears the counters it needs first): calls that could overlap on the GPU -- on different
 * streams, or from several host threads -- race and must be ordered on one stream. */
lcl_status lcl_select_sphere_static(const lcl_atlas *atlas, void *layer, lcl_dtype dtype, const lcl_sphere *strokes,
                                    int32_t n, uint64_t *hits_out, lcl_stream stream);

/* Device workspace bytes for lcl_depth_render. */
size_t lcl_depth_workspace_bytes(const lcl_mesh *mesh, int32_t width, int32_t height);

/* Depth texture (Section 4.3.1: scene depth from the current viewpoint, refreshed when the
 * camera changes).  Vertices quantised as in the atlas, projected by camera->m in FP32 in
 * the order ((m0 x + m1 y) + m2 z) + m3 without fused multiply-add; triangles with a corner
 * at w <= 0, NDC depth outside [0, 1] or more than 2^20 px off screen are dropped; screen
 * x = (x/w * 0.5 + 0.5) * width (row 0 at the bottom), snapped to 1/256 px; the same edge
 * and ownership rules as the atlas at pixel centres; depth = minimum over triangles of the
 * barycentric interpolation of corner NDC depth (double, rounded to float); +inf where
 * nothing is drawn.  depth: device float32, camera->height rows x camera->width. */
lcl_status lcl_depth_render(const lcl_mesh *mesh, const lcl_atlas *atlas, const lcl_camera *camera, float *depth,
                            void *workspace, size_t ws_bytes, lcl_stream stream);

/* Lasso selection: the paper's Texture Editing Algorithm (Section 4.3.1, Fig. 3) with the
 * tool shape given as a polygon: for every covered texel, project its grid position as in
 * lcl_depth_render; keep it if w > 0, NDC depth in [0, 1] and the point is on screen;
 * inside by the even-odd rule (an edge (a, b) counts when (a.y > y) != (b.y > y) and
 * x < (b.x - a.x) * (y - a.y) / (b.y - a.y) + a.x, FP32 in that order); visible iff
 * z <= depth[floor(y)][floor(x)] + bias (Fig. 3a, the depth test's small bias).  Selected texels get
 * `label`.  poly_xy: host, n_vertices (3..64) x 2 float32 screen pixels.  depth: device,
 * the map of the same camera.  flags: texture padding (Section 4.3.2) as for sphere strokes,
 * radius = bits 0-3, outline thickness = bits 4-7, both <= 8, other bits 0 (0 = none): uncovered
 * texels within the thickness of a covered texel and within the radius of a selected texel (square
 * kernels) get `label` too.  hits_out: device, one uint64 (nullable), selected texels (padded
 * texels not counted). */
lcl_status lcl_select_lasso(const lcl_atlas *atlas, void *layer, lcl_dtype dtype, const lcl_camera *camera,
                            const float *depth, const float *poly_xy, int32_t n_vertices, uint32_t label,
                            uint32_t flags, float bias, uint64_t *hits_out, void *workspace, size_t ws_bytes,
                            lcl_stream stream);

/* The paper's editing tool (Section 4.3.1, Fig. 3): a tool window of tw x th pixels centred on the
 * tool position (px, py) is mapped by projective texturing onto the tool's shape texture (the
 * scale and translate factors S_f, T_f), points outside it are discarded (Fig. 3b) and the shape
 * masks the rest (Fig. 3c), after the depth test with a small bias (Fig. 3a). */
typedef struct {
    float px, py;             /* tool position (window centre), screen pixels, row 0 at the bottom */
    float tw, th;             /* tool window size in pixels, > 0 (a circle of radius R: 2R x 2R) */
    const uint8_t *shape;     /* device, shape_h rows x shape_w bytes, row 0 at the bottom, non-zero =
                                 inside; NULL = the circle (ellipse) inscribed in the window */
    int32_t shape_w, shape_h; /* 1..4096 each when shape is given */
    uint32_t flags;           /* texture padding (Section 4.3.2) as for sphere strokes: radius = bits 0-3,
                                 outline thickness = bits 4-7, both <= 8, other bits 0; 0 = none */
    int32_t _pad;
} lcl_tool;

/* Tool selection: for every covered texel, the screen point (xs, ys) and depth test as in
 * lcl_select_lasso; then, in FP32 in this order,
 *   with a shape: fu = (xs - x0) * su, fv = (ys - y0) * sv, x0 = float(px - tw/2),
 *     su = float(shape_w / tw) (y0, sv likewise, each from double, rounded once); inside iff
 *     0 <= fu < shape_w, 0 <= fv < shape_h and shape[floor(fv)][floor(fu)] != 0;
 *   without: ex = (xs - px) * float(2/tw), ey = (ys - py) * float(2/th); inside iff
 *     ex*ex + ey*ey <= 1.
 * Selected texels get `label`; with padding flags, uncovered texels within the outline thickness
 * of a covered texel and within the radius of a selected texel (square kernels) get it too.
 * Workspace: lcl_select_workspace_bytes(atlas, 1).  hits_out: device, one uint64 (nullable),
 * selected texels (padded texels not counted).  Errors: as lcl_select_lasso;
 * LCL_ERR_INVALID_ARG for a non-finite or non-positive window, shape sizes outside 1..4096 or
 * padding flags out of range. */
lcl_status lcl_select_tool(const lcl_atlas *atlas, void *layer, lcl_dtype dtype, const lcl_camera *camera,
                           const float *depth, const lcl_tool *tool, uint32_t label, float bias, uint64_t *hits_out,
                           void *workspace, size_t ws_bytes, lcl_stream stream);

/* ---- batched edits -------------------------------------------------------- */

#define LCL_BATCH_MAX_STROKES 64  /* queued strokes per model per batch */
enum { LCL_STROKE_SPHERE = 0, LCL_STROKE_LASSO = 1 };

/* One model of a batch: its built atlas (host struct), the layer its strokes edit, and its queue:
 * strokes [first_stroke, first_stroke + n_strokes) of the batch's stroke array, in queue order. */
typedef struct {
    const lcl_atlas *atlas;
    void *layer; /* device, 16-byte aligned */
    lcl_dtype dtype;
    int32_t first_stroke, n_strokes;
    int32_t _pad;
} lcl_batch_model;

/* One queued stroke: a sphere (kind LCL_STROKE_SPHERE, `sphere`) or a lasso (kind LCL_STROKE_LASSO,
 * `lasso` indexes the batch's lasso array). */
typedef struct {
    int32_t kind, lasso;
    lcl_sphere sphere;
} lcl_batch_stroke;

/* One lasso of a batch: camera, its depth map (device), polygon (host, n_vertices x 2 floats),
 * label and bias, with the meaning of lcl_select_lasso. */
typedef struct {
    lcl_camera camera;
    const float *depth;
    const float *poly_xy;
    int32_t n_vertices;
    uint32_t label;
    float bias;
    uint32_t flags; /* texture padding as for lcl_select_lasso (0 = none) */
} lcl_batch_lasso;

/* Capacity of a batch workspace: every batch run on it has at most `models` models, `strokes`
 * strokes, `lassos` lassos, and its models' atlases have at most `supers` super-tiles and `tiles`
 * tiles in total.  The workspace layout and the launch shape depend only on the limits and the
 * config, and the kernels read the actual counts from the workspace, so one launch (or one
 * captured CUDA graph) serves every batch uploaded within the same limits. */
typedef struct {
    int32_t models, strokes, lassos, _pad;
    int64_t supers, tiles;
} lcl_batch_limits;

/* Launch shape of the batched apply (all zero = the default {256, 0, 1}):
 *   threads      threads per CTA: 64, 128 or 256;
 *   ctas_per_sm  CTAs per SM, 0 = as many as fit, else 1..32 (capped at what fits);
 *   split        parts each (model, tile) work item is cut into (contiguous rows of the tile),
 *                1, 2, 4 or 8; a part is the unit a CTA takes from the work queue.
 * Results do not depend on it. */
typedef struct {
    int32_t threads, ctas_per_sm, split, _pad;
} lcl_batch_config;

/* The limits of exactly this batch (sums over its models).  Errors: LCL_ERR_INVALID_ARG. */
lcl_status lcl_batch_limits_of(const lcl_batch_model *models, int32_t n_models, int32_t n_strokes, int32_t n_lassos,
                               lcl_batch_limits *out);
/* Device workspace and host staging bytes for a batch workspace of these limits (0 if invalid). */
size_t lcl_batch_workspace_bytes(const lcl_batch_limits *limits);
size_t lcl_batch_staging_bytes(const lcl_batch_limits *limits);

/* Checks a batch against the limits, packs its model, stroke and lasso descriptors into
 * host_staging (lcl_batch_staging_bytes, host memory) and copies them to the workspace on
 * `stream`; with pinned memory the copy is asynchronous and the staging must stay untouched until
 * the stream has passed it.  No kernel runs.  Models must be distinct layers (two models writing
 * one layer race); depth maps must be rendered before the batch is launched.
 * Errors: LCL_ERR_INVALID_ARG (bad descriptors, counts above the limits), LCL_ERR_UNSUPPORTED (more
 * than LCL_BATCH_MAX_STROKES strokes for a model, lassos outside 3..64
 * vertices), LCL_ERR_OUT_OF_MEMORY (workspace or staging smaller than required), LCL_ERR_CUDA. */
lcl_status lcl_batch_upload(const lcl_batch_limits *limits, const lcl_batch_model *models, int32_t n_models,
                            const lcl_batch_stroke *strokes, int32_t n_strokes, const lcl_batch_lasso *lassos,
                            int32_t n_lassos, void *workspace, size_t ws_bytes, void *host_staging,
                            size_t staging_bytes, lcl_stream stream);

/* Edits the models of the batch last uploaded to `workspace`: every model's queued strokes are
 * applied to its layer in queue order, with results identical to calling lcl_select_sphere /
 * lcl_select_lasso once per stroke in that order (Section 4.3.1 applied per stroke; batching is a
 * serving-side schedule the paper does not discuss).  Two cull launches give every touched tile of
 * every model a mask of the strokes that can reach it (tested per (super-tile, stroke) pair, then
 * compacted into work items); one persistent apply launch takes
 * (model, tile part) units from a work queue, loads each texel's position once and evaluates its
 * masked strokes from the newest down, stopping at the first that selects it (the label the
 * sequence leaves).  No host-to-device copy and a launch shape fixed by (limits, config): the call
 * can be captured in a CUDA graph and replayed after later uploads.  Launching a batch again
 * repeats its strokes, which leaves every label as it is.  config may be NULL (default).
 * Errors: LCL_ERR_INVALID_ARG (limits, config, workspace), LCL_ERR_CUDA. */
lcl_status lcl_batch_launch(const lcl_batch_limits *limits, const lcl_batch_config *config, void *workspace,
                            size_t ws_bytes, lcl_stream stream);

/* lcl_batch_upload followed by lcl_batch_launch. */
lcl_status lcl_batch_edit(const lcl_batch_limits *limits, const lcl_batch_config *config,
                          const lcl_batch_model *models, int32_t n_models, const lcl_batch_stroke *strokes,
                          int32_t n_strokes, const lcl_batch_lasso *lassos, int32_t n_lassos, void *workspace,
                          size_t ws_bytes, void *host_staging, size_t staging_bytes, lcl_stream stream);

/* Autotuner: launches the batch last uploaded to `workspace` under each candidate launch shape
 * (threads 64/128/256 x split 1/2/4/8 x CTAs per SM as many as fit / half of that), `reps` timed
 * launches each after one warm-up, timed with CUDA events on `stream`, and writes the fastest
 * shape and its mean time per launch.  Synchronises the stream.  The batch's strokes are applied
 * (1 + reps) x candidates times, which leaves the same labels as one application.
 * Errors: LCL_ERR_INVALID_ARG, LCL_ERR_CUDA. */
lcl_status lcl_batch_tune(const lcl_batch_limits *limits, void *workspace, size_t ws_bytes, int32_t reps,
                          lcl_stream stream, lcl_batch_config *best, float *best_ms);

/* ---- served edits (native request loop) ------------------------------------ */

/* A request server: many models' atlases, layers and depth maps kept in device memory while a budget
 * allows, edit and query requests arriving continuously, batched into launches.  The paper keeps all
 * layers on the GPU and lets the CPU only manage (Section 4, Fig. 2), its texture manager commits
 * texture memory on demand (Section 4.2), and every request performs the edit of Section 4.3.1; the
 * server is that manager for many models at once:
 *  - resident models: a model's device image (atlas buffer | layers | depth maps) lives in a caller
 *    arena (the HBM budget) while it fits; a model that has work and is not resident is admitted by a
 *    host-to-device copy of its image on a copy stream, evicting idle resident models with the lowest
 *    recent request rate (requests decayed with a 1 s time constant), whose layers are first copied
 *    back to their host images; a model's requests join the first epoch after its copy completed;
 *  - per-model FIFO order; continuous batching: each epoch takes, for every ready model with queued
 *    work, the leading run of edits (at most max_edits per layer) and the query that follows them, if
 *    any, uploads the edits as one batch (lcl_batch_upload) and replays a captured graph of
 *    lcl_batch_launch, then the queries
 *    (lcl_overlay into scratch + lcl_label_area, the tables copied to the request's host buffer);
 *    epochs overlap (max_in_flight), each with its own workspace, staging and graph;
 *  - open-loop arrivals: requests are submitted with their arrival times on the server clock and
 *    taken only once that time has come; a request is done when the host sees its epoch's completion
 *    event (t_done, same clock).
 * The loop runs in a host thread of the server (lcl_serve_start .. lcl_serve_destroy); the calls
 * below may come from any one other thread.  Device memory is the caller's (arena and work buffer);
 * the server object holds host memory (queues, copies of the requests), two streams and events. */
typedef struct lcl_server lcl_server;

enum { LCL_REQ_SPHERE = 0, LCL_REQ_LASSO = 1, LCL_REQ_QUERY = 2 };

typedef struct {
    size_t arena_bytes;     /* device arena for model images: the HBM budget */
    int32_t max_in_flight;  /* epochs in flight, 1..8 (0: 4) */
    int32_t max_edits;      /* edits per layer per epoch, 1..LCL_BATCH_MAX_STROKES (0: 64) */
    int32_t max_queries;    /* queries per epoch, 1..1024 (0: 16) */
    int32_t max_labels;     /* largest n_labels of a query, 1..65536 (0: 256) */
    int32_t max_admitting;  /* admissions in flight, 1..1024 (0: 16) */
    int32_t _pad;
} lcl_serve_config;

/* A model, registered from its host image: pinned host memory of image_bytes bytes holding exactly
 * the device image [atlas buffer of lcl_atlas_bytes(side, side, tile, n_tri) bytes (built) |
 * n_layers uint8 layers of side x side at layer_offset + k layer_stride | depth map c (float32,
 * cams[c].height x cams[c].width) at depth_offsets[c]], offsets 256-byte aligned.  The server copies
 * it in on admission and writes the layers back on eviction; the caller keeps it alive and untouched
 * until lcl_serve_destroy.  cams and depth_offsets are copied. */
typedef struct {
    int32_t side, tile;
    int64_t n_tri;
    float bbox_min[3];   /* the built atlas's quantisation */
    int32_t n_layers;
    double scale;
    const lcl_camera *cams;
    const size_t *depth_offsets;
    int32_t n_cams, _pad;
    void *host_image;
    size_t image_bytes, layer_offset, layer_stride;
} lcl_serve_model;

/* One request.  Sphere: centre and radius in world units (quantised with lcl_quantize_sphere),
 * `label` into `layer`.  Lasso: polygon of n_vertices (3..64) screen pixels on camera `cam`, `label`
 * into `layer`, bias 2^-10.  Query: the overlay op(layer, layer_b) (an lcl_op, no flags) and its
 * per-label counts and areas over n_labels labels, written to result (host, 2 n_labels uint64:
 * counts then areas) before the request is reported done. */
typedef struct {
    double t_arrive;    /* seconds on the server clock (lcl_serve_clock) */
    uint64_t tag;       /* returned by lcl_serve_poll */
    int32_t model, kind, layer, label;
    double centre[3], radius;
    int32_t cam, n_vertices;
    int32_t op, layer_b, n_labels, _pad;
    uint64_t *result;
    float poly[2 * LCL_MAX_LASSO_VERTICES];
} lcl_serve_request;

typedef struct {
    uint64_t tag;
    double t_done;      /* server clock: the host saw the request's epoch complete */
    double t_launch;    /* server clock: its epoch was launched */
    double t_gpu;       /* seconds the GPU spent on its epoch (CUDA events before and after the epoch's
                           work on the compute stream), -1 if unavailable */
} lcl_serve_done;

typedef struct {
    uint64_t submitted, done, epochs, admissions, spills;
    uint64_t resident_bytes, resident_models;
    double host_busy_s;        /* loop time spent building epochs, admitting and spilling */
    uint64_t admitted_bytes;   /* bytes copied in by admissions */
    uint64_t deferred;         /* admissions put off: no room could be made at that moment */
} lcl_serve_stats;

/* Seconds on the server clock (a monotonic host clock). */
double lcl_serve_clock(void);

/* Creates a server on the current device.  Errors: LCL_ERR_INVALID_ARG. */
lcl_status lcl_serve_create(const lcl_serve_config *config, lcl_server **out);

/* Registers a model (before lcl_serve_start); *id = its index.  Errors: LCL_ERR_INVALID_ARG (sizes,
 * layout, an image larger than the arena), LCL_ERR_UNSUPPORTED (after start). */
lcl_status lcl_serve_add_model(lcl_server *server, const lcl_serve_model *model, int32_t *id);

/* Device and pinned host work memory the server needs for its registered models (batch workspaces,
 * staging, query scratch), for lcl_serve_start. */
size_t lcl_serve_work_bytes(const lcl_server *server);
size_t lcl_serve_host_work_bytes(const lcl_server *server);

/* Starts the loop thread.  arena: device, config.arena_bytes, 256-byte aligned; work: device,
 * lcl_serve_work_bytes; host_work: pinned host, lcl_serve_host_work_bytes.  When host_work is mapped
 * into the device's address space (pinned memory under unified addressing is), each epoch reads its
 * descriptors from it and writes its query tables to it with copy kernels, so epochs do not wait
 * behind admission and spill copies on the copy engines; otherwise they use cudaMemcpyAsync.  Models
 * are admitted in registration order while they fit.  Errors: LCL_ERR_INVALID_ARG, LCL_ERR_CUDA. */
lcl_status lcl_serve_start(lcl_server *server, void *arena, void *work, size_t work_bytes, void *host_work,
                           size_t host_work_bytes);

/* Queues n requests (copied), in order of arrival time (non-decreasing t_arrive over all submits).
 * Errors: LCL_ERR_INVALID_ARG (a bad model, layer, camera, label, polygon or query), nothing queued. */
lcl_status lcl_serve_submit(lcl_server *server, const lcl_serve_request *requests, int32_t n);

/* Takes up to max completions (in completion order); *n_out = how many.  Non-blocking.  A failure of
 * the loop (a CUDA error) is returned here as LCL_ERR_CUDA. */
lcl_status lcl_serve_poll(lcl_server *server, lcl_serve_done *out, int32_t max, int32_t *n_out);

lcl_status lcl_serve_stats_get(lcl_server *server, lcl_serve_stats *out);

/* Copies layer `layer` of model `model` (side x side bytes) to host memory `dst`, once every
 * submitted request is done (waits for that).  Errors: LCL_ERR_INVALID_ARG, LCL_ERR_CUDA. */
lcl_status lcl_serve_read_layer(lcl_server *server, int32_t model, int32_t layer, void *dst);

/* Stops the loop (queued requests that have not run are dropped), waits for the device, destroys
 * the streams and the server. */
lcl_status lcl_serve_destroy(lcl_server *server);

/* ---- layer operations --------------------------------------------------- */

/* Boolean overlay of two layers (layer systems combine layers with logic operations,
 * Section 3.4.2): per texel, a' = NOT_A ? ~a : a, b' = NOT_B ? ~b : b (within the label
 * width), r = a' & b' | a' | b' | a' ^ b' | (b' != 0 ? a' : 0) for AND, OR, XOR, MASK,
 * out = NOT_OUT ? ~r : r; uncovered texels get 0.  a, b, out: device layers of `dtype`;
 * out may alias a or b. */
lcl_status lcl_overlay(const lcl_atlas *atlas, const void *a, const void *b, void *out, lcl_dtype dtype, lcl_op op,
                       uint32_t flags, lcl_stream stream);

/* Per-label surface area (Section 5, Table 1: the area one texel stands for): over covered
 * texels with label l < n_labels, count_out[l] = number of texels and area_out[l] = sum of
 * their triangles' area weights (grid^2 units with 8 fractional bits; physical area =
 * area * 2^-8 / scale^2).  Labels >= n_labels are ignored.  count_out, area_out: device,
 * n_labels uint64 each (overwritten).  n_labels in [1, 65536]. */
lcl_status lcl_label_area(const lcl_atlas *atlas, const void *layer, lcl_dtype dtype, uint32_t n_labels,
                          uint64_t *count_out, uint64_t *area_out, lcl_stream stream);

/* ---- numeric layers ------------------------------------------------------- */

/* Numeric layers (Section 4.2): besides label layers, a layer can hold numeric properties
 * (curvature, rugosity, age ...) as a data texture of integers (8, 16 or 32 bits) or floats
 * (16 or 32 bits) with a mask texture that tells which texels hold valid data.  Type codes:
 * low nibble = bytes per texel, high nibble = 1 unsigned, 2 signed, 3 IEEE float. */
typedef enum {
    LCL_NUM_U8 = 0x11, LCL_NUM_U16 = 0x12, LCL_NUM_U32 = 0x14,
    LCL_NUM_I8 = 0x21, LCL_NUM_I16 = 0x22, LCL_NUM_I32 = 0x24,
    LCL_NUM_F16 = 0x32, LCL_NUM_F32 = 0x34
} lcl_num_type;

/* A numeric layer: data, device, width x height values of `type`, row-major, 16-byte aligned;
 * mask, device, one bit per texel, bit (y * width + x) of a linear uint32 array
 * ((width * height + 31) / 32 words, 16-byte aligned), set = the texel holds data.  Values are
 * passed to and from the library as their bit patterns in a uint32 (float16: the 16 bits of the
 * binary16 value; narrower integers: the value's bits in the low bits, higher bits 0). */
typedef struct {
    void *data;
    uint32_t *mask;
    lcl_num_type type;
    int32_t _pad;
} lcl_numeric_layer;

#define LCL_ERASE 0x100u  /* numeric edit flag: store 0 and clear the mask instead of the value */

/* Sphere strokes on a numeric layer: the texels lcl_select_sphere would select (texture padding
 * included, flags bits 0-7) get the stroke's value -- the bits in strokes[k].label -- in the data
 * texture and a set mask bit, the last step of Section 4.3.1 (the selected value is stored in the
 * data texture and true in the mask texture); with LCL_ERASE in flags they get 0 and a clear mask
 * bit.  hits_out, workspace: as lcl_select_sphere.  Errors: as lcl_select_sphere;
 * LCL_ERR_INVALID_ARG for a value wider than the type or flags outside bits 0-8. */
lcl_status lcl_numeric_sphere(const lcl_atlas *atlas, const lcl_numeric_layer *layer, const lcl_sphere *strokes,
                              int32_t n, uint64_t *hits_out, void *workspace, size_t ws_bytes, lcl_stream stream);

/* A lasso on a numeric layer: the texels lcl_select_lasso would select or pad (flags bits 0-7) get
 * `value` and a set mask bit (with LCL_ERASE in flags: 0 and a clear bit). */
lcl_status lcl_numeric_lasso(const lcl_atlas *atlas, const lcl_numeric_layer *layer, const lcl_camera *camera,
                             const float *depth, const float *poly_xy, int32_t n_vertices, uint32_t value,
                             uint32_t flags, float bias, uint64_t *hits_out, void *workspace, size_t ws_bytes,
                             lcl_stream stream);

/* The paper's tool on a numeric layer (tool->flags: padding as for lcl_select_tool; flags:
 * LCL_ERASE or 0). */
lcl_status lcl_numeric_tool(const lcl_atlas *atlas, const lcl_numeric_layer *layer, const lcl_camera *camera,
                            const float *depth, const lcl_tool *tool, uint32_t value, uint32_t flags, float bias,
                            uint64_t *hits_out, void *workspace, size_t ws_bytes, lcl_stream stream);

typedef enum { LCL_ADD = 0, LCL_SUB = 1, LCL_MUL = 2, LCL_DIV = 3, LCL_MIN = 4, LCL_MAX = 5 } lcl_arith;

/* Arithmetic overlay of numeric layers (layer systems compute arithmetic operations between layers,
 * Section 3.4.2): out = a <op> b per texel, all three of one type; b == NULL uses the scalar `b_value`
 * (bits, always valid) for every texel.  Integers: add, subtract and multiply modulo 2^bits
 * (two's complement), min / max by signed or unsigned value, no division.  float32: IEEE single,
 * round to nearest even.  float16: both operands widened to float32 (exact), one float32 operation,
 * the result rounded to float16 (nearest even) -- the correctly rounded float16 operation.  MIN /
 * MAX: a < b ? a : b and a > b ? a : b.  A result is valid where a, b (if given) are valid and the
 * texel is covered; other texels get data 0 and a clear mask bit.  out may alias a or b (data and
 * mask).  NaN results are NaN, their bit pattern is not specified.
 * Errors: LCL_ERR_INVALID_ARG (types differ, bad pointers, scalar wider than the type);
 * LCL_ERR_UNSUPPORTED (LCL_DIV on integers). */
lcl_status lcl_numeric_arith(const lcl_atlas *atlas, const lcl_numeric_layer *a, const lcl_numeric_layer *b,
                             uint32_t b_value, const lcl_numeric_layer *out, lcl_arith op, lcl_stream stream);

typedef enum { LCL_LT = 0, LCL_LE = 1, LCL_GT = 2, LCL_GE = 3, LCL_EQ = 4, LCL_NE = 5 } lcl_cmp;

/* Selection by value, from a numeric layer into a label layer: covered texels whose mask bit is set
 * and whose value v satisfies v <cmp> threshold (bits of the layer's type; integers compare by
 * value, floats as IEEE floats, a NaN satisfies only LCL_NE) get `label`; no other texel changes.
 * hits_out: device, one uint64 (nullable), the number of texels selected. */
lcl_status lcl_numeric_select(const lcl_atlas *atlas, const lcl_numeric_layer *values, lcl_cmp cmp,
                              uint32_t threshold, void *layer, lcl_dtype dtype, uint32_t label, uint64_t *hits_out,
                              lcl_stream stream);

/* Zonal statistics of one zone (48 bytes). */
typedef struct {
    uint64_t count;  /* texels */
    uint64_t area;   /* sum of their area weights (as lcl_label_area) */
    double vmin, vmax;  /* smallest and largest value (+inf / -inf for an empty zone) */
    double sum;      /* sum of the values */
    double wsum;     /* sum of area weight x value: the integral over the zone's surface */
} lcl_zone_stats;

/* Zonal statistics of a numeric layer over the zones of a label layer (quantitative layers measured
 * with the area one texel stands for, Section 5, Table 1): over covered texels whose mask bit is
 * set, whose value is not NaN and whose zone label z < n_labels (zones == NULL: every such texel is
 * in zone 0 and n_labels must be 1), per zone: count, area, min, max (values as double; -0 counts
 * as +0), sum of values and sum of weight x value in double.  count, area, vmin and vmax are
 * exact; the sums are accumulated in an unspecified order, the weighted one per stretch of texels
 * of one triangle as weight x (sum of their values): errors at most (count - 1) * 2^-53 * sum |v|
 * for sum and 2 * count * 2^-53 * sum |w v| for wsum.  out: device, n_labels records (overwritten).  n_labels in [1, 65536]. */
lcl_status lcl_numeric_stats(const lcl_atlas *atlas, const lcl_numeric_layer *values, const void *zones,
                             lcl_dtype zone_dtype, uint32_t n_labels, lcl_zone_stats *out, lcl_stream stream);

/* ---- sparse layer pool ------------------------------------------------------ */

/* The texture manager of Section 4.2: layers of one (width, height, type) live in one texture array
 * found by a hash of that key, and sparse textures separate reserving room for many layers from
 * committing memory to the layers in use.  Here a key's array is a reserved range of device virtual
 * addresses with max_layers_per_array equal slots (a slot holds a layer's data texture and, for
 * numeric types, its mask bits, rounded up to the allocation granularity); acquiring a layer
 * creates and maps physical memory for one slot, releasing it unmaps and frees that memory.  A
 * layer's address never changes while it lives.  This is the one part of the library that
 * allocates device memory, and only inside these calls.  A pool belongs to the device that was
 * current at lcl_pool_create; its calls may come from several host threads. */
typedef struct lcl_pool lcl_pool;

typedef struct {
    void *data;       /* device: width x height values of the type, row-major, 256-byte aligned */
    uint32_t *mask;   /* device: mask bits of a numeric layer (lcl_numeric_layer.mask), NULL for label layers */
    uint64_t handle;  /* names the layer to lcl_pool_release */
    int32_t width, height;
    int32_t type;     /* LCL_U8 / LCL_U16 (label layer) or an lcl_num_type (numeric layer) */
    int32_t _pad;
} lcl_pool_layer;

typedef struct {
    uint64_t reserved_bytes;   /* virtual address space reserved by all arrays */
    uint64_t committed_bytes;  /* physical device memory mapped for live layers */
    int64_t layers;            /* live layers */
    int32_t arrays;            /* distinct (width, height, type) keys seen */
    int32_t _pad;
    uint64_t granularity;      /* allocation granularity (bytes) */
} lcl_pool_stats;

/* Creates an empty pool on the current device.  max_layers_per_array in [1, 2^20]: the slots each
 * array reserves address space for.  Errors: LCL_ERR_INVALID_ARG; LCL_ERR_CUDA without a device or
 * without the driver's virtual-memory entry points. */
lcl_status lcl_pool_create(int32_t max_layers_per_array, lcl_pool **out);

/* Commits one layer of (width, height, type) -- width a multiple of 4 in [4, 16384], height in
 * [1, 16384] -- and enqueues on `stream` the clearing of its data and mask to 0 ("no data"); use
 * the layer on other streams only after that.  Errors: LCL_ERR_INVALID_ARG;
 * LCL_ERR_OUT_OF_MEMORY when the key's slots are all in use or the device has no memory left;
 * LCL_ERR_CUDA. */
lcl_status lcl_pool_acquire(lcl_pool *pool, int32_t width, int32_t height, int32_t type, lcl_stream stream,
                            lcl_pool_layer *out);

/* Releases a layer: synchronises `stream` (every other stream that used the layer must have been
 * synchronised by the caller), then unmaps and frees its memory; the slot can be acquired again.
 * Errors: LCL_ERR_INVALID_ARG for a handle that names no live layer of this pool; LCL_ERR_CUDA. */
lcl_status lcl_pool_release(lcl_pool *pool, uint64_t handle, lcl_stream stream);

lcl_status lcl_pool_stats_get(lcl_pool *pool, lcl_pool_stats *out);

/* Synchronises the device, releases every live layer and the reserved ranges, frees the pool. */
lcl_status lcl_pool_destroy(lcl_pool *pool);

/* ---- diagnostics -------------------------------------------------------- */

const char *lcl_status_str(lcl_status status);
/* One-line reason for the last non-OK status returned on this thread ("" if none). */
const char *lcl_last_error(void);
/* Number of kernels this library has launched in this process (all devices). */
uint64_t lcl_kernel_launches(void);

/* Device-side status of the work enqueued so far (the CPU manages, the GPU computes and keeps the
 * data: Section 4, Fig. 2 -- so faults and checks made on the GPU have to be fetched by the CPU).
 * Synchronises `stream`; returns LCL_ERR_CUDA (with the CUDA error text) if the stream reports an
 * error.  In a library built with bounds checks (lcl_build_flags() & LCL_BUILD_BOUNDS_CHECKS, the
 * LCL_DEBUG_BOUNDS build), every index a kernel computes into a plane, layer, candidate list,
 * depth map or table is checked before its access; an index out of range skips that access (no
 * trap: the context stays usable) and is counted, and this call returns LCL_ERR_INTERNAL with
 * lcl_last_error() naming the first such site (file:line), its index and the buffer's extent, then
 * clears the records.  Kernels on other streams must have finished (synchronise them first) for
 * their checks to be seen.  In the normal build there are no checks and the call returns LCL_OK
 * once the stream has finished without error.  No kernel of this library waits on another, so
 * no call returns LCL_ERR_TIMEOUT (reserved). */
lcl_status lcl_last_device_status(lcl_stream stream);

/* Self-check of the library's division (device diagnostic).  The edits project texels with IEEE
 * binary32 division (Section 4.3.1's projective texturing, written out in lcl_select_lasso); the
 * library computes it on a faster route for operands in [2^-30, 2^31) and must give exactly the
 * correctly rounded quotient everywhere.  This call compares the two on n operand pairs drawn
 * from `seed` (random operands across and beyond that window, quotients next to rounding
 * midpoints, the window's edges, zeros, subnormals, infinities, NaN).  For each pair with a
 * positive divisor it also checks the depth test's decisions on the quotient (q >= 0 and q <= t,
 * taken without dividing where one FMA settles them) against the same tests on the correctly
 * rounded quotient, for t on the quotient, one ulp either side, 1 and a random value.  It adds to
 * counts[0] the checks made (at least n) and to counts[1] those that differ (NaN equals NaN).
 * counts: device, two uint64 (not cleared by the call). */
lcl_status lcl_check_division(uint64_t n, uint32_t seed, uint64_t *counts, lcl_stream stream);

#define LCL_BUILD_BOUNDS_CHECKS 1u  /* lcl_build_flags bit: kernels check their indices */
/* How this library was built (LCL_BUILD_* bits). */
uint32_t lcl_build_flags(void);

/* Writes "file:line" of a bounds-check site as recorded on the device (site = 16-bit hash of the
 * source file name << 16 | line) into buf (n bytes, NUL-terminated; buf may be NULL) and returns
 * the full length.  Unknown files are written as "file#hhhh:line". */
size_t lcl_describe_site(uint32_t site, char *buf, size_t n);

#ifdef __cplusplus
}
#endif
#endif /* LCL_H */
