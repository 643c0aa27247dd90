// noalloc.cu -- lcl_select_sphere_static: the sphere brush for callers that cannot allocate
// device memory, with its scratch space in a fixed array compiled into this library.
//
// The scratch (per-stroke candidate counters and the candidate-tile lists) lives in the
// file-scope device array below, which exists once in every CUDA context that has loaded this
// file's module and stays until that context ends.  Host code cannot hand the array's name to a
// kernel (on the host it is only a stand-in for the device symbol), so every call looks up the
// device address with cudaGetSymbolAddress in the context current at the call and passes it on
// as the workspace of the ordinary lcl_select_sphere.  The lookup is not cached: a cached
// address would be wrong for a call made under another context of the same device (a host
// application's own driver context, or one re-created after cudaDeviceReset).  Nothing here
// calls cudaMalloc, cudaFree or any allocating library routine; the one allocation is the
// module load itself (see the header).
#include "lcl_impl.cuh"

namespace lcl {
namespace {

constexpr int32_t kStaticMaxStrokes = LCL_STATIC_MAX_STROKES;
constexpr int64_t kStaticMaxTiles = LCL_STATIC_MAX_TILES;
// Candidate counters (two per stroke) and six tile lists (three for per-stroke candidates, three
// more for the second item set of grouped calls), laid out as the workspace of lcl_select_sphere for
// kStaticMaxStrokes strokes on an atlas of kStaticMaxTiles tiles.
constexpr size_t kStaticScratchBytes =
    ((size_t(2) * (kStaticMaxStrokes + 1) * 4 + 255) & ~size_t(255)) + 6 * size_t(kStaticMaxTiles) * 4;

static __device__ __align__(256) unsigned char g_sphere_scratch[kStaticScratchBytes];

}  // namespace
}  // namespace lcl

using namespace lcl;

extern "C" lcl_status lcl_select_sphere_static(const lcl_atlas *atlas, void *layer, lcl_dtype dtype,
                                               const lcl_sphere *strokes, int32_t n, uint64_t *hits_out,
                                               lcl_stream stream) {
    bool proceed = false;
    lcl_status s = check_sphere_call(atlas, layer, dtype, strokes, n, hits_out, &proceed);
    if (s != LCL_OK || !proceed) return s;
    if (n > kStaticMaxStrokes)
        return fail(LCL_ERR_UNSUPPORTED, "lcl_select_sphere_static takes at most LCL_STATIC_MAX_STROKES (4096) "
                                         "strokes per call");
    if ((int64_t)atlas->tiles_x * atlas->tiles_y > kStaticMaxTiles)
        return fail(LCL_ERR_UNSUPPORTED, "lcl_select_sphere_static supports atlases of at most "
                                         "LCL_STATIC_MAX_TILES (262144) tiles");
    void *scratch = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&scratch, g_sphere_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "lcl_select_sphere_static: cudaGetSymbolAddress of the scratch array");
    if (select_ws_bytes(atlas, n) > kStaticScratchBytes)
        return fail(LCL_ERR_INTERNAL, "lcl_select_sphere_static: scratch array smaller than the workspace layout");
    return lcl_select_sphere(atlas, layer, dtype, strokes, n, hits_out, scratch, kStaticScratchBytes, stream);
}
