// noalloc.cu -- lcl_select_sphere_static: the sphere brush for callers that cannot allocate
// device memory, with its scratch space in a fixed array compiled into this library.
//
// The scratch (per-stroke candidate counters and the candidate-tile lists) lives in the
// file-scope device array below: every GPU that loads the library holds it until the process
// exits.  Host code cannot hand the array's name to a kernel (on the host it is only a
// stand-in for the device symbol), so the device address is looked up once per device with
// cudaGetSymbolAddress, with that device current, and passed on as the workspace of the
// ordinary lcl_select_sphere.  Nothing here calls cudaMalloc, cudaFree or any allocating
// library routine.
#include <mutex>

#include "lcl_impl.cuh"

namespace lcl {
namespace {

constexpr int32_t kStaticMaxStrokes = LCL_STATIC_MAX_STROKES;
constexpr int64_t kStaticMaxTiles = LCL_STATIC_MAX_TILES;
// Candidate counters (one per stroke) and three candidate-tile lists, laid out as the workspace
// of lcl_select_sphere for kStaticMaxStrokes strokes on an atlas of kStaticMaxTiles tiles.
constexpr size_t kStaticScratchBytes =
    ((size_t(kStaticMaxStrokes + 1) * 4 + 255) & ~size_t(255)) + 3 * size_t(kStaticMaxTiles) * 4;

static __device__ __align__(256) unsigned char g_sphere_scratch[kStaticScratchBytes];

std::mutex g_setup_mu;
void *g_scratch_addr[64] = {nullptr};

// Device address of the scratch array on the current device (looked up on first use).
lcl_status scratch_address(void **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "lcl_select_sphere_static: cudaGetDevice");
    if (dev < 0 || dev >= 64) return fail(LCL_ERR_UNSUPPORTED, "lcl_select_sphere_static: device index above 63");
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_sphere_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "lcl_select_sphere_static: cudaGetSymbolAddress");
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return LCL_OK;
}

}  // namespace
}  // namespace lcl

using namespace lcl;

extern "C" lcl_status lcl_select_sphere_static(const lcl_atlas *atlas, void *layer, lcl_dtype dtype,
                                               const lcl_sphere *strokes, int32_t n, uint64_t *hits_out,
                                               lcl_stream stream) {
    if (!atlas) return fail(LCL_ERR_INVALID_ARG, "atlas is NULL");
    if (n > kStaticMaxStrokes)
        return fail(LCL_ERR_UNSUPPORTED, "lcl_select_sphere_static takes at most LCL_STATIC_MAX_STROKES (4096) "
                                         "strokes per call");
    if ((int64_t)atlas->tiles_x * atlas->tiles_y > kStaticMaxTiles)
        return fail(LCL_ERR_UNSUPPORTED, "lcl_select_sphere_static supports atlases of at most "
                                         "LCL_STATIC_MAX_TILES (262144) tiles");
    void *scratch = nullptr;
    lcl_status s = scratch_address(&scratch);
    if (s != LCL_OK) return s;
    return lcl_select_sphere(atlas, layer, dtype, strokes, n, hits_out, scratch, kStaticScratchBytes, stream);
}
