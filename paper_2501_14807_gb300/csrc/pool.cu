// pool.cu -- sparse layer pool: the paper's texture manager (arXiv 2501.14807, Section 4.2) on CUDA
// virtual memory management.
//
// The paper keeps textures of one (width, height, data type) in one texture array, found through a
// hash of that key, and uses sparse textures so that a texture array can reserve room for very
// many layers while physical memory is committed only for the layers in use.  Here a key's array
// is one reserved range of device virtual addresses with a fixed number of equal slots; a layer
// occupies one slot, whose physical memory is created and mapped when the layer is acquired and
// unmapped and released when it is released.  A layer's device address never changes while it
// lives, and an acquired layer starts zeroed (label 0 / mask clear: "no data").
//
// The driver's virtual-memory entry points are looked up through the runtime
// (cudaGetDriverEntryPointByVersion), so the library needs no link against the driver library.
#include <cuda.h>

#include <cstring>
#include <mutex>
#include <unordered_map>
#include <vector>

#include "lcl_impl.cuh"

struct lcl_pool {
    struct Array {
        int32_t width, height, type;
        size_t data_bytes, mask_bytes, slot_bytes;
        CUdeviceptr base;
        std::vector<CUmemGenericAllocationHandle> handle;
        std::vector<uint8_t> used;  // 1: the slot holds a live layer
        std::vector<int32_t> free_slots;
    };
    int device;
    int32_t max_layers;
    size_t granularity;
    std::unordered_map<uint64_t, int32_t> index;  // (width, height, type) -> array
    std::vector<Array> arrays;
    uint64_t committed;
    int64_t live;
    std::mutex mu;
};

namespace lcl {
namespace {

struct Driver {
    CUresult (*reserve)(CUdeviceptr *, size_t, size_t, CUdeviceptr, unsigned long long);
    CUresult (*addr_free)(CUdeviceptr, size_t);
    CUresult (*create)(CUmemGenericAllocationHandle *, size_t, const CUmemAllocationProp *, unsigned long long);
    CUresult (*release)(CUmemGenericAllocationHandle);
    CUresult (*map)(CUdeviceptr, size_t, size_t, CUmemGenericAllocationHandle, unsigned long long);
    CUresult (*unmap)(CUdeviceptr, size_t);
    CUresult (*set_access)(CUdeviceptr, size_t, const CUmemAccessDesc *, size_t);
    CUresult (*granularity)(size_t *, const CUmemAllocationProp *, CUmemAllocationGranularity_flags);
    bool ok;
};

template <typename F>
bool entry(const char *name, F *fn) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion(name, &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !p)
        return false;
    *fn = reinterpret_cast<F>(p);
    return true;
}

const Driver &driver() {
    static Driver d = [] {
        Driver x;
        std::memset(&x, 0, sizeof(x));
        x.ok = entry("cuMemAddressReserve", &x.reserve) && entry("cuMemAddressFree", &x.addr_free) &&
               entry("cuMemCreate", &x.create) && entry("cuMemRelease", &x.release) && entry("cuMemMap", &x.map) &&
               entry("cuMemUnmap", &x.unmap) && entry("cuMemSetAccess", &x.set_access) &&
               entry("cuMemGetAllocationGranularity", &x.granularity);
        return x;
    }();
    return d;
}

lcl_status cu_fail(CUresult r, const char *where) {
    return fail(r == CUDA_ERROR_OUT_OF_MEMORY ? LCL_ERR_OUT_OF_MEMORY : LCL_ERR_CUDA,
                std::string(where) + " failed with CUresult " + std::to_string((int)r));
}

CUmemAllocationProp device_prop(int device) {
    CUmemAllocationProp prop;
    std::memset(&prop, 0, sizeof(prop));
    prop.type = CU_MEM_ALLOCATION_TYPE_PINNED;
    prop.location.type = CU_MEM_LOCATION_TYPE_DEVICE;
    prop.location.id = device;
    return prop;
}

size_t round_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Bytes per texel of a pool layer type: label layers (LCL_U8, LCL_U16) and numeric types.
int type_bytes(int32_t t) {
    switch (t) {
    case LCL_U8: return 1;
    case LCL_U16: return 2;
    case LCL_NUM_U8: case LCL_NUM_I8: return 1;
    case LCL_NUM_U16: case LCL_NUM_I16: case LCL_NUM_F16: return 2;
    case LCL_NUM_U32: case LCL_NUM_I32: case LCL_NUM_F32: return 4;
    default: return 0;
    }
}

bool is_numeric(int32_t t) { return t >= 0x10; }

}  // namespace
}  // namespace lcl

using namespace lcl;

extern "C" {

lcl_status lcl_pool_create(int32_t max_layers_per_array, lcl_pool **out) {
    if (!out) return fail(LCL_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (max_layers_per_array < 1 || max_layers_per_array > (1 << 20))
        return fail(LCL_ERR_INVALID_ARG, "max_layers_per_array must be in [1, 2^20]");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "lcl_pool_create: cudaGetDevice");
    const Driver &d = driver();
    if (!d.ok) return fail(LCL_ERR_CUDA, "lcl_pool_create: the driver's virtual-memory entry points are unavailable");
    const CUmemAllocationProp prop = device_prop(dev);
    size_t gran = 0;
    CUresult r = d.granularity(&gran, &prop, CU_MEM_ALLOC_GRANULARITY_RECOMMENDED);
    if (r != CUDA_SUCCESS || gran == 0) return cu_fail(r, "cuMemGetAllocationGranularity");
    lcl_pool *p = new lcl_pool();
    p->device = dev;
    p->max_layers = max_layers_per_array;
    p->granularity = gran;
    p->committed = 0;
    p->live = 0;
    *out = p;
    return LCL_OK;
}

lcl_status lcl_pool_acquire(lcl_pool *pool, int32_t width, int32_t height, int32_t type, lcl_stream stream,
                            lcl_pool_layer *out) {
    if (!pool || !out) return fail(LCL_ERR_INVALID_ARG, "pool or out is NULL");
    const int tb = type_bytes(type);
    if (!tb) return fail(LCL_ERR_INVALID_ARG, "unknown layer type");
    if (width < 4 || width > 16384 || (width & 3) || height < 1 || height > 16384)
        return fail(LCL_ERR_INVALID_ARG, "layer size: width a multiple of 4 in [4, 16384], height in [1, 16384]");
    const Driver &d = driver();
    std::lock_guard<std::mutex> lock(pool->mu);
    const uint64_t key = ((uint64_t)(uint32_t)type << 32) | ((uint64_t)height << 16) | (uint64_t)width;
    auto it = pool->index.find(key);
    int32_t ai;
    if (it == pool->index.end()) {
        lcl_pool::Array A;
        A.width = width;
        A.height = height;
        A.type = type;
        const size_t n = (size_t)width * height;
        A.data_bytes = round_up(n * tb, 256);
        A.mask_bytes = is_numeric(type) ? round_up((n + 31) / 32 * 4, 16) : 0;
        A.slot_bytes = round_up(A.data_bytes + A.mask_bytes, pool->granularity);
        A.base = 0;
        CUresult r = d.reserve(&A.base, A.slot_bytes * (size_t)pool->max_layers, pool->granularity, 0, 0);
        if (r != CUDA_SUCCESS) return cu_fail(r, "cuMemAddressReserve");
        A.handle.assign((size_t)pool->max_layers, 0);
        A.used.assign((size_t)pool->max_layers, 0);
        for (int32_t s = pool->max_layers - 1; s >= 0; --s) A.free_slots.push_back(s);
        ai = (int32_t)pool->arrays.size();
        pool->arrays.push_back(std::move(A));
        pool->index[key] = ai;
    } else {
        ai = it->second;
    }
    lcl_pool::Array &A = pool->arrays[(size_t)ai];
    if (A.free_slots.empty())
        return fail(LCL_ERR_OUT_OF_MEMORY, "layer array full: every reserved slot of this (width, height, type) is in use");
    const int32_t slot = A.free_slots.back();
    const CUdeviceptr va = A.base + (CUdeviceptr)(A.slot_bytes * (size_t)slot);
    const CUmemAllocationProp prop = device_prop(pool->device);
    CUmemGenericAllocationHandle h = 0;
    CUresult r = d.create(&h, A.slot_bytes, &prop, 0);
    if (r != CUDA_SUCCESS) return cu_fail(r, "cuMemCreate");
    r = d.map(va, A.slot_bytes, 0, h, 0);
    if (r != CUDA_SUCCESS) {
        d.release(h);
        return cu_fail(r, "cuMemMap");
    }
    CUmemAccessDesc acc;
    std::memset(&acc, 0, sizeof(acc));
    acc.location = prop.location;
    acc.flags = CU_MEM_ACCESS_FLAGS_PROT_READWRITE;
    r = d.set_access(va, A.slot_bytes, &acc, 1);
    if (r != CUDA_SUCCESS) {
        d.unmap(va, A.slot_bytes);
        d.release(h);
        return cu_fail(r, "cuMemSetAccess");
    }
    const cudaError_t e = cudaMemsetAsync(reinterpret_cast<void *>(va), 0, A.data_bytes + A.mask_bytes,
                                          reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) {
        d.unmap(va, A.slot_bytes);
        d.release(h);
        return cuda_fail(e, "lcl_pool_acquire: clearing the layer");
    }
    A.free_slots.pop_back();
    A.handle[(size_t)slot] = h;
    A.used[(size_t)slot] = 1;
    pool->committed += A.slot_bytes;
    pool->live += 1;
    std::memset(out, 0, sizeof(*out));
    out->data = reinterpret_cast<void *>(va);
    out->mask = A.mask_bytes ? reinterpret_cast<uint32_t *>(va + A.data_bytes) : nullptr;
    out->handle = ((uint64_t)(uint32_t)ai << 32) | (uint32_t)slot;
    out->width = width;
    out->height = height;
    out->type = type;
    return LCL_OK;
}

lcl_status lcl_pool_release(lcl_pool *pool, uint64_t handle, lcl_stream stream) {
    if (!pool) return fail(LCL_ERR_INVALID_ARG, "pool is NULL");
    const Driver &d = driver();
    std::lock_guard<std::mutex> lock(pool->mu);
    const uint32_t ai = (uint32_t)(handle >> 32), slot = (uint32_t)handle;
    if (ai >= pool->arrays.size() || slot >= (uint32_t)pool->max_layers || !pool->arrays[ai].used[slot])
        return fail(LCL_ERR_INVALID_ARG, "not a live layer of this pool");
    lcl_pool::Array &A = pool->arrays[ai];
    const cudaError_t e = cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "lcl_pool_release: cudaStreamSynchronize");
    const CUdeviceptr va = A.base + (CUdeviceptr)(A.slot_bytes * slot);
    CUresult r = d.unmap(va, A.slot_bytes);
    if (r != CUDA_SUCCESS) return cu_fail(r, "cuMemUnmap");
    r = d.release(A.handle[slot]);
    if (r != CUDA_SUCCESS) return cu_fail(r, "cuMemRelease");
    A.handle[slot] = 0;
    A.used[slot] = 0;
    A.free_slots.push_back((int32_t)slot);
    pool->committed -= A.slot_bytes;
    pool->live -= 1;
    return LCL_OK;
}

lcl_status lcl_pool_stats_get(lcl_pool *pool, lcl_pool_stats *out) {
    if (!pool || !out) return fail(LCL_ERR_INVALID_ARG, "pool or out is NULL");
    std::lock_guard<std::mutex> lock(pool->mu);
    std::memset(out, 0, sizeof(*out));
    for (const auto &A : pool->arrays) out->reserved_bytes += A.slot_bytes * (uint64_t)pool->max_layers;
    out->committed_bytes = pool->committed;
    out->layers = pool->live;
    out->arrays = (int32_t)pool->arrays.size();
    out->granularity = pool->granularity;
    return LCL_OK;
}

lcl_status lcl_pool_destroy(lcl_pool *pool) {
    if (!pool) return LCL_OK;
    const Driver &d = driver();
    lcl_status s = LCL_OK;
    const cudaError_t e = cudaDeviceSynchronize();  // nothing may still use a layer
    if (e != cudaSuccess) s = cuda_fail(e, "lcl_pool_destroy: cudaDeviceSynchronize");
    {
        std::lock_guard<std::mutex> lock(pool->mu);
        for (auto &A : pool->arrays) {
            for (size_t slot = 0; slot < A.handle.size(); ++slot) {
                if (!A.used[slot]) continue;
                const CUdeviceptr va = A.base + (CUdeviceptr)(A.slot_bytes * slot);
                if (d.unmap(va, A.slot_bytes) != CUDA_SUCCESS || d.release(A.handle[slot]) != CUDA_SUCCESS)
                    s = fail(LCL_ERR_CUDA, "lcl_pool_destroy: unmapping a layer failed");
            }
            if (d.addr_free(A.base, A.slot_bytes * (size_t)pool->max_layers) != CUDA_SUCCESS)
                s = fail(LCL_ERR_CUDA, "lcl_pool_destroy: freeing a reserved range failed");
        }
    }
    delete pool;
    return s;
}

}  // extern "C"
