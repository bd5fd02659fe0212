// Device memory of plans, weight computations and feature searches, from one stream-ordered
// memory pool per device that keeps up to kPoolKeepBytes of freed memory reserved: creating and
// destroying plans ping after ping then reuses memory instead of mapping and unmapping it with
// cudaMalloc / cudaFree (tens of microseconds per call).

#include "ftcg_internal.cuh"

#include <cstdlib>
#include <map>
#include <mutex>

namespace ftcg {

namespace {

constexpr uint64_t kPoolKeepBytes = 4ull << 30;
std::mutex g_pool_mu;
std::map<int, cudaMemPool_t> g_pools;

bool pool_disabled() {
    static const bool off = std::getenv("FTCG_NO_POOL") != nullptr;
    return off;
}

}  // namespace

cudaError_t pool_free(void* p, cudaStream_t s) {
    if (!p) return cudaSuccess;
    return pool_disabled() ? cudaFree(p) : cudaFreeAsync(p, s);
}

cudaError_t pool_malloc(void** p, size_t bytes, cudaStream_t s) {
    *p = nullptr;
    if (bytes == 0) return cudaSuccess;
    if (pool_disabled()) return cudaMalloc(p, bytes);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    cudaMemPool_t pool = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_pool_mu);
        auto it = g_pools.find(dev);
        if (it == g_pools.end()) {
            cudaMemPoolProps props = {};
            props.allocType = cudaMemAllocationTypePinned;
            props.location.type = cudaMemLocationTypeDevice;
            props.location.id = dev;
            if ((e = cudaMemPoolCreate(&pool, &props)) != cudaSuccess) return e;
            uint64_t keep = kPoolKeepBytes;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
            g_pools.emplace(dev, pool);
        } else {
            pool = it->second;
        }
    }
    return cudaMallocFromPoolAsync(p, bytes, pool, s);
}

}  // namespace ftcg
