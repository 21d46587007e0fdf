// Device memory for the library's buffers: cudaMalloc behind a small cache of
// freed blocks keyed by (device, exact size).
//
// A problem of a given shape allocates the same set of buffers every time (the
// factors alone are 8 (s/2+1) m_p^2 bytes), and cudaMalloc / cudaFree of
// gigabyte buffers cost milliseconds each, with cudaFree synchronising the
// device.  Repeated create / solve / destroy cycles (the end-to-end use of the
// API) therefore reuse the blocks of the previous problem.  The cache holds at
// most DEVMEM_CACHE_LIMIT bytes (oldest blocks are released first) and is
// emptied for the device when cudaMalloc runs out of memory, and entirely by
// fde_release_cached_memory().
//
// dev_free() callers guarantee that no queued GPU work still uses the block
// (every call site synchronises the problem's streams first); the block may be
// handed to another problem, on another stream, by the next dev_alloc().
#include <deque>
#include <mutex>
#include <unordered_map>

#include "fde_internal.h"

namespace fde {

namespace {

constexpr size_t DEVMEM_CACHE_LIMIT = size_t(16) << 30;

struct Block {
    void* p;
    size_t bytes;
    int dev;
};

std::mutex g_mu;
std::deque<Block> g_cache;                     // freed blocks, oldest first
size_t g_cached = 0;                           // bytes held in g_cache
std::unordered_map<void*, Block> g_live;       // blocks handed out

void release_cached(int dev) {  // g_mu held
    for (auto it = g_cache.begin(); it != g_cache.end();) {
        if (dev < 0 || it->dev == dev) {
            cudaFree(it->p);
            g_cached -= it->bytes;
            it = g_cache.erase(it);
        } else {
            ++it;
        }
    }
}

}  // namespace

int dev_alloc(void** p, size_t bytes) {
    *p = nullptr;
    if (bytes == 0) return FDE_OK;
    int dev = 0;
    FDE_CUDA_TRY(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(g_mu);
    for (auto it = g_cache.begin(); it != g_cache.end(); ++it) {
        if (it->dev == dev && it->bytes == bytes) {
            *p = it->p;
            g_cached -= bytes;
            g_live[*p] = *it;
            g_cache.erase(it);
            return FDE_OK;
        }
    }
    cudaError_t e = cudaMalloc(p, bytes);
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();  // clear, then retry with the cache of this device released
        release_cached(dev);
        e = cudaMalloc(p, bytes);
    }
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return set_error(FDE_ERR_ALLOC, std::string("cudaMalloc failed: ") + cudaGetErrorString(e));
    }
    g_live[*p] = Block{*p, bytes, dev};
    return FDE_OK;
}

void dev_free(void* p) {
    if (!p) return;
    std::lock_guard<std::mutex> lock(g_mu);
    auto it = g_live.find(p);
    if (it == g_live.end()) {  // not from dev_alloc
        cudaFree(p);
        return;
    }
    const Block b = it->second;
    g_live.erase(it);
    if (b.bytes > DEVMEM_CACHE_LIMIT) {
        cudaFree(p);
        return;
    }
    g_cache.push_back(b);
    g_cached += b.bytes;
    while (g_cached > DEVMEM_CACHE_LIMIT && !g_cache.empty()) {
        cudaFree(g_cache.front().p);
        g_cached -= g_cache.front().bytes;
        g_cache.pop_front();
    }
}

int dev_release_cached() {
    std::lock_guard<std::mutex> lock(g_mu);
    cudaError_t first = cudaSuccess;
    for (const Block& b : g_cache) {
        const cudaError_t e = cudaFree(b.p);
        if (e != cudaSuccess && first == cudaSuccess) first = e;
    }
    g_cache.clear();
    g_cached = 0;
    if (first != cudaSuccess) {
        cudaGetLastError();
        return set_error(FDE_ERR_CUDA, std::string("cudaFree failed: ") + cudaGetErrorString(first));
    }
    return FDE_OK;
}

}  // namespace fde
