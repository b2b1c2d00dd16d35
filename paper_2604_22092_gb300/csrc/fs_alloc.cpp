// fs_alloc.cpp -- device memory of the library (graphs, simulations,
// ensembles, batches and their scratch).
//
// Every allocation goes through fs::dmalloc / fs::dfree. By default freed
// blocks are kept in a per-device cache of exact (rounded) sizes and handed
// out again, so that creating and destroying graphs and simulations in a loop
// does not pay for cudaMalloc's mapping and cudaFree's unmapping each time.
// A block enters the cache only after a device-wide synchronisation (the same
// guarantee cudaFree gives: no launched work can still use it). When the
// device runs out of memory the cache is released and the allocation retried.
// A caller may instead install its own allocator (fs_set_allocator); the
// library then caches nothing.
#include <cuda_runtime.h>

#include <cstdint>
#include <map>
#include <mutex>
#include <vector>

#include "fs.h"
#include "fs_objects.h"

namespace fs {

namespace {

constexpr int kMaxDevices = 64;
constexpr size_t kSmallGrain = 512;                  // rounding below 1 MiB
constexpr size_t kLargeGrain = 2u << 20;             // rounding from 1 MiB on
constexpr size_t kCacheCap = (size_t)64 << 30;       // bytes kept per device at most

struct DeviceCache {
    std::map<size_t, std::vector<void*>> free_blocks;   // rounded size -> blocks
    std::map<void*, size_t> live;                       // block -> rounded size
    size_t cached = 0;
};

std::mutex g_mu;
DeviceCache g_cache[kMaxDevices];
fs_alloc_fn g_user_alloc = nullptr;
fs_free_fn g_user_free = nullptr;
void* g_user_ctx = nullptr;
// blocks from a caller's allocator, with the functions that must free them
std::map<void*, std::pair<fs_free_fn, void*>> g_user_live;

size_t round_size(size_t b)
{
    if (b == 0)
        b = 1;
    const size_t g = b < ((size_t)1 << 20) ? kSmallGrain : kLargeGrain;
    return (b + g - 1) / g * g;
}

int current_device()
{
    int d = 0;
    if (cudaGetDevice(&d) != cudaSuccess || d < 0 || d >= kMaxDevices)
        return -1;
    return d;
}

void release_locked(DeviceCache& c)
{
    for (auto& kv : c.free_blocks)
        for (void* p : kv.second)
            cudaFree(p);
    c.free_blocks.clear();
    c.cached = 0;
}

}  // namespace

cudaError_t dmalloc_raw(void** p, size_t bytes)
{
    *p = nullptr;
    std::unique_lock<std::mutex> lock(g_mu);
    if (g_user_alloc) {
        fs_alloc_fn fn = g_user_alloc;
        fs_free_fn ffn = g_user_free;
        void* ctx = g_user_ctx;
        lock.unlock();
        void* q = fn(bytes ? bytes : 1, ctx);
        if (!q)
            return cudaErrorMemoryAllocation;
        lock.lock();
        g_user_live[q] = {ffn, ctx};
        *p = q;
        return cudaSuccess;
    }
    const int d = current_device();
    if (d < 0) {
        lock.unlock();
        return cudaMalloc(p, bytes ? bytes : 1);
    }
    DeviceCache& c = g_cache[d];
    const size_t r = round_size(bytes);
    auto it = c.free_blocks.find(r);
    if (it != c.free_blocks.end() && !it->second.empty()) {
        *p = it->second.back();
        it->second.pop_back();
        c.cached -= r;
        c.live[*p] = r;
        return cudaSuccess;
    }
    cudaError_t e = cudaMalloc(p, r);
    if (e == cudaErrorMemoryAllocation && c.cached) {
        (void)cudaGetLastError();
        release_locked(c);
        e = cudaMalloc(p, r);
    }
    if (e == cudaSuccess)
        c.live[*p] = r;
    return e;
}

cudaError_t dfree(void* p)
{
    if (!p)
        return cudaSuccess;
    std::unique_lock<std::mutex> lock(g_mu);
    const int d = current_device();
    if (d >= 0) {
        DeviceCache& c = g_cache[d];
        auto it = c.live.find(p);
        if (it != c.live.end()) {
            const size_t r = it->second;
            c.live.erase(it);
            lock.unlock();
            // no work launched before this point may still use the block
            // when it is handed out again
            const cudaError_t e = cudaDeviceSynchronize();
            lock.lock();
            if (e == cudaSuccess && c.cached + r <= kCacheCap) {
                c.free_blocks[r].push_back(p);
                c.cached += r;
                return cudaSuccess;
            }
            lock.unlock();
            return cudaFree(p);
        }
    }
    auto u = g_user_live.find(p);
    if (u != g_user_live.end()) {
        const fs_free_fn fn = u->second.first;
        void* ctx = u->second.second;
        g_user_live.erase(u);
        lock.unlock();
        cudaDeviceSynchronize();
        fn(p, ctx);
        return cudaSuccess;
    }
    lock.unlock();
    return cudaFree(p);
}

}  // namespace fs

extern "C" {

fs_status fs_set_allocator(fs_alloc_fn alloc, fs_free_fn free_fn, void* ctx)
{
    fsapi::g_err.clear();
    if ((alloc == nullptr) != (free_fn == nullptr))
        return fsapi::fail(FS_EINVAL, "fs_set_allocator: give both functions or neither");
    std::lock_guard<std::mutex> lock(fs::g_mu);
    fs::g_user_alloc = alloc;
    fs::g_user_free = free_fn;
    fs::g_user_ctx = ctx;
    return FS_OK;
}

fs_status fs_release_cached_memory(void)
{
    fsapi::g_err.clear();
    cudaDeviceSynchronize();
    std::lock_guard<std::mutex> lock(fs::g_mu);
    const int d = fs::current_device();
    if (d >= 0)
        fs::release_locked(fs::g_cache[d]);
    return FS_OK;
}

fs_status fs_cached_memory(uint64_t* cached_bytes, uint64_t* live_blocks)
{
    if (!cached_bytes || !live_blocks)
        return fsapi::fail(FS_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lock(fs::g_mu);
    const int d = fs::current_device();
    *cached_bytes = d >= 0 ? fs::g_cache[d].cached : 0;
    *live_blocks = d >= 0 ? fs::g_cache[d].live.size() : 0;
    return FS_OK;
}

}  // extern "C"
