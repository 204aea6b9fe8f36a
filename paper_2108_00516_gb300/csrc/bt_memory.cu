// bt_memory.cu -- process-wide cache of idle device blocks behind the
// per-graph pools (bthost::DevPool).
//
// A graph hands every block of its pool over when it is destroyed (after its
// stream has been synchronised, so the blocks are idle) and a graph that
// needs a block takes one of the same size class before it allocates: a
// series of graphs -- a tracker restarted per session, a test suite, the
// end-to-end benchmark -- reuses device memory instead of paying cudaMalloc
// for every new frame and cudaFree (which synchronises the whole device) for
// every destroyed graph.  Size classes are those of DevPool (multiples of
// 256 B up to 64 KiB, of 64 KiB above); the small classes are carved from
// 2 MiB slabs.  bt_device_cache_trim frees the idle large blocks.
#include "bt_host.h"

#include <cuda_runtime.h>

#include <atomic>
#include <map>
#include <mutex>
#include <utility>
#include <vector>

namespace {

constexpr size_t kSmallMax = 65536;          // classes carved from slabs
constexpr size_t kSlabBytes = 2u << 20;

struct DeviceCache {
    std::mutex mu;
    // (device, class) -> idle blocks
    std::map<std::pair<int, size_t>, std::vector<void*>> idle;
    // device -> (current slab, bytes used)
    std::map<int, std::pair<char*, size_t>> slab;
    std::vector<void*> slabs;                 // never freed before exit
    int64_t idle_bytes = 0;
};

DeviceCache& cache()
{
    static DeviceCache* c = new DeviceCache();   // outlives every graph
    return *c;
}

}  // namespace

cudaError_t bthost::cache_take(size_t cls, void** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    DeviceCache& c = cache();
    std::lock_guard<std::mutex> lock(c.mu);
    auto it = c.idle.find(std::make_pair(dev, cls));
    if (it != c.idle.end() && !it->second.empty()) {
        *out = it->second.back();
        it->second.pop_back();
        c.idle_bytes -= (int64_t)cls;
        return cudaSuccess;
    }
    if (cls > kSmallMax) return alloc_should_fail() ? cudaErrorMemoryAllocation : cudaMalloc(out, cls);
    auto& s = c.slab[dev];
    if (!s.first || s.second + cls > kSlabBytes) {
        void* p = nullptr;
        if (alloc_should_fail()) return cudaErrorMemoryAllocation;
        e = cudaMalloc(&p, kSlabBytes);
        if (e != cudaSuccess) return e;
        c.slabs.push_back(p);
        s = std::make_pair(static_cast<char*>(p), size_t(0));
    }
    *out = s.first + s.second;
    s.second += cls;
    return cudaSuccess;
}

void bthost::cache_give(int device, size_t cls, void* p)
{
    if (!p) return;
    DeviceCache& c = cache();
    std::lock_guard<std::mutex> lock(c.mu);
    c.idle[std::make_pair(device, cls)].push_back(p);
    c.idle_bytes += (int64_t)cls;
}

extern "C" {

int64_t bt_device_cache_bytes(void)
{
    DeviceCache& c = cache();
    std::lock_guard<std::mutex> lock(c.mu);
    return c.idle_bytes;
}

int64_t bt_device_cache_trim(void)
{
    DeviceCache& c = cache();
    std::lock_guard<std::mutex> lock(c.mu);
    int64_t freed = 0;
    int cur = 0;
    cudaGetDevice(&cur);
    for (auto& kv : c.idle) {
        if (kv.first.second <= kSmallMax) continue;
        if (!kv.second.empty()) cudaSetDevice(kv.first.first);
        for (void* p : kv.second) {
            cudaFree(p);
            freed += (int64_t)kv.first.second;
        }
        kv.second.clear();
    }
    cudaSetDevice(cur);
    c.idle_bytes -= freed;
    return freed;
}

}  // extern "C"

namespace {
std::atomic<int> g_fail_allocs{0};
}

bool bthost::alloc_should_fail()
{
    int n = g_fail_allocs.load(std::memory_order_relaxed);
    while (n > 0) {
        if (g_fail_allocs.compare_exchange_weak(n, n - 1, std::memory_order_relaxed)) return true;
    }
    return false;
}

extern "C" int32_t bt_debug_fail_allocations(int32_t n)
{
    return g_fail_allocs.exchange(n > 0 ? n : 0);
}
