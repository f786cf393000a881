// Caching allocator of the library's device and pinned host memory.
//
// A setup allocates some sixty device buffers (patch matrices, inverses,
// sketches, tile tables, the Krylov workspace, the SELL copy of A) and a
// destroy frees them; through the driver each call costs tens of
// microseconds and a free synchronises the device.  Here a freed block goes
// to a per-device cache instead, and a later allocation of a similar size
// takes it back:
//   * a block freed since the last device synchronisation is "pending": it
//     is handed out again only after one cudaDeviceSynchronize (which then
//     clears every pending block), so no kernel still in flight can see its
//     memory reused -- the guarantee the code had from cudaFree's implicit
//     synchronisation;
//   * best fit among cached blocks of 1x to 1.25x the rounded request;
//   * the cache holds at most CACHE_CAP bytes; beyond that a freed block
//     goes back to the driver;
//   * when the driver reports out-of-memory, every cached block is released
//     and the allocation is retried once;
//   * a pointer freed twice is ignored; a pointer the cache never handed out
//     goes to cudaFree unchanged.
// psr_release_cached_memory() returns all cached blocks to the driver.
#include "psr_internal.cuh"

#include <atomic>
#include <map>
#include <mutex>
#include <unordered_map>
#include <unordered_set>

namespace psr {
namespace {

constexpr size_t ROUND = 512;                       // bytes
constexpr size_t CACHE_CAP = size_t(16) << 30;      // cached bytes per kind and device

struct Pool {
    std::multimap<size_t, void*> clean;    // size -> block, reusable now
    std::multimap<size_t, void*> pending;  // freed since the last device synchronisation
    std::unordered_map<void*, size_t> live;    // handed out: block -> size
    std::unordered_set<void*> cached;          // in clean or pending
    size_t cached_bytes = 0;
};

struct Cache {
    std::mutex mu;
    std::map<int, Pool> dev;    // device id -> pool
    std::map<int, Pool> host;   // pinned host blocks, by the device current at allocation
};

Cache& cache() {
    static Cache* c = new Cache();   // never destroyed: frees may run during process exit
    return *c;
}

size_t round_up(size_t n) { return ((n ? n : 1) + ROUND - 1) / ROUND * ROUND; }

bool take(std::multimap<size_t, void*>& m, size_t n, void** p, size_t* got) {
    auto it = m.lower_bound(n);
    if (it == m.end() || it->first > n + n / 4) return false;
    *p = it->second;
    *got = it->first;
    m.erase(it);
    return true;
}

void release_all(Pool& P, bool host) {
    for (auto* m : {&P.clean, &P.pending}) {
        for (auto& kv : *m) {
            if (host) cudaFreeHost(kv.second);
            else cudaFree(kv.second);
        }
        m->clear();
    }
    P.cached.clear();
    P.cached_bytes = 0;
}

// Injected failure (psr_debug_inject): the countdown's last device
// allocation fails as if the device were out of memory.
std::atomic<long long> g_fail_countdown{0};

// The open AllocScope of this thread (null: none, or paused).
thread_local std::unordered_map<void*, bool>* t_scope = nullptr;

cudaError_t alloc_impl(void** p, size_t bytes, bool host) {
    *p = nullptr;
    if (!host && g_fail_countdown.load(std::memory_order_relaxed) > 0 &&
        g_fail_countdown.fetch_sub(1, std::memory_order_relaxed) == 1)
        return cudaErrorMemoryAllocation;
    int d = 0;
    cudaGetDevice(&d);
    const size_t n = round_up(bytes);
    Cache& C = cache();
    std::lock_guard<std::mutex> lk(C.mu);
    Pool& P = host ? C.host[d] : C.dev[d];
    size_t got = 0;
    bool hit = take(P.clean, n, p, &got);
    if (!hit && !P.pending.empty()) {
        auto it = P.pending.lower_bound(n);
        if (it != P.pending.end() && it->first <= n + n / 4) {
            cudaError_t e = cudaDeviceSynchronize();
            if (e != cudaSuccess) return e;
            P.clean.insert(P.pending.begin(), P.pending.end());
            P.pending.clear();
            hit = take(P.clean, n, p, &got);
        }
    }
    if (hit) {
        P.cached.erase(*p);
        P.cached_bytes -= got;
        P.live[*p] = got;
        if (t_scope) (*t_scope)[*p] = host;
        return cudaSuccess;
    }
    cudaError_t e = host ? cudaMallocHost(p, n) : cudaMalloc(p, n);
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        cudaDeviceSynchronize();
        release_all(P, host);
        e = host ? cudaMallocHost(p, n) : cudaMalloc(p, n);
    }
    if (e != cudaSuccess) { *p = nullptr; return e; }
    P.live[*p] = n;
    if (t_scope) (*t_scope)[*p] = host;
    return cudaSuccess;
}

cudaError_t free_impl(void* p, bool host) {
    if (!p) return cudaSuccess;
    if (t_scope) t_scope->erase(p);
    Cache& C = cache();
    std::lock_guard<std::mutex> lk(C.mu);
    auto& pools = host ? C.host : C.dev;
    for (auto& kv : pools) {
        Pool& P = kv.second;
        auto it = P.live.find(p);
        if (it != P.live.end()) {
            const size_t n = it->second;
            P.live.erase(it);
            if (P.cached_bytes + n > CACHE_CAP) {
                // over the cap: back to the driver (its free synchronises)
                int cur = 0;
                cudaGetDevice(&cur);
                if (cur != kv.first) cudaSetDevice(kv.first);
                cudaError_t e = host ? cudaFreeHost(p) : cudaFree(p);
                if (cur != kv.first) cudaSetDevice(cur);
                return e;
            }
            P.pending.emplace(n, p);
            P.cached.insert(p);
            P.cached_bytes += n;
            return cudaSuccess;
        }
        if (P.cached.count(p)) return cudaSuccess;   // freed twice
    }
    return host ? cudaFreeHost(p) : cudaFree(p);
}

}  // namespace

void inject_alloc_fail(long long k) { g_fail_countdown.store(k, std::memory_order_relaxed); }

AllocScope::AllocScope() : prev_(t_scope) { t_scope = &held_; }

AllocScope::~AllocScope() {
    t_scope = prev_;
    if (committed_) {
        if (prev_)
            for (auto& kv : held_) (*prev_)[kv.first] = kv.second;
        return;
    }
    std::unordered_map<void*, bool> left;
    left.swap(held_);
    for (auto& kv : left) free_impl(kv.first, kv.second);
}

AllocPause::AllocPause() : prev_(t_scope) { t_scope = nullptr; }
AllocPause::~AllocPause() { t_scope = prev_; }

cudaError_t dev_alloc(void** p, size_t bytes) { return alloc_impl(p, bytes, false); }
cudaError_t dev_free(void* p) { return free_impl(p, false); }
cudaError_t host_alloc(void** p, size_t bytes) { return alloc_impl(p, bytes, true); }
cudaError_t host_free(void* p) { return free_impl(p, true); }

}  // namespace psr

extern "C" int psr_memory_in_use(int64_t* device_bytes, int64_t* host_bytes) {
    using namespace psr;
    Cache& C = cache();
    std::lock_guard<std::mutex> lk(C.mu);
    int64_t d = 0, h = 0;
    for (auto& kv : C.dev)
        for (auto& b : kv.second.live) d += (int64_t)b.second;
    for (auto& kv : C.host)
        for (auto& b : kv.second.live) h += (int64_t)b.second;
    if (device_bytes) *device_bytes = d;
    if (host_bytes) *host_bytes = h;
    return PSR_OK;
}

extern "C" int psr_release_cached_memory(void) {
    using namespace psr;
    Cache& C = cache();
    std::lock_guard<std::mutex> lk(C.mu);
    int cur = 0;
    cudaGetDevice(&cur);
    for (auto* pools : {&C.dev, &C.host}) {
        for (auto& kv : *pools) {
            cudaSetDevice(kv.first);
            cudaDeviceSynchronize();
            release_all(kv.second, pools == &C.host);
        }
    }
    cudaSetDevice(cur);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? PSR_OK : PSR_ERR_CUDA;
}
