// da_alloc.cu -- the library's device allocations (contexts, workspaces,
// tensor-core operands, batched launches, requests of the request loop).
//
// Every one goes through dev_malloc / pool_malloc_async, which
//  - keep a count of the live allocations and their bytes, so that a test can
//    check that a failed call leaves nothing behind (da_diag_live_allocations);
//  - can be told to fail on the host, without touching the device, as if the
//    device were out of memory (da_diag_fail_alloc): the next `after`
//    allocations succeed and the `count` after them fail.  This exercises the
//    error paths of allocation failure without exhausting a shared GPU.
#include <atomic>
#include <mutex>
#include <unordered_map>

#include "da.h"
#include "da_internal.h"

namespace {

std::mutex g_mu;
std::unordered_map<void*, size_t> g_live;   // pointer -> bytes
long long g_live_bytes = 0;
long long g_skip = 0, g_fail = 0;            // injected: succeed g_skip more, then fail g_fail
long long g_injected = 0;

// True if this allocation is to fail (consumes the injection budget).
bool injected()
{
    if (g_fail <= 0) return false;
    if (g_skip > 0) {
        --g_skip;
        return false;
    }
    --g_fail;
    ++g_injected;
    return true;
}

void track(void* p, size_t bytes)
{
    g_live.emplace(p, bytes);
    g_live_bytes += (long long)bytes;
}

void untrack(void* p)
{
    auto it = g_live.find(p);
    if (it == g_live.end()) return;
    g_live_bytes -= (long long)it->second;
    g_live.erase(it);
}

}  // namespace

namespace da {

cudaError_t dev_malloc(void** p, size_t bytes)
{
    *p = nullptr;
    std::lock_guard<std::mutex> lk(g_mu);
    if (injected()) return cudaErrorMemoryAllocation;
    const cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        return e;
    }
    track(*p, bytes);
    return cudaSuccess;
}

cudaError_t dev_free(void* p)
{
    if (!p) return cudaSuccess;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        untrack(p);
    }
    return cudaFree(p);
}

cudaError_t pool_malloc_async(void** p, size_t bytes, cudaMemPool_t pool, cudaStream_t st)
{
    *p = nullptr;
    std::lock_guard<std::mutex> lk(g_mu);
    if (injected()) return cudaErrorMemoryAllocation;
    const cudaError_t e = cudaMallocFromPoolAsync(p, bytes, pool, st);
    if (e != cudaSuccess) {
        *p = nullptr;
        return e;
    }
    track(*p, bytes);
    return cudaSuccess;
}

cudaError_t pool_free_async(void* p, cudaStream_t st)
{
    if (!p) return cudaSuccess;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        untrack(p);
    }
    return cudaFreeAsync(p, st);
}

}  // namespace da

extern "C" {

da_status da_diag_fail_alloc(int32_t after, int32_t count)
{
    if (after < 0 || count < 0) {
        da::set_last_error("after and count must be >= 0");
        return DA_EINVAL;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    g_skip = after;
    g_fail = count;
    return DA_OK;
}

da_status da_diag_live_allocations(int64_t* count, int64_t* bytes, int64_t* injected_failures)
{
    std::lock_guard<std::mutex> lk(g_mu);
    if (count) *count = (int64_t)g_live.size();
    if (bytes) *bytes = g_live_bytes;
    if (injected_failures) *injected_failures = g_injected;
    return DA_OK;
}

}  // extern "C"
