// da_static.cu -- an anneal entry point that allocates no memory.
//
// Some callers cannot allocate device memory when they want to run an anneal:
// a service that reserves all of the GPU's memory up front and forbids any
// later allocation, code running inside another framework's allocator-free
// region, or a program about to capture its work into a CUDA graph.  For them
// da_anneal_static runs the integer (DA_INT8) anneal with every intermediate
// buffer placed in one file-scope device array of fixed size; the caller
// passes the instance, the schedule and the result buffers in device memory.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdint>
#include <mutex>
#include <string>

#include "da.h"
#include "da_internal.h"

namespace {

constexpr size_t kStaticBytes = 16u << 20;  // 16 MiB, held by every device that loads the library
__device__ __align__(256) unsigned char g_static_scratch[kStaticBytes];

constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
// The array's device address per device, with the CUDA context it was looked
// up in: a context that is destroyed and created again (cudaDeviceReset) loads
// the module again, possibly at another address.
void* g_static_ptr[kMaxDevices] = {};
void* g_static_ctx[kMaxDevices] = {};

// The calling thread's current CUDA context (driver handle), through the
// runtime's driver entry point so that the library needs no link to libcuda;
// nullptr if it cannot be had.
void* current_context()
{
    using GetCurrent = int (*)(void**);
    static GetCurrent fn = [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            f = nullptr;
        }
        return reinterpret_cast<GetCurrent>(f);
    }();
    void* ctx = nullptr;
    if (!fn || fn(&ctx) != 0) return nullptr;
    return ctx;
}

da_status fail(da_status s, const char* why)
{
    da::set_last_error(why);
    return s;
}

bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

size_t align256(size_t v) { return (v + 255) / 256 * 256; }

__global__ void static_finalize_kernel(int R, const da::ReplicaScalars* sc, const long long* eex, double* final_E,
                                       double* best_E, double* drift, int64_t* flips)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    if (final_E) final_E[r] = (double)eex[r];
    if (best_E) best_E[r] = (double)eex[R + r];
    if (drift) drift[r] = fabs((double)sc[r].E - (double)eex[r]);
    if (flips) flips[r] = sc[r].flips;
}

}  // namespace

extern "C" int64_t da_static_pitch(int64_t N)
{
    if (N < 1 || N > 1024) return 0;
    int64_t V = 4;
    while (32 * V < N) V *= 2;
    return 32 * V;
}

extern "C" da_status da_anneal_static(const int8_t* W, const int32_t* diag, int64_t N, int64_t ldw,
                                      const float* beta, int64_t steps, float offset_inc, int32_t replicas,
                                      uint64_t seed, const da_dev_result* out, void* stream)
{
    da::set_last_error("");
    if (!W || !diag || N < 1 || N > 1024) return fail(DA_EINVAL, "need W, diag and 1 <= N <= 1024");
    const int64_t pitch = da_static_pitch(N);
    if (ldw < pitch || ldw % 16 != 0 || ldw > INT_MAX)
        return fail(DA_EINVAL, "ldw must be a multiple of 16, at least da_static_pitch(N) and at most INT_MAX");
    // the step kernel reads a lane's slice of a row of W with 16-byte loads
    // and diag as 4-byte words: a misaligned pointer would fault the device
    if (!aligned(W, 16)) return fail(DA_EINVAL, "W must be 16-byte aligned");
    if (!aligned(diag, 4) || (beta && !aligned(beta, 4))) return fail(DA_EINVAL, "diag and beta must be 4-byte aligned");
    if (out && (!aligned(out->final_E, 8) || !aligned(out->best_E, 8) || !aligned(out->max_drift, 8) ||
                !aligned(out->flips, 8) || !aligned(out->final_x, 4) || !aligned(out->best_x, 4) ||
                !aligned(out->trace, 4)))
        return fail(DA_EINVAL, "result arrays must be aligned to their element size");
    if (replicas < 1 || steps < 0 || steps >= (1ll << 32) || (steps > 0 && !beta))
        return fail(DA_EINVAL, "need replicas >= 1, 0 <= steps < 2^32 and a schedule");
    if (!(offset_inc >= 0.f) || !std::isfinite(offset_inc)) return fail(DA_EINVAL, "offset_inc must be finite and >= 0");

    da::StepShape s;
    s.V = (int)(pitch / 32);
    s.G = 1;
    s.rpb = 4;
    const int R = replicas;
    const int n = (int)N;
    const size_t tiles = ((size_t)s.npad() + 63) / 64;
    const size_t o_h = 0;
    const size_t o_x = o_h + align256((size_t)R * s.npad() * 4);
    const size_t o_sc = o_x + align256((size_t)2 * R * s.nwords() * 4);
    const size_t o_part = o_sc + align256((size_t)R * sizeof(da::ReplicaScalars));
    const size_t o_eex = o_part + align256(tiles * 16 * 2 * (size_t)R);
    const size_t total = o_eex + align256((size_t)2 * R * 8);
    if (total > kStaticBytes)
        return fail(DA_EINVAL, ("the replica state needs " + std::to_string(total) +
                                " bytes, more than the fixed 16 MiB array").c_str());

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return fail(DA_ECUDA, "no usable CUDA device");
    }
    char* base = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_static_mu);
        void* ctx = current_context();
        if (!g_static_ptr[dev] || ctx != g_static_ctx[dev]) {
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p) {
                cudaGetLastError();
                return fail(DA_ECUDA, "cudaGetSymbolAddress of the scratch array failed");
            }
            g_static_ptr[dev] = p;
            g_static_ctx[dev] = ctx;
        }
        base = static_cast<char*>(g_static_ptr[dev]);
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    void* h = base + o_h;
    uint32_t* x = reinterpret_cast<uint32_t*>(base + o_x);
    da::ReplicaScalars* sc = reinterpret_cast<da::ReplicaScalars*>(base + o_sc);
    long long* part = reinterpret_cast<long long*>(base + o_part);
    long long* eex = reinterpret_cast<long long*>(base + o_eex);

    // the array keeps the previous call's contents: start from x = 0, g = diag
    if (da::launch_init_state(true, diag, n, R, h, s.npad(), st) != cudaSuccess) return DA_ECUDA;
    if (cudaMemsetAsync(x, 0, (size_t)2 * R * s.nwords() * 4, st) != cudaSuccess) return DA_ECUDA;
    if (cudaMemsetAsync(sc, 0, (size_t)R * sizeof(da::ReplicaScalars), st) != cudaSuccess) return DA_ECUDA;

    da::StepParams p;
    p.W = W;
    p.diag = diag;
    p.N = n;
    p.ldw = (int)ldw;
    p.R = R;
    p.npad = s.npad();
    p.nw = s.nwords();
    p.h = h;
    p.x = x;
    p.bestx = x + (size_t)R * s.nwords();
    p.sc = sc;
    p.beta = beta;
    p.inc = offset_inc;
    da::set_seed(p, seed);
    if (out && out->trace) {
        p.trace = out->trace;
        p.trace_T = steps;
    }
    for (long long t0 = 0; t0 < steps; t0 = p.t1) {
        p.t0 = t0;
        p.t1 = std::min<long long>(steps, t0 + (1ll << 14));
        if (da::launch_step(da::kWInt8, s, p, out && out->trace, st) != cudaSuccess) return DA_ECUDA;
    }
    if (da::launch_best_fixup(R, sc, true, x, p.bestx, s.nwords(), st) != cudaSuccess) return DA_ECUDA;
    if (da::launch_recompute(true, W, diag, n, (int)ldw, 0, x, s.nwords(), 2 * R, nullptr, s.npad(), eex, 1, st,
                             part) != cudaSuccess)
        return DA_ECUDA;
    if (!out) return DA_OK;
    static_finalize_kernel<<<(R + 127) / 128, 128, 0, st>>>(R, sc, eex, out->final_E, out->best_E, out->max_drift,
                                                            out->flips);
    if (cudaGetLastError() != cudaSuccess) return DA_ECUDA;
    const size_t words = (size_t)((N + 31) / 32);
    if (out->final_x &&
        cudaMemcpy2DAsync(out->final_x, words * 4, x, (size_t)s.nwords() * 4, words * 4, R, cudaMemcpyDeviceToDevice,
                          st) != cudaSuccess)
        return DA_ECUDA;
    if (out->best_x &&
        cudaMemcpy2DAsync(out->best_x, words * 4, p.bestx, (size_t)s.nwords() * 4, words * 4, R,
                          cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return DA_ECUDA;
    return DA_OK;
}
