// da_diag.cu -- diagnostic entry points that run the device's own Philox and
// exponential (the exact functions every annealer kernel uses) on host
// arrays, so that tests can compare them with independent implementations.
#include <algorithm>
#include <string>
#include <vector>

#include "da.h"
#include "da_device.cuh"
#include "da_fixed.cuh"
#include "da_step_common.cuh"
#include "da_tc.cuh"

namespace {

__global__ void expf_kernel(const float* x, float* y, long long n)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) y[i] = da::exp_neg(x[i]);
}

__global__ void philox_kernel(const uint32_t* in, uint32_t* out, long long n)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t* c = in + 6 * i;
    const da::u32x4 r = da::philox4x32_10(c[0], c[1], c[2], c[3], c[4], c[5]);
    out[4 * i + 0] = r.x;
    out[4 * i + 1] = r.y;
    out[4 * i + 2] = r.z;
    out[4 * i + 3] = r.w;
}

// The bounded mbarrier wait of the pipelined kernels: one barrier that receives
// its arrival (the wait succeeds) and one that never does (the wait must give
// up after `ns` nanoseconds instead of hanging).  out = {arrived wait result,
// abandoned wait result, ns spent in the abandoned wait}.
__global__ void wait_probe_kernel(unsigned long long ns, unsigned long long* out)
{
    __shared__ uint64_t bars[2];
    if (threadIdx.x != 0) return;
    da::tc::mbar_init(&bars[0], 1);
    da::tc::mbar_init(&bars[1], 1);
    da::tc::mbar_arrive(&bars[0]);
    out[0] = da::tc::mbar_wait(&bars[0], 0, 1u << 20, ns) ? 1ull : 0ull;
    const uint64_t t0 = da::tc::global_ns();
    out[1] = da::tc::mbar_wait(&bars[1], 0, 0xffffffffu, ns) ? 1ull : 0ull;
    out[2] = da::tc::global_ns() - t0;
}

__global__ void log_uniform_kernel(const uint32_t* w, float* L, long long n)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) L[i] = da::lg2_draw(w[i]);
}

// The step kernels' decision for one trial, made by their own decide_log (the
// trial as both of a pair, x = 0, E_off = +0, so that Delta E = delta) and, when
// it reports the band, by the exact test decide_exact applies: bit 0 the
// decision, bit 1 set when it came from the exact test.
__global__ void accept_log_kernel(const float* delta, const float* beta, const uint32_t* w, uint8_t* out, long long n)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float c = __fmul_rn(beta[i], da::kLog2e);
    const float lg = da::lg2_draw(w[i]);
    const float h[2] = {delta[i], delta[i]};
    const float L[2] = {lg, lg};
    bool band;
    const uint32_t m = da::step_detail::decide_log<da::step_detail::Arith<float>, 2>(h, 0u, 0.0f, c, L, band);
    bool acc = (m & 1u) != 0;
    if (band) acc = delta[i] <= 0.0f || da::uniform01(w[i]) < da::exp_neg(-__fmul_rn(beta[i], delta[i]));
    out[i] = (uint8_t)((acc ? 1 : 0) | (band ? 2 : 0));
}

// The recompute's fixed-point conversions in integer arithmetic, beside the
// same conversions written with the 64-bit conversion instructions.
__global__ void fixed_kernel(const float* w, const int32_t* S, long long* got, long long* ref, long long n)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    got[i] = da::fixed_of_f32(w[i], S[i]);
    ref[i] = __float2ll_rn(ldexpf(w[i], S[i]));
}

__global__ void scaled_kernel(const long long* v, const int32_t* S, float* got, float* ref, long long n)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    got[i] = da::scaled_f32_of(v[i], S[i]);
    ref[i] = ldexpf(__ll2float_rn(v[i]), -S[i]);
}

// Read bandwidth of a device buffer: a grid-stride loop of 16-byte loads that
// bypass L1 (ld.global.cg), four independent loads in flight per thread, the
// whole buffer `passes` times.  A buffer that fits L2 is served from L2 after
// the first pass, so the kernel measures the L2 read bandwidth the step
// kernel's rows come from; a larger one measures HBM.  The xor of the words
// is stored only when it equals an arbitrary constant (so that no load can be
// dropped).
__device__ __forceinline__ uint4 ld_cg(const uint4* p)
{
    uint4 v;
    asm volatile("ld.global.cg.v4.u32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p));
    return v;
}

__global__ void read_bw_kernel(const uint4* __restrict__ p, long long n16, int passes, unsigned* sink)
{
    uint32_t acc = 0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long t0 = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    for (int k = 0; k < passes; ++k) {
        long long i = t0;
        for (; i + 3 * stride < n16; i += 4 * stride) {
            const uint4 a = ld_cg(p + i), b = ld_cg(p + i + stride), c = ld_cg(p + i + 2 * stride),
                        d = ld_cg(p + i + 3 * stride);
            acc ^= a.x ^ a.y ^ a.z ^ a.w ^ b.x ^ b.y ^ b.z ^ b.w ^ c.x ^ c.y ^ c.z ^ c.w ^ d.x ^ d.y ^ d.z ^ d.w;
        }
        for (; i < n16; i += stride) {
            const uint4 a = ld_cg(p + i);
            acc ^= a.x ^ a.y ^ a.z ^ a.w;
        }
    }
    if (acc == 0x9E3779B9u) sink[0] = acc;
}

thread_local std::string g_diag_err;

template <typename Fn>
da_status run(size_t in_bytes, size_t out_bytes, const void* in_h, void* out_h, Fn launch)
{
    void *din = nullptr, *dout = nullptr;
    cudaError_t e = cudaMalloc(&din, in_bytes ? in_bytes : 1);
    if (e == cudaSuccess) e = cudaMalloc(&dout, out_bytes ? out_bytes : 1);
    if (e == cudaSuccess) e = cudaMemcpy(din, in_h, in_bytes, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        launch(din, dout);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(out_h, dout, out_bytes, cudaMemcpyDeviceToHost);
    if (din) cudaFree(din);
    if (dout) cudaFree(dout);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return DA_ECUDA;
    }
    return DA_OK;
}

}  // namespace

extern "C" da_status da_diag_expf(const float* x, float* y, int64_t n)
{
    if (n < 0 || (n > 0 && (!x || !y))) return DA_EINVAL;
    if (n == 0) return DA_OK;
    return run((size_t)n * 4, (size_t)n * 4, x, y, [&](void* a, void* b) {
        expf_kernel<<<(unsigned)((n + 255) / 256), 256>>>(static_cast<const float*>(a), static_cast<float*>(b), n);
    });
}

extern "C" da_status da_diag_philox(const uint32_t* ctr_key, uint32_t* out, int64_t n)
{
    if (n < 0 || (n > 0 && (!ctr_key || !out))) return DA_EINVAL;
    if (n == 0) return DA_OK;
    return run((size_t)n * 24, (size_t)n * 16, ctr_key, out, [&](void* a, void* b) {
        philox_kernel<<<(unsigned)((n + 255) / 256), 256>>>(static_cast<const uint32_t*>(a), static_cast<uint32_t*>(b), n);
    });
}

extern "C" da_status da_diag_fixed(const float* w, const int32_t* S, int64_t* got, int64_t* ref, int64_t n)
{
    if (n < 0 || (n > 0 && (!w || !S || !got || !ref))) return DA_EINVAL;
    if (n == 0) return DA_OK;
    std::vector<char> in((size_t)n * 8);
    std::copy((const char*)w, (const char*)w + n * 4, in.begin());
    std::copy((const char*)S, (const char*)S + n * 4, in.begin() + n * 4);
    std::vector<long long> out((size_t)n * 2);
    da_status s = run((size_t)n * 8, (size_t)n * 16, in.data(), out.data(), [&](void* a, void* b) {
        const float* wa = static_cast<const float*>(a);
        long long* o = static_cast<long long*>(b);
        fixed_kernel<<<(unsigned)((n + 255) / 256), 256>>>(wa, reinterpret_cast<const int32_t*>(wa + n), o, o + n, n);
    });
    if (s != DA_OK) return s;
    std::copy(out.begin(), out.begin() + n, got);
    std::copy(out.begin() + n, out.end(), ref);
    return DA_OK;
}

extern "C" da_status da_diag_scaled(const int64_t* v, const int32_t* S, float* got, float* ref, int64_t n)
{
    if (n < 0 || (n > 0 && (!v || !S || !got || !ref))) return DA_EINVAL;
    if (n == 0) return DA_OK;
    std::vector<char> in((size_t)n * 12);
    std::copy((const char*)v, (const char*)v + n * 8, in.begin());
    std::copy((const char*)S, (const char*)S + n * 4, in.begin() + n * 8);
    std::vector<float> out((size_t)n * 2);
    da_status s = run((size_t)n * 12, (size_t)n * 8, in.data(), out.data(), [&](void* a, void* b) {
        const long long* va = static_cast<const long long*>(a);
        float* o = static_cast<float*>(b);
        scaled_kernel<<<(unsigned)((n + 255) / 256), 256>>>(va, reinterpret_cast<const int32_t*>(va + n), o, o + n, n);
    });
    if (s != DA_OK) return s;
    std::copy(out.begin(), out.begin() + n, got);
    std::copy(out.begin() + n, out.end(), ref);
    return DA_OK;
}

extern "C" da_status da_diag_log_uniform(const uint32_t* w, float* L, int64_t n)
{
    if (n < 0 || (n > 0 && (!w || !L))) return DA_EINVAL;
    if (n == 0) return DA_OK;
    return run((size_t)n * 4, (size_t)n * 4, w, L, [&](void* a, void* b) {
        log_uniform_kernel<<<(unsigned)((n + 255) / 256), 256>>>(static_cast<const uint32_t*>(a), static_cast<float*>(b), n);
    });
}

extern "C" da_status da_diag_accept_log(const float* delta, const float* beta, const uint32_t* w, uint8_t* out,
                                        int64_t n)
{
    if (n < 0 || (n > 0 && (!delta || !beta || !w || !out))) return DA_EINVAL;
    if (n == 0) return DA_OK;
    std::vector<char> in((size_t)n * 12);
    std::copy((const char*)delta, (const char*)delta + n * 4, in.begin());
    std::copy((const char*)beta, (const char*)beta + n * 4, in.begin() + n * 4);
    std::copy((const char*)w, (const char*)w + n * 4, in.begin() + n * 8);
    return run((size_t)n * 12, (size_t)n, in.data(), out, [&](void* a, void* b) {
        const float* da_ = static_cast<const float*>(a);
        accept_log_kernel<<<(unsigned)((n + 255) / 256), 256>>>(da_, da_ + n, reinterpret_cast<const uint32_t*>(da_ + 2 * n),
                                                                static_cast<uint8_t*>(b), n);
    });
}

extern "C" da_status da_diag_bounded_wait(int64_t ns, int64_t* out3)
{
    if (ns < 1 || ns > 1000000000ll || !out3) return DA_EINVAL;
    const int64_t zero = 0;
    return run(sizeof(zero), 3 * sizeof(unsigned long long), &zero, out3, [&](void*, void* b) {
        wait_probe_kernel<<<1, 32>>>((unsigned long long)ns, static_cast<unsigned long long*>(b));
    });
}

extern "C" da_status da_diag_read_bandwidth(const void* buf, int64_t bytes, int32_t passes, double* seconds)
{
    if (!buf || !seconds || bytes < 16 || bytes % 16 != 0 || passes < 1 ||
        reinterpret_cast<uintptr_t>(buf) % 16 != 0)
        return DA_EINVAL;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return DA_ECUDA;
    }
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    unsigned* sink = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = cudaMalloc(&sink, sizeof(unsigned));
    const long long n16 = bytes / 16;
    const unsigned blocks = (unsigned)sms * 8u;
    const uint4* p = static_cast<const uint4*>(buf);
    if (e == cudaSuccess) {
        read_bw_kernel<<<blocks, 256, 0, st>>>(p, n16, 1, sink);   // brings an L2-sized buffer into L2
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e0, st);
    if (e == cudaSuccess) {
        read_bw_kernel<<<blocks, 256, 0, st>>>(p, n16, passes, sink);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (sink) cudaFree(sink);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return DA_ECUDA;
    }
    *seconds = ms * 1e-3;
    return DA_OK;
}
