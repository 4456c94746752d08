// da_plain.cu -- the plain GPU form of the DA step, kept as the baseline the
// library's own kernels are measured against: one kernel launch per step of
// Algorithm 2, one thread block per replica, one thread per variable, fp32
// fields and state in global memory between launches, no persistence.
// It draws the same random numbers as the main path and uses the same fp32
// arithmetic (integer couplings are exact in fp32), without the periodic
// recompute, so its trajectories equal the oracle's fp32 mode without
// recompute.
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "da.h"
#include "da_device.cuh"
#include "da_internal.h"

namespace da {
namespace {

struct PlainScalars {
    double E, best;
    long long flips;
    uint32_t m, pad;
};

__device__ __forceinline__ float coupling(const void* W, bool int8, size_t idx)
{
    return int8 ? (float)static_cast<const int8_t*>(W)[idx] : static_cast<const float*>(W)[idx];
}

__global__ void plain_init_kernel(const void* diag, bool int8, int N, int R, float* g, uint8_t* x, uint8_t* bx,
                                  PlainScalars* sc)
{
    const int r = blockIdx.x;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        g[(size_t)r * N + i] = int8 ? (float)static_cast<const int32_t*>(diag)[i] : static_cast<const float*>(diag)[i];
        x[(size_t)r * N + i] = 0;
        bx[(size_t)r * N + i] = 0;
    }
    if (threadIdx.x == 0) sc[r] = PlainScalars{0.0, 0.0, 0, 0, 0};
}

// One DA step of replica blockIdx.x.
__global__ void __launch_bounds__(1024) plain_step_kernel(const void* W, bool int8, int N, int ldw, float* g, uint8_t* x,
                                                          uint8_t* bx, PlainScalars* sc, const float* beta_sched,
                                                          long long t, float inc, uint64_t seed, int* trace,
                                                          long long trace_T)
{
    __shared__ int warp_cnt[32];
    __shared__ int s_rank;      // rank j of the chosen trial, -1 if none accepted
    __shared__ int s_k;         // its index
    __shared__ float s_dE;
    __shared__ int s_x;
    __shared__ int s_best;
    const int r = blockIdx.x;
    const int i = threadIdx.x;
    const int lane = i & 31, warp = i >> 5;
    float* gr = g + (size_t)r * N;
    uint8_t* xr = x + (size_t)r * N;
    const PlainScalars s0 = sc[r];
    const float beta = beta_sched[t];
    const float Eoff = __fmul_rn(__uint2float_rn(s0.m), inc);
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    bool acc = false;
    float dE = 0.f;
    int xi = 0;
    if (i < N) {
        xi = xr[i];
        dE = xi ? -gr[i] : gr[i];
        const float delta = __fsub_rn(dE, Eoff);
        if (delta <= 0.0f) {
            acc = true;
        } else {
            const float a = -__fmul_rn(beta, delta);
            if (a > kExpCut) {
                const u32x4 rr = philox4x32_10((uint32_t)(i >> 2), (uint32_t)t, (uint32_t)r, 0u, k0, k1);
                acc = uniform01(pick(rr, i & 3)) < exp_neg(a);
            }
        }
    }
    const uint32_t b = __ballot_sync(0xffffffffu, acc);
    if (lane == 0) warp_cnt[warp] = __popc(b);
    __syncthreads();
    if (warp == 0) {
        const int nw = (blockDim.x + 31) / 32;
        const int c = lane < nw ? warp_cnt[lane] : 0;
        int incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int n = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += n;
        }
        const int total = __shfl_sync(0xffffffffu, incl, 31);
        __syncwarp();
        if (lane < nw) warp_cnt[lane] = incl - c;  // exclusive prefix
        if (lane == 0) {
            s_rank = -1;
            s_k = -1;
            if (total > 0) {
                const u32x4 cr = philox4x32_10(0u, (uint32_t)(t & ~3ll), (uint32_t)r, 1u, k0, k1);
                s_rank = (int)__umulhi(pick(cr, (int)(t & 3)), (uint32_t)total);
            }
        }
    }
    __syncthreads();
    if (acc && warp_cnt[warp] + __popc(b & ((1u << lane) - 1u)) == s_rank) {
        s_k = i;
        s_dE = dE;
        s_x = xi;
    }
    __syncthreads();
    const int k = s_k;
    if (k >= 0 && i < N) {
        const float w = coupling(W, int8, (size_t)k * ldw + i);
        gr[i] = s_x ? __fsub_rn(gr[i], w) : __fadd_rn(gr[i], w);
        if (i == k) xr[i] = (uint8_t)(xi ^ 1);
    }
    if (i == 0) {
        PlainScalars s = s0;
        if (k >= 0) {
            s.E = __dadd_rn(s.E, (double)s_dE);
            s.flips += 1;
            s.m = 0;
        } else {
            s.m += 1;
        }
        if (trace) trace[(size_t)r * trace_T + t] = k;
        s_best = (k >= 0 && s.E < s.best) ? 1 : 0;
        if (s_best) s.best = s.E;
        sc[r] = s;
    }
    __syncthreads();
    if (s_best && i < N) bx[(size_t)r * N + i] = xr[i];
}

__global__ void plain_pack_kernel(const uint8_t* x, int N, int R, uint32_t* words, int nw)
{
    const int r = blockIdx.x;
    for (int wi = threadIdx.x; wi < nw; wi += blockDim.x) {
        uint32_t v = 0;
        for (int b = 0; b < 32; ++b) {
            const int i = wi * 32 + b;
            if (i < N && x[(size_t)r * N + i]) v |= 1u << b;
        }
        words[(size_t)r * nw + wi] = v;
    }
}

}  // namespace

// Host driver: steps [0, T) as T launches on `st`.
cudaError_t plain_anneal(const void* W, const void* diag, bool int8, int N, int ldw, int S, const float* beta_dev,
                         long long T, float inc, int R, uint64_t seed, void* ws, int* trace, uint32_t* words_out,
                         long long* eex, long long* part, double* tracked_E, int64_t* flips, cudaStream_t st)
{
    char* base = static_cast<char*>(ws);
    float* g = reinterpret_cast<float*>(base);
    uint8_t* x = reinterpret_cast<uint8_t*>(g + (size_t)R * N);
    uint8_t* bx = x + (size_t)R * N;
    PlainScalars* sc = reinterpret_cast<PlainScalars*>(base + (((size_t)R * N * 6 + 255) / 256) * 256);
    const int threads = std::min(1024, (N + 31) / 32 * 32);
    plain_init_kernel<<<R, 256, 0, st>>>(diag, int8, N, R, g, x, bx, sc);
    cudaError_t e = cudaGetLastError();
    for (long long t = 0; t < T && e == cudaSuccess; ++t) {
        plain_step_kernel<<<R, threads, 0, st>>>(W, int8, N, ldw, g, x, bx, sc, beta_dev, t, inc, seed, trace, T);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return e;
    const int nw = (N + 31) / 32;
    plain_pack_kernel<<<R, 64, 0, st>>>(x, N, R, words_out, nw);
    plain_pack_kernel<<<R, 64, 0, st>>>(bx, N, R, words_out + (size_t)R * nw, nw);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    e = launch_recompute(int8, W, diag, N, ldw, S, words_out, nw, 2 * R, nullptr, N, eex, 1, st, part);
    if (e != cudaSuccess) return e;
    std::vector<PlainScalars> hs((size_t)R);
    e = cudaMemcpyAsync(hs.data(), sc, (size_t)R * sizeof(PlainScalars), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return e;
    for (int r = 0; r < R; ++r) {
        tracked_E[r] = hs[r].E;
        flips[r] = hs[r].flips;
    }
    return cudaSuccess;
}

size_t plain_workspace_bytes(int N, int R)
{
    return (((size_t)R * N * 6 + 255) / 256) * 256 + (size_t)R * sizeof(PlainScalars);
}

}  // namespace da
