// da_serve_kernel.cuh -- the persistent kernel of the request loop (da_serve.cu).
//
// Warps pull work units (request slot, replica) from a ring that the host
// keeps filling while the kernel runs, so requests that arrive while others
// are on the GPU join the same launch (continuous batching).  A unit is one
// replica annealed for all its steps by one warp with its state in registers
// (WarpReplica); its exact final and best energies are evaluated by the warp
// itself.  The last unit of a request raises the request's completion flag in
// host-mapped memory.
//
// Every wait is bounded.  The host ends the kernel through the stop flag once
// no request of this path has been in flight for a while, and relaunches it
// when new units arrive; so the warps of one launch leave together and a
// launch never drains to a few warps while units wait.  A warp that finds no
// unit for `idle_polls` rounds (seconds) leaves on its own all the same.
#pragma once
#include <cuda/atomic>

#include "da_internal.h"
#include "da_replica.cuh"

namespace da {

// One admitted request, as the kernel sees it (device memory, by slot).
struct alignas(16) ServeDesc {
    const void* W;
    const void* diag;
    const float* beta;
    uint32_t* xs;           // [2R][V] words: final states, then best states
    double* E;              // [3R]: exact final, exact best, |tracked - exact final|
    long long* flips;       // [R]
    unsigned int* done;     // device counter of finished replicas
    volatile unsigned int* flag;  // host-mapped completion flag
    long long T, P;
    uint64_t seed;
    int N, ldw, S, R, V;
    int int8;
    float inc;
};

struct ServeUnit {
    int slot;
    int replica;
};

struct ServeParams {
    const ServeDesc* descs;              // [max_slots], device
    const ServeUnit* ring;               // [cap], host-mapped
    const unsigned long long* tail;      // host-mapped, written by the host
    unsigned long long* head;            // device, units claimed
    const volatile int* stop;            // host-mapped
    unsigned long long cap;
    int idle_polls;
};

namespace serve_detail {

using step_detail::Arith;
using step_detail::WarpReplica;

template <typename Tw, int V>
__device__ __noinline__ void run_unit(const ServeDesc& d, int r)
{
    using R_ = WarpReplica<Tw, V, true>;
    using H = typename R_::H;
    const int lane = threadIdx.x & 31;
    R_ rp;
    rp.init(static_cast<const Tw*>(d.W), d.N, d.ldw, (uint32_t)r, d.xs + ((size_t)d.R + r) * V);
#pragma unroll
    for (int v = 0; v < V; ++v)
        rp.h[v] = ((rp.valid >> v) & 1u) ? step_detail::ldx<true>(static_cast<const H*>(d.diag) + rp.base + v) : H(0);
    rp.xm = 0;
    rp.m = 0;
    rp.Ecur = 0;
    rp.Ebest = 0;
    rp.flips = 0;
    // zero the best-state words (the slot's memory is reused)
    if (lane % R_::P == 0) d.xs[((size_t)d.R + r) * V + (rp.base >> 5)] = 0u;
    __syncwarp();
    const PhiloxKeys keys(d.seed);
    if (d.T > 0) rp.draw(0u, keys);
    float beta_next = d.T > 0 ? __ldcg(d.beta) : 0.f;
    for (long long t = 0; t < d.T; ++t) {
        const float beta = beta_next;
        if (t + 1 < d.T) beta_next = __ldcg(d.beta + t + 1);
        rp.template step<false>(t, t + 1 < d.T, beta, d.inc, keys);
        if constexpr (sizeof(Tw) == 4) {
            if (d.P > 0 && (t + 1) % d.P == 0) {
                rp.recompute(static_cast<const float*>(d.diag), d.S);
                if (t + 1 < d.T) rp.draw((uint32_t)(t + 1), keys);
            }
        }
    }
    rp.flush_best();
    const uint32_t word = rp.word();
    if (lane % R_::P == 0) d.xs[(size_t)r * V + (rp.base >> 5)] = word;
    double ef, eb, drift;
    if constexpr (sizeof(Tw) == 4) {
        const double tracked = rp.Ecur;
        rp.recompute(static_cast<const float*>(d.diag), d.S);   // exact energy of the final state
        ef = rp.Ecur;
        drift = fabs(tracked - ef);
        __syncwarp();
        const uint32_t bw = d.xs[((size_t)d.R + r) * V + (rp.base >> 5)];
        rp.xm = (bw >> (rp.base & 31)) & R_::VMASK;
        rp.recompute(static_cast<const float*>(d.diag), d.S);   // exact energy of the best state
        eb = rp.Ecur;
    } else {
        ef = (double)rp.Ecur;   // integer energies are tracked exactly
        eb = (double)rp.Ebest;
        drift = 0.0;
    }
    if (lane == 0) {
        d.E[r] = ef;
        d.E[d.R + r] = eb;
        d.E[2 * d.R + r] = drift;
        d.flips[r] = rp.flips;
    }
}

}  // namespace serve_detail

__global__ void __launch_bounds__(128) serve_kernel(const __grid_constant__ ServeParams sp);

}  // namespace da
