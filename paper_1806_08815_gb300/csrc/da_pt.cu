// da_pt.cu -- replica exchange of the parallel-tempering Digital Annealer
// (PTDA, Sec. II; the exchange rule is the Metropolis swap of Algorithm 4).
//
// After every sweep (N DA steps of every replica) each ladder proposes swaps
// between temperature indices (0,1), (1,2), ..., (K-2,K-1) in that order.
// The pair (p, p+1), holding replicas a and c, swaps its temperature labels
// with probability min(1, exp((beta_p - beta_{p+1})(E_a - E_c))).  The paper
// runs this step on a CPU; here it runs on the device between step launches,
// one thread per ladder, so the ladder's state never leaves HBM.
#include "da_device.cuh"
#include "da_internal.h"

namespace da {
namespace {

template <bool INT8>
__device__ __forceinline__ double energy_of(const ReplicaScalars& s)
{
    if constexpr (INT8) return (double)s.E;
    else return __longlong_as_double(s.E);
}

template <bool INT8>
__global__ void pt_exchange_kernel(const float* __restrict__ betas, int K, int L, const ReplicaScalars* __restrict__ sc,
                                   int* temp_of, int* rep_at, long long* swaps, uint8_t* swap_trace,
                                   long long sweep, long long sweeps, uint64_t seed)
{
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= L) return;
    const uint32_t key0 = (uint32_t)seed, key1 = (uint32_t)(seed >> 32);
    int* at = rep_at + (size_t)l * K;
    int* tof = temp_of + (size_t)l * K;
    const ReplicaScalars* s = sc + (size_t)l * K;
    for (int p = 0; p + 1 < K; ++p) {
        const int a = at[p], c = at[p + 1];
        const double arg = __dmul_rn(__dsub_rn((double)betas[p], (double)betas[p + 1]),
                                     __dsub_rn(energy_of<INT8>(s[a]), energy_of<INT8>(s[c])));
        bool acc = arg >= 0.0;
        if (!acc) {
            const u32x4 rr = philox4x32_10((uint32_t)p, (uint32_t)sweep, (uint32_t)l, 2u, key0, key1);
            acc = uniform01(rr.x) < exp_neg(__double2float_rn(arg));
        }
        if (swap_trace) swap_trace[((size_t)l * sweeps + sweep) * (K - 1) + p] = acc ? 1 : 0;
        if (acc) {
            at[p] = c;
            at[p + 1] = a;
            tof[a] = p + 1;
            tof[c] = p;
            if (swaps) swaps[(size_t)l * (K - 1) + p] += 1;
        }
    }
}

}  // namespace

cudaError_t launch_pt_exchange(bool is_int8, const float* betas, int K, int L,
                               const ReplicaScalars* sc, int* temp_of, int* rep_at,
                               long long* swaps, uint8_t* swap_trace, long long sweep, long long sweeps,
                               uint64_t seed, cudaStream_t st)
{
    if (L <= 0 || K < 2) return cudaSuccess;
    const int tb = 64;
    if (is_int8)
        pt_exchange_kernel<true><<<(L + tb - 1) / tb, tb, 0, st>>>(betas, K, L, sc, temp_of, rep_at, swaps,
                                                                   swap_trace, sweep, sweeps, seed);
    else
        pt_exchange_kernel<false><<<(L + tb - 1) / tb, tb, 0, st>>>(betas, K, L, sc, temp_of, rep_at, swaps,
                                                                    swap_trace, sweep, sweeps, seed);
    return cudaGetLastError();
}

}  // namespace da
