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

// The same exchange pass with one warp per ladder: the lanes stage what does
// not depend on the order of the labels (the replicas' energies, the fp64 gaps
// beta_p - beta_{p+1}, each pair's uniform draw) in shared memory, lane 0 makes
// the sequential pass (the same fp64 and fp32 operations in the same order as
// the one-thread form, so every decision is identical), and the lanes write the
// labels, counts and trace back.  Shared memory: K * 32 bytes per ladder.
template <bool INT8>
__global__ void pt_exchange_warp_kernel(const float* __restrict__ betas, int K, int L,
                                        const ReplicaScalars* __restrict__ sc, int* temp_of, int* rep_at,
                                        long long* swaps, uint8_t* swap_trace, long long sweep, long long sweeps,
                                        uint64_t seed)
{
    extern __shared__ __align__(16) unsigned char pt_smem[];
    double* E = reinterpret_cast<double*>(pt_smem);   // [K] energy of replica r
    double* gap = E + K;                               // [K - 1] beta_p - beta_{p+1}
    float* u = reinterpret_cast<float*>(gap + K);      // [K - 1] the pair's uniform draw
    int* at = reinterpret_cast<int*>(u + K);           // [K] replica at temperature index k
    uint8_t* acc = reinterpret_cast<uint8_t*>(at + K); // [K - 1] decisions
    const int l = blockIdx.x;
    if (l >= L) return;
    const int lane = threadIdx.x;
    const uint32_t key0 = (uint32_t)seed, key1 = (uint32_t)(seed >> 32);
    const ReplicaScalars* s = sc + (size_t)l * K;
    for (int k = lane; k < K; k += 32) {
        E[k] = energy_of<INT8>(s[k]);
        at[k] = rep_at[(size_t)l * K + k];
        if (k + 1 < K) {
            gap[k] = __dsub_rn((double)betas[k], (double)betas[k + 1]);
            u[k] = uniform01(philox4x32_10((uint32_t)k, (uint32_t)sweep, (uint32_t)l, 2u, key0, key1).x);
        }
    }
    __syncwarp();
    if (lane == 0) {
        for (int p = 0; p + 1 < K; ++p) {
            const int a = at[p], c = at[p + 1];
            const double arg = __dmul_rn(gap[p], __dsub_rn(E[a], E[c]));
            const bool ok = arg >= 0.0 || u[p] < exp_neg(__double2float_rn(arg));
            acc[p] = ok ? 1 : 0;
            if (ok) {
                at[p] = c;
                at[p + 1] = a;
            }
        }
    }
    __syncwarp();
    for (int k = lane; k < K; k += 32) {
        const int r = at[k];
        rep_at[(size_t)l * K + k] = r;
        temp_of[(size_t)l * K + r] = k;
        if (k + 1 < K) {
            if (swap_trace) swap_trace[((size_t)l * sweeps + sweep) * (K - 1) + k] = acc[k];
            if (swaps && acc[k]) swaps[(size_t)l * (K - 1) + k] += 1;
        }
    }
}

// The adaptive ladder (Sec. II: highest and lowest temperature fixed, the
// others moved towards equal exchange acceptance of neighbouring pairs):
// win[p] = exchanges of pair p accepted over all ladders since the last
// update, out of `proposals`; each gap beta_{p+1} - beta_p is multiplied by
// w^(1/8), w = (win[p] + 1) / (proposals + 2) (three correctly rounded square
// roots; the damping keeps the feedback stable down to acceptances near
// 1e-3), and the gaps are rescaled to the fixed span.  One block: the counts
// are summed over ladders in parallel, the ladder is updated by one thread in
// fp64 in pair order (the same operations, in the same order, as the CPU
// reference), then rounded to fp32.
__device__ __forceinline__ double gap_weight(long long accepted, long long proposals)
{
    const double w = __ddiv_rn(__dadd_rn((double)accepted, 1.0), __dadd_rn((double)proposals, 2.0));
    return __dsqrt_rn(__dsqrt_rn(__dsqrt_rn(w)));
}

__global__ void pt_adapt_kernel(float* betas, int K, int L, const long long* __restrict__ swaps, long long* seen,
                                long long proposals)
{
    extern __shared__ long long win[];
    const int P = K - 1;
    for (int p = threadIdx.x; p < P; p += blockDim.x) {
        long long tot = 0;
        for (int l = 0; l < L; ++l) tot += swaps[(size_t)l * P + p];
        win[p] = tot - seen[p];
        seen[p] = tot;
    }
    __syncthreads();
    if (threadIdx.x != 0 || K < 3 || proposals < 1) return;
    double total = 0.0;
    for (int p = 0; p < P; ++p) {
        const double gap = __dsub_rn((double)betas[p + 1], (double)betas[p]);
        total = __dadd_rn(total, __dmul_rn(gap, gap_weight(win[p], proposals)));
    }
    if (!(total > 0.0)) return;
    const double span = __dsub_rn((double)betas[K - 1], (double)betas[0]);
    double b = (double)betas[0];
    float prev = betas[0];   // betas[p] before its update, for the gap of pair p
    for (int p = 0; p + 2 < K; ++p) {
        const float next = betas[p + 1];
        const double gap = __dsub_rn((double)next, (double)prev);
        b = __dadd_rn(b, __ddiv_rn(__dmul_rn(__dmul_rn(gap, gap_weight(win[p], proposals)), span), total));
        betas[p + 1] = __double2float_rn(b);
        prev = next;
    }
}

}  // namespace

cudaError_t launch_pt_adapt(float* betas, int K, int L, const long long* swaps, long long* seen, long long proposals,
                            cudaStream_t st)
{
    if (K < 2 || L < 1) return cudaSuccess;
    pt_adapt_kernel<<<1, 256, (size_t)(K - 1) * sizeof(long long), st>>>(betas, K, L, swaps, seen, proposals);
    return cudaGetLastError();
}

cudaError_t launch_pt_exchange(bool is_int8, const float* betas, int K, int L,
                               const ReplicaScalars* sc, int* temp_of, int* rep_at,
                               long long* swaps, uint8_t* swap_trace, long long sweep, long long sweeps,
                               uint64_t seed, cudaStream_t st)
{
    if (L <= 0 || K < 2) return cudaSuccess;
    const size_t smem = (size_t)K * 32;
    if (smem <= 48 * 1024) {   // one warp per ladder
        if (is_int8) {
            prefer_shared<pt_exchange_warp_kernel<true>>();
            pt_exchange_warp_kernel<true><<<L, 32, smem, st>>>(betas, K, L, sc, temp_of, rep_at, swaps, swap_trace,
                                                               sweep, sweeps, seed);
        } else {
            prefer_shared<pt_exchange_warp_kernel<false>>();
            pt_exchange_warp_kernel<false><<<L, 32, smem, st>>>(betas, K, L, sc, temp_of, rep_at, swaps, swap_trace,
                                                                sweep, sweeps, seed);
        }
        return cudaGetLastError();
    }
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
