// da_fields.cu -- exact full recompute of the local fields h = W x for many
// states, and the energies that go with it.
//
// The DA never computes fields from scratch during a run: all runs start at
// x = 0, where h = 0 and E = 0 (Sec. II, "avoiding the calculation of the
// initial N effective fields").  This library recomputes them only to bound
// the drift of the fp32 fields (one rounding per update) and to evaluate the
// final and best states exactly:
//   int8 couplings:  h_i = sum_j W_ij x_j in int32 (exact);
//   fp32 couplings:  every W_ij is put on the grid 2^-S (S from max|W| and N
//                    so that no sum can overflow), the products are summed
//                    exactly in int64, and h_i is the single fp32 rounding of
//                    that sum.  The result does not depend on the order of the
//                    summation, so any tiling gives the same bits.
// The recompute returns the effective fields g_i = Q_ii + sum_j W_ij x_j that
// the step kernel keeps (Delta E_i = (1 - 2 x_i) g_i); for fp32, Q_ii joins
// the fixed-point sum as one more term.
// Energies: E = sum_i x_i (Q_ii + h_i / 2), exact in int64 for int8; for fp32
// the terms use h_i = (sum_i - round(Q_ii 2^S)) 2^-S in fp64 and are added in
// index order.
#include <cmath>

#include "da_internal.h"

namespace da {
namespace {

constexpr int kRowsPerBlock = 128;
constexpr int kRepsPerThread = 16;

// Thread = one row i (variable) and kRepsPerThread states.  W is symmetric,
// so row j of the matrix is read as column j: consecutive threads read
// consecutive addresses of row j.
template <bool INT8>
__device__ __forceinline__ long long fixed_diag(const void* diag, int i, int S)
{
    if constexpr (INT8) return (long long)static_cast<const int32_t*>(diag)[i];
    else return __float2ll_rn(ldexpf(static_cast<const float*>(diag)[i], S));
}

template <bool INT8>
__global__ void __launch_bounds__(kRowsPerBlock) recompute_kernel(const void* __restrict__ Wv,
                                                                  const void* __restrict__ diag, int N, int ldw,
                                                                  int S, const uint32_t* __restrict__ xs, int nw,
                                                                  int R, void* hout, int npad, long long* sums_t)
{
    const int i = blockIdx.x * kRowsPerBlock + threadIdx.x;
    const int r0 = blockIdx.y * kRepsPerThread;
    const bool row_ok = i < N;
    const long long d0 = row_ok ? fixed_diag<INT8>(diag, i, S) : 0ll;
    long long acc[kRepsPerThread];
#pragma unroll
    for (int q = 0; q < kRepsPerThread; ++q) acc[q] = d0;
    __shared__ uint32_t xw[kRepsPerThread][33];
    for (int j0 = 0; j0 < N; j0 += 32) {
        __syncthreads();
        if (threadIdx.x < kRepsPerThread) {
            const int rr = r0 + threadIdx.x;
            xw[threadIdx.x][0] = rr < R ? xs[(size_t)rr * nw + (j0 >> 5)] : 0u;
        }
        __syncthreads();
        uint32_t bits[kRepsPerThread];
#pragma unroll
        for (int q = 0; q < kRepsPerThread; ++q) bits[q] = xw[q][0];
        const int jn = min(32, N - j0);
        for (int jj = 0; jj < jn; ++jj) {
            long long mval = 0;
            if (row_ok) {
                const int j = j0 + jj;
                if constexpr (INT8) {
                    mval = (long long)static_cast<const int8_t*>(Wv)[(size_t)j * ldw + i];
                } else {
                    const float wf = static_cast<const float*>(Wv)[(size_t)j * ldw + i];
                    mval = __float2ll_rn(ldexpf(wf, S));
                }
            }
#pragma unroll
            for (int q = 0; q < kRepsPerThread; ++q)
                acc[q] += ((bits[q] >> jj) & 1u) ? mval : 0ll;
        }
    }
    if (i >= npad) return;
#pragma unroll
    for (int q = 0; q < kRepsPerThread; ++q) {
        const int rr = r0 + q;
        if (rr >= R) break;
        if (hout) {
            if constexpr (INT8)
                static_cast<int32_t*>(hout)[(size_t)rr * npad + i] = row_ok ? (int32_t)acc[q] : 0;
            else
                static_cast<float*>(hout)[(size_t)rr * npad + i] = row_ok ? ldexpf(__ll2float_rn(acc[q]), -S) : 0.f;
        }
        if (sums_t && row_ok) sums_t[(size_t)i * R + rr] = acc[q];
    }
}

// One thread per state: E = sum_i x_i (d_i + h_i / 2) in index order.
template <bool INT8>
__global__ void energy_kernel(const void* __restrict__ diag, int N, int S, const uint32_t* __restrict__ xs, int nw,
                              int R, const long long* __restrict__ sums_t, long long* E, int Estride)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    const uint32_t* x = xs + (size_t)r * nw;
    if constexpr (INT8) {
        long long lin = 0, quad = 0;
        for (int i = 0; i < N; ++i) {
            if (!((x[i >> 5] >> (i & 31)) & 1u)) continue;
            const long long di = static_cast<const int32_t*>(diag)[i];
            lin += di;
            quad += sums_t[(size_t)i * R + r] - di;
        }
        E[(size_t)r * Estride] = lin + quad / 2;
    } else {
        double e = 0.0;
        for (int i = 0; i < N; ++i) {
            if (!((x[i >> 5] >> (i & 31)) & 1u)) continue;
            const long long hfix = sums_t[(size_t)i * R + r] - fixed_diag<false>(diag, i, S);
            const double hd = ldexp(__ll2double_rn(hfix), -S);
            e = __dadd_rn(e, __dadd_rn((double)static_cast<const float*>(diag)[i], __dmul_rn(0.5, hd)));
        }
        E[(size_t)r * Estride] = __double_as_longlong(e);
    }
}

// g[r][i] = diag[i] for i < N, 0 on the padding.
template <bool INT8>
__global__ void init_state_kernel(const void* __restrict__ diag, int N, int R, void* g, int npad)
{
    const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= (long long)R * npad) return;
    const int i = (int)(idx % npad);
    if constexpr (INT8)
        static_cast<int32_t*>(g)[idx] = i < N ? static_cast<const int32_t*>(diag)[i] : 0;
    else
        static_cast<float*>(g)[idx] = i < N ? static_cast<const float*>(diag)[i] : 0.f;
}

}  // namespace

int fix_scale(float amax, int N)
{
    if (!(amax > 0.0f)) return 0;
    int e = 0;
    std::frexp(amax, &e);  // amax = f 2^e, f in [0.5, 1)
    int L = 0;
    while ((1ll << L) < (long long)N + 1) ++L;
    return 62 - L - e;
}

cudaError_t launch_init_state(bool is_int8, const void* diag, int N, int R, void* g, int npad, cudaStream_t st)
{
    const long long n = (long long)R * npad;
    if (n == 0) return cudaSuccess;
    const int tb = 256;
    const unsigned blocks = (unsigned)((n + tb - 1) / tb);
    if (is_int8)
        init_state_kernel<true><<<blocks, tb, 0, st>>>(diag, N, R, g, npad);
    else
        init_state_kernel<false><<<blocks, tb, 0, st>>>(diag, N, R, g, npad);
    return cudaGetLastError();
}

cudaError_t launch_recompute(bool is_int8, const void* W, const void* diag, int N, int ldw, int S,
                             const uint32_t* xs, int nw, int R, void* hout, int npad,
                             long long* E, int Estride, cudaStream_t st, long long* sums_t)
{
    if (R <= 0) return cudaSuccess;
    const int rows = hout ? npad : N;
    dim3 grid((rows + kRowsPerBlock - 1) / kRowsPerBlock, (R + kRepsPerThread - 1) / kRepsPerThread);
    if (is_int8)
        recompute_kernel<true><<<grid, kRowsPerBlock, 0, st>>>(W, diag, N, ldw, S, xs, nw, R, hout, npad, sums_t);
    else
        recompute_kernel<false><<<grid, kRowsPerBlock, 0, st>>>(W, diag, N, ldw, S, xs, nw, R, hout, npad, sums_t);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess || !E) return err;
    const int tb = 128;
    if (is_int8)
        energy_kernel<true><<<(R + tb - 1) / tb, tb, 0, st>>>(diag, N, S, xs, nw, R, sums_t, E, Estride);
    else
        energy_kernel<false><<<(R + tb - 1) / tb, tb, 0, st>>>(diag, N, S, xs, nw, R, sums_t, E, Estride);
    return cudaGetLastError();
}

}  // namespace da
