// da_fields.cu -- exact full recompute of the effective fields
// g = diag(Q) + W x for many states, and the energies that go with it.
//
// The DA never computes fields from scratch during a run: all runs start at
// x = 0, where the fields are the linear terms and E = 0 (Sec. II, "avoiding
// the calculation of the initial N effective fields").  This library
// recomputes them only to bound the drift of the fp32 fields (one rounding per
// update) and to evaluate final and best states exactly:
//   integer couplings (int8, int16):  g_i = Q_ii + sum_j W_ij x_j in integers (exact);
//   fp32 couplings:  Q_ii and every W_ij are put on the grid 2^-S (S from
//                    max(|W|, |Q_ii|) and N, so that no sum can overflow),
//                    summed exactly in int64, and g_i is the single fp32
//                    rounding of that sum.
// Energies: E = sum_{x_i=1} (Q_ii + g_i) / 2, summed exactly (int64 for int8;
// on the fixed-point grid in 128-bit integers for fp32, then rounded once to
// fp64).  Every sum is exact, so the tiling and the reduction order do not
// change a single bit.
//
// Tiling: a block owns 64 rows (variables i) and 32 states (4 per warp).  For
// each chunk of 32 columns j it stages the fixed-point tile of W in shared
// memory once, and every warp walks the set bits of its states' word j/32:
// only x_j = 1 contributes, and the loop is uniform across the warp.
#include <algorithm>
#include <cmath>

#include "da.h"
#include "da_fixed.cuh"
#include "da_internal.h"

namespace da {
namespace {

constexpr int kRows = 64;           // rows per block
constexpr int kStatesPerWarp = 4;
constexpr int kWarps = 8;
constexpr int kStates = kWarps * kStatesPerWarp;

// Coupling types of the recompute: the da_dtype values (kWInt8, kWFp32, kWInt16).
template <int K>
__device__ __forceinline__ long long fixed_of(const void* a, size_t idx, int S)
{
    if constexpr (K == kWInt8) return (long long)static_cast<const int8_t*>(a)[idx];
    else if constexpr (K == kWInt16) return (long long)static_cast<const int16_t*>(a)[idx];
    else return fixed_of_f32(static_cast<const float*>(a)[idx], S);
}

template <int K>
__device__ __forceinline__ long long fixed_diag(const void* diag, int i, int S)
{
    if constexpr (K != kWFp32) return (long long)static_cast<const int32_t*>(diag)[i];
    else return fixed_of_f32(static_cast<const float*>(diag)[i], S);
}

struct I128 {
    unsigned long long lo;
    long long hi;
};

__device__ __forceinline__ I128 i128_of(long long v) { return {(unsigned long long)v, v < 0 ? -1ll : 0ll}; }

__device__ __forceinline__ I128 i128_add(I128 a, I128 b)
{
    I128 c;
    c.lo = a.lo + b.lo;
    c.hi = a.hi + b.hi + (c.lo < a.lo ? 1 : 0);
    return c;
}

__device__ __forceinline__ I128 warp_sum(I128 v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        I128 n;
        n.lo = __shfl_xor_sync(0xffffffffu, v.lo, o);
        n.hi = __shfl_xor_sync(0xffffffffu, v.hi, o);
        v = i128_add(v, n);
    }
    return v;
}

// Fields of states xs[R][nw] for rows [64 bx, 64 bx + 64); partial energy
// sums of those rows into part[bx][R] (two 64-bit words each).
template <int K>
__global__ void __launch_bounds__(kWarps * 32) recompute_kernel(const void* __restrict__ Wv,
                                                                const void* __restrict__ diag, int N, int ldw, int S,
                                                                const uint32_t* __restrict__ xs, int nw, int R,
                                                                void* hout, int npad, I128* part)
{
    __shared__ long long M[32][kRows];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int i0 = blockIdx.x * kRows;
    const int r0 = blockIdx.y * kStates + warp * kStatesPerWarp;
    const int ia = i0 + lane, ib = i0 + 32 + lane;
    long long acc[kStatesPerWarp][2];
    constexpr bool INT8 = K != kWFp32;   // integer fields and energies
    const long long da_ = ia < N ? fixed_diag<K>(diag, ia, S) : 0ll;
    const long long db_ = ib < N ? fixed_diag<K>(diag, ib, S) : 0ll;
#pragma unroll
    for (int q = 0; q < kStatesPerWarp; ++q) { acc[q][0] = da_; acc[q][1] = db_; }

    // staging: thread t loads 8 consecutive entries of row j0 + t/8
    const int sj = threadIdx.x >> 3;
    const int sc = (threadIdx.x & 7) * 8;
    for (int j0 = 0; j0 < N; j0 += 32) {
        __syncthreads();
        const int j = j0 + sj;
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const int i = i0 + sc + c;
            M[sj][sc + c] = (j < N && i < N) ? fixed_of<K>(Wv, (size_t)j * ldw + i, S) : 0ll;
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < kStatesPerWarp; ++q) {
            const int r = r0 + q;
            uint32_t word = r < R ? xs[(size_t)r * nw + (j0 >> 5)] : 0u;
            while (word) {
                const int jj = __ffs(word) - 1;
                word &= word - 1;
                acc[q][0] += M[jj][lane];
                acc[q][1] += M[jj][32 + lane];
            }
        }
    }

#pragma unroll
    for (int q = 0; q < kStatesPerWarp; ++q) {
        const int r = r0 + q;
        if (r >= R) break;     // warp-uniform
        if (hout) {
            if (ia < npad) {
                if constexpr (INT8)
                    static_cast<int32_t*>(hout)[(size_t)r * npad + ia] = ia < N ? (int32_t)acc[q][0] : 0;
                else
                    static_cast<float*>(hout)[(size_t)r * npad + ia] = ia < N ? scaled_f32_of(acc[q][0], S) : 0.f;
            }
            if (ib < npad) {
                if constexpr (INT8)
                    static_cast<int32_t*>(hout)[(size_t)r * npad + ib] = ib < N ? (int32_t)acc[q][1] : 0;
                else
                    static_cast<float*>(hout)[(size_t)r * npad + ib] = ib < N ? scaled_f32_of(acc[q][1], S) : 0.f;
            }
        }
        if (part) {
            const uint32_t xa = ia < N ? (xs[(size_t)r * nw + (ia >> 5)] >> (ia & 31)) & 1u : 0u;
            const uint32_t xb = ib < N ? (xs[(size_t)r * nw + (ib >> 5)] >> (ib & 31)) & 1u : 0u;
            I128 t = i128_add(i128_of(xa ? da_ + acc[q][0] : 0ll), i128_of(xb ? db_ + acc[q][1] : 0ll));
            t = warp_sum(t);
            if (lane == 0) part[(size_t)blockIdx.x * R + r] = t;
        }
    }
}

// E[r] = (sum over row tiles of the partial sums) / 2^(S+1), exact for int8,
// rounded once to fp64 for fp32.
template <bool INT8>
__global__ void energy_kernel(const I128* __restrict__ part, int tiles, int R, int S, long long* E, int Estride)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    I128 s = {0ull, 0ll};
    for (int b = 0; b < tiles; ++b) s = i128_add(s, part[(size_t)b * R + r]);
    if constexpr (INT8) {
        E[(size_t)r * Estride] = (long long)s.lo / 2;   // |2E| < 2^63
    } else {
        // value = hi 2^64 + lo; top = value >> 32 (exact in fp64, |value| < 2^76)
        const long long top = (long long)((unsigned long long)s.hi << 32 | (s.lo >> 32));
        const double bottom = (double)(uint32_t)(s.lo & 0xFFFFFFFFull);
        const double v = __fma_rn((double)top, 4294967296.0, bottom);
        E[(size_t)r * Estride] = __double_as_longlong(ldexp(v, -(S + 1)));
    }
}

// g[r][i] = diag[i] for i < N, 0 on the padding (MODE 0: int32 diag and
// fields, 1: fp32, 2: int32 diag into fp32 fields, exact below 2^24).
template <int MODE>
__global__ void init_state_kernel(const void* __restrict__ diag, int N, int R, void* g, int npad)
{
    const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= (long long)R * npad) return;
    const int i = (int)(idx % npad);
    if constexpr (MODE == 0)
        static_cast<int32_t*>(g)[idx] = i < N ? static_cast<const int32_t*>(diag)[i] : 0;
    else if constexpr (MODE == 1)
        static_cast<float*>(g)[idx] = i < N ? static_cast<const float*>(diag)[i] : 0.f;
    else
        static_cast<float*>(g)[idx] = i < N ? __int2float_rn(static_cast<const int32_t*>(diag)[i]) : 0.f;
}

__global__ void best_fixup_kernel(int R, ReplicaScalars* sc, bool int8, const uint32_t* x, uint32_t* bestx, int nw)
{
    const int r = blockIdx.x;
    ReplicaScalars s = sc[r];
    if (!s.check) return;
    const bool better = int8 ? s.E < s.best : __longlong_as_double(s.E) < __longlong_as_double(s.best);
    if (better) {
        for (int w = threadIdx.x; w < nw; w += blockDim.x) bestx[(size_t)r * nw + w] = x[(size_t)r * nw + w];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (better) s.best = s.E;
        s.check = 0;
        sc[r] = s;
    }
}

}  // namespace

cudaError_t launch_best_fixup(int R, ReplicaScalars* sc, bool is_int8, const uint32_t* x, uint32_t* bestx, int nw,
                              cudaStream_t st)
{
    if (R <= 0) return cudaSuccess;
    prefer_shared<best_fixup_kernel>();
    best_fixup_kernel<<<R, 64, 0, st>>>(R, sc, is_int8, x, bestx, nw);
    return cudaGetLastError();
}

int fix_scale(float amax, int N)
{
    if (!(amax > 0.0f)) return 0;
    int e = 0;
    std::frexp(amax, &e);  // amax = f 2^e, f in [0.5, 1)
    int L = 0;
    while ((1ll << L) < (long long)N + 1) ++L;
    return 62 - L - e;
}

// The instance in device layout from Q (n x n, row-major; only the upper
// triangle is read): 32 x 32 tiles of W, each filled from the Q tile that
// holds its entries (its mirror image below the diagonal), staged in shared
// memory so that the reads and writes of a warp stay on one row.
template <typename Tq, typename Tw>
__global__ void __launch_bounds__(256) expand_kernel(const Tq* __restrict__ Q, int n, int ldw, Tw* __restrict__ W,
                                                     float* __restrict__ Wf, Tq* __restrict__ diag)
{
    __shared__ Tq tile[32][33];
    const int bi = blockIdx.y, bj = blockIdx.x;
    const int a = min(bi, bj), b = max(bi, bj);
    const int tx = threadIdx.x, ty = threadIdx.y;
    for (int r = ty; r < 32; r += 8) {
        const int row = a * 32 + r, col = b * 32 + tx;
        tile[r][tx] = (row < n && col < n) ? Q[(size_t)row * n + col] : Tq(0);
    }
    __syncthreads();
    for (int r = ty; r < 32; r += 8) {
        const int i = bi * 32 + r, j = bj * 32 + tx;
        if (i >= n || j >= n) continue;
        // i < j: Q[i][j] (bi <= bj, the tile as read); i > j: Q[j][i] (the mirror)
        const Tq v = i < j ? tile[r][tx] : i > j ? tile[tx][r] : Tq(0);
        if (W) W[(size_t)i * ldw + j] = (Tw)v;
        if (Wf) Wf[(size_t)i * ldw + j] = (float)v;
        if (i == j) diag[i] = tile[r][tx];
    }
}

__global__ void zero_kernel(uint4* __restrict__ p, size_t n16)
{
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n16; k += (size_t)gridDim.x * blockDim.x)
        p[k] = make_uint4(0u, 0u, 0u, 0u);
}

cudaError_t launch_zero(void* p, size_t bytes, cudaStream_t st)
{
    if (bytes == 0) return cudaSuccess;
    if ((reinterpret_cast<uintptr_t>(p) | bytes) & 15u) return cudaErrorInvalidValue;
    const size_t n16 = bytes / 16;
    const unsigned blocks = (unsigned)std::min<size_t>((n16 + 255) / 256, 4096);
    prefer_shared<zero_kernel>();
    zero_kernel<<<blocks, 256, 0, st>>>(static_cast<uint4*>(p), n16);
    return cudaGetLastError();
}

// One thread per entry m of the reordered rows (pitch 32 V G): in warp slice
// s = m / 32 V, entry m' = 128 q + 4 l + e holds variable i = s 32 V + l V + 4 q + e
// (see step_uses_coal in da_internal.h).
__global__ void __launch_bounds__(256) coalesce_kernel(const float* __restrict__ W, int N, int ldw, int V, int P,
                                                       float* __restrict__ Wc)
{
    const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= (long long)N * P) return;
    const int k = (int)(idx / P), m = (int)(idx - (long long)k * P);
    const int slice = m / (32 * V), mm = m - slice * 32 * V;
    const int q = mm >> 7, l = (mm & 127) >> 2, e = mm & 3;
    const int i = slice * 32 * V + l * V + 4 * q + e;
    Wc[idx] = i < N ? W[(size_t)k * ldw + i] : 0.f;
}

bool step_uses_coal(int wtype, const StepShape& s)
{
    return (wtype == kWFp32 || wtype == kWInt8AsF32) && !s.ws && s.V >= 8;
}

size_t coal_W_bytes(int N, const StepShape& s) { return (size_t)N * s.npad() * sizeof(float); }

cudaError_t launch_coalesce_W(const float* W, int N, int ldw, int V, int G, float* Wc, cudaStream_t st)
{
    const int P = 32 * V * G;
    const long long n = (long long)N * P;
    if (n == 0) return cudaSuccess;
    if (V < 8 || V > 32 || (V & (V - 1)) || G < 1 || G > 8 || (G & (G - 1)) || P < N) return cudaErrorInvalidValue;
    prefer_shared<coalesce_kernel>();
    coalesce_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(W, N, ldw, V, P, Wc);
    return cudaGetLastError();
}

cudaError_t prepare_field_kernels()
{
    prefer_shared<coalesce_kernel>();
    prefer_shared<zero_kernel>();
    prefer_shared<expand_kernel<int32_t, int8_t>>();
    prefer_shared<expand_kernel<int32_t, int16_t>>();
    prefer_shared<expand_kernel<float, float>>();
    prefer_shared<init_state_kernel<0>>();
    prefer_shared<init_state_kernel<1>>();
    prefer_shared<init_state_kernel<2>>();
    prefer_shared<best_fixup_kernel>();
    prefer_shared<recompute_kernel<kWInt8>>();
    prefer_shared<recompute_kernel<kWInt16>>();
    prefer_shared<recompute_kernel<kWFp32>>();
    prefer_shared<energy_kernel<true>>();
    prefer_shared<energy_kernel<false>>();
    return cudaGetLastError();
}

cudaError_t launch_expand_instance(const void* Q, int n, int ldw, int dtype, void* W, float* Wf, void* diag,
                                   cudaStream_t st)
{
    const size_t entries = (size_t)n * ldw + 8192;
    const size_t esz = dtype == DA_INT8 ? 1 : dtype == DA_INT16 ? 2 : 4;
    cudaError_t e = W ? launch_zero(W, entries * esz, st) : cudaSuccess;
    if (e == cudaSuccess && Wf) e = launch_zero(Wf, entries * sizeof(float), st);
    if (e != cudaSuccess) return e;
    const dim3 grid((unsigned)((n + 31) / 32), (unsigned)((n + 31) / 32)), block(32, 8);
    prefer_shared<expand_kernel<int32_t, int8_t>>();
    prefer_shared<expand_kernel<int32_t, int16_t>>();
    prefer_shared<expand_kernel<float, float>>();
    if (dtype == DA_INT8)
        expand_kernel<int32_t, int8_t><<<grid, block, 0, st>>>(static_cast<const int32_t*>(Q), n, ldw,
                                                               static_cast<int8_t*>(W), Wf,
                                                               static_cast<int32_t*>(diag));
    else if (dtype == DA_INT16)
        expand_kernel<int32_t, int16_t><<<grid, block, 0, st>>>(static_cast<const int32_t*>(Q), n, ldw,
                                                                static_cast<int16_t*>(W), Wf,
                                                                static_cast<int32_t*>(diag));
    else
        expand_kernel<float, float><<<grid, block, 0, st>>>(static_cast<const float*>(Q), n, ldw,
                                                            static_cast<float*>(W), Wf, static_cast<float*>(diag));
    return cudaGetLastError();
}

cudaError_t launch_init_state(bool is_int8, const void* diag, int N, int R, void* g, int npad, cudaStream_t st,
                              bool float_fields)
{
    const long long n = (long long)R * npad;
    if (n == 0) return cudaSuccess;
    const int tb = 256;
    const unsigned blocks = (unsigned)((n + tb - 1) / tb);
    prefer_shared<init_state_kernel<0>>();
    prefer_shared<init_state_kernel<1>>();
    prefer_shared<init_state_kernel<2>>();
    if (is_int8 && float_fields)
        init_state_kernel<2><<<blocks, tb, 0, st>>>(diag, N, R, g, npad);
    else if (is_int8)
        init_state_kernel<0><<<blocks, tb, 0, st>>>(diag, N, R, g, npad);
    else
        init_state_kernel<1><<<blocks, tb, 0, st>>>(diag, N, R, g, npad);
    return cudaGetLastError();
}

cudaError_t launch_energy_sum(bool is_int8, const long long* part, int tiles, int R, int S, long long* E, int Estride,
                              cudaStream_t st)
{
    if (R <= 0) return cudaSuccess;
    const int tb = 128;
    const I128* pp = reinterpret_cast<const I128*>(part);
    if (is_int8) {
        prefer_shared<energy_kernel<true>>();
        energy_kernel<true><<<(R + tb - 1) / tb, tb, 0, st>>>(pp, tiles, R, S, E, Estride);
    } else {
        prefer_shared<energy_kernel<false>>();
        energy_kernel<false><<<(R + tb - 1) / tb, tb, 0, st>>>(pp, tiles, R, S, E, Estride);
    }
    return cudaGetLastError();
}

cudaError_t launch_recompute_w(int wtype, const void* W, const void* diag, int N, int ldw, int S,
                               const uint32_t* xs, int nw, int R, void* hout, int npad,
                               long long* E, int Estride, cudaStream_t st, long long* scratch)
{
    if (R <= 0) return cudaSuccess;
    const int rows = hout ? std::max(npad, N) : N;
    const int tiles = (rows + kRows - 1) / kRows;
    dim3 grid(tiles, (R + kStates - 1) / kStates);
    I128* part = E ? reinterpret_cast<I128*>(scratch) : nullptr;
    if (wtype == kWInt8) {
        prefer_shared<recompute_kernel<kWInt8>>();
        recompute_kernel<kWInt8><<<grid, kWarps * 32, 0, st>>>(W, diag, N, ldw, S, xs, nw, R, hout, npad, part);
    } else if (wtype == kWInt16) {
        prefer_shared<recompute_kernel<kWInt16>>();
        recompute_kernel<kWInt16><<<grid, kWarps * 32, 0, st>>>(W, diag, N, ldw, S, xs, nw, R, hout, npad, part);
    } else {
        prefer_shared<recompute_kernel<kWFp32>>();
        recompute_kernel<kWFp32><<<grid, kWarps * 32, 0, st>>>(W, diag, N, ldw, S, xs, nw, R, hout, npad, part);
    }
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess || !E) return err;
    return launch_energy_sum(wtype != kWFp32, scratch, tiles, R, S, E, Estride, st);
}

cudaError_t launch_recompute(bool is_int8, const void* W, const void* diag, int N, int ldw, int S,
                             const uint32_t* xs, int nw, int R, void* hout, int npad,
                             long long* E, int Estride, cudaStream_t st, long long* scratch)
{
    return launch_recompute_w(is_int8 ? kWInt8 : kWFp32, W, diag, N, ldw, S, xs, nw, R, hout, npad, E, Estride, st,
                              scratch);
}

}  // namespace da
