// da_mma.cu -- the exact field recompute on the tensor cores (tcgen05).
//
// The recompute g = diag + W x of R states is a dense contraction
// G[r][i] = sum_j X[r][j] W[j][i] with X in {0, 1}: the states are the M side
// (128 per tile, one per TMEM lane), the variables i the N side (64 per tile)
// and the couplings j the K side.  Its value is defined exactly (da_fields.cu):
// every coupling is put on the fixed-point grid, v_ij = round(W_ij 2^S) (the
// int8 couplings themselves), and summed in integers.  The tensor cores reach
// the same integers: v is split into balanced digits of b bits,
//   v = sum_l d_l 2^(b l),   d_l in [-2^(b-1), 2^(b-1)),
// every digit is exact in fp16 (|d| <= 2048), and b is chosen so that no
// partial sum of digits over the K side exceeds 2^21 in magnitude, far inside
// the 24-bit integer range of the fp32 accumulator.  Each digit plane is one
// accumulator in tensor memory; the epilogue combines the planes in 64-bit
// integers, adds the fixed-point diagonal and rounds once, exactly like the
// CUDA-core form.
//
// Operands use the tensor core's canonical K-major layout (8-row x 16-byte
// core matrices, [K chunk][row group][8][8] halves per tile).  The digit planes
// of the instance are built once per context in that layout in HBM, so a
// pipeline stage takes them in one contiguous bulk copy; the states are not
// staged in HBM at all: two warps of the block expand the tile's state bits
// (2 words per state and stage) to f16 {0, 1} directly into the stage.
//
// Block: 16 warps, 128 states x 64 variables.  Warp 0 allocates tensor memory
// and one of its threads issues the digit planes' bulk copies into a 3-stage
// ring; warps 2-3 write the stage's state tile (the words of the next chunk
// loaded while the current one is written); one thread of warp 1 issues the
// MMAs (4 K-steps of 16 per stage, one per digit plane each) and commits the
// stage back to both producers; then all 16 warps read their TMEM lanes (warp
// w: states 32 (w % 4).., 16 variables from 16 (w / 4)) and write fields and
// 128-bit partial energies.  (32-variable tiles, two blocks an SM, measured
// slower: every block expands its states again, and at 6 digit planes only one
// block fits.)
#include <cuda_fp16.h>

#include <algorithm>
#include <mutex>
#include <set>
#include <utility>

#include "da_fixed.cuh"
#include "da_internal.h"
#include "da_tc.cuh"

namespace da {
namespace {

constexpr int kBM = 128;   // states per tile (TMEM lanes)
constexpr int kBN = 64;    // variables per tile (TMEM columns per digit plane)
constexpr int kBK = 64;    // couplings per pipeline stage
constexpr int kStages = 3;
constexpr int kThreads = 128 * (kBN / 16);   // warp w reads TMEM lanes 32 (w % 4).., columns 16 (w / 4)..
constexpr int kMinBlocks = 512 / kThreads;   // blocks per SM the launch bounds plan for
constexpr int kExpanders = 64;  // threads of warps 2-3: the state tile of each stage, 2 states each
constexpr uint32_t kATile = kBM * kBK * 2;   // bytes of one state tile (16 KB)
constexpr uint32_t kBTile = kBN * kBK * 2;   // bytes of one digit-plane tile (8 KB)
constexpr uint32_t kWaitLimit = 1u << 26;    // polls of one mbarrier before giving up ...
constexpr uint64_t kWaitNs = 2000000000ull;  // ... or 2 s, whichever comes first
constexpr int kMaxLimbs = 6;                 // digit planes for any N <= 8192 (tc_digits)

// Offset (in halves) of element (row, k) inside a tile of `rows` x 64 halves
// in the canonical K-major layout without swizzling.
__device__ __forceinline__ size_t core_offset(int rows, int row, int k)
{
    return (size_t)((k >> 3) * (rows >> 3) + (row >> 3)) * 64 + (row & 7) * 8 + (k & 7);
}

template <typename Tw>
__device__ __forceinline__ long long fixed_w(const void* W, size_t idx, int S)
{
    if constexpr (sizeof(Tw) == 4) return fixed_of_f32(static_cast<const float*>(W)[idx], S);
    else return (long long)static_cast<const Tw*>(W)[idx];   // integer couplings are their own grid
}

template <bool INT8>
__device__ __forceinline__ long long fixed_d(const void* diag, int i, int S)
{
    if constexpr (INT8) return (long long)static_cast<const int32_t*>(diag)[i];
    else return fixed_of_f32(static_cast<const float*>(diag)[i], S);
}

// The diagonal on the fixed-point grid, zero-padded to n entries.
template <bool INT8>
__global__ void build_dfix_kernel(const void* __restrict__ diag, int N, int S, long long* __restrict__ dfix, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dfix[i] = i < N ? fixed_d<INT8>(diag, i, S) : 0ll;
}

// Digit planes: one thread per (tile i, chunk j, row i, group of 8 j).
template <typename Tw>
__global__ void build_digits_kernel(const void* __restrict__ W, int N, int ldw, int S, int bits, int limbs,
                                    int kchunks, __half* __restrict__ B, long long total)
{
    const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= total) return;
    const int g = (int)(idx & 7);
    const int row = (int)((idx >> 3) % kBN);
    const long long tile = idx / (8 * kBN);    // itile * kchunks + kchunk
    const int kchunk = (int)(tile % kchunks);
    const int itile = (int)(tile / kchunks);
    const int i = itile * kBN + row;
    const int jb = kchunk * kBK + g * 8;
    long long v[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
        const int j = jb + e;
        v[e] = (i < N && j < N) ? fixed_w<Tw>(W, (size_t)j * ldw + i, S) : 0ll;
    }
    const long long half_range = 1ll << (bits - 1);
    const long long mask = (1ll << bits) - 1;
    for (int l = 0; l < limbs; ++l) {
        __align__(16) __half h[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            long long d = v[e] & mask;
            if (d >= half_range) d -= mask + 1;
            v[e] = (v[e] - d) >> bits;
            h[e] = __int2half_rn((int)d);
        }
        __half* dst = B + ((size_t)tile * limbs + l) * (kBN * kBK) + core_offset(kBN, row, g * 8);
        *reinterpret_cast<uint4*>(dst) = *reinterpret_cast<const uint4*>(h);
    }
}

// Two f16 values {0, 1} from two state bits (bit 0 -> the lower half).
__device__ __forceinline__ uint32_t half_pair(uint32_t two)
{
    return (two & 1u) * 0x3C00u + (two >> 1) * 0x3C000000u;   // f16 1.0 = 0x3C00
}

// Makes this thread's shared-memory writes visible to the asynchronous proxy
// (the tensor cores' operand reads).
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

struct I128 {
    unsigned long long lo;
    long long hi;
};

__device__ __forceinline__ void i128_add(I128& a, long long v)
{
    const unsigned long long lo = a.lo + (unsigned long long)v;
    a.hi += (v < 0 ? -1ll : 0ll) + (lo < a.lo ? 1ll : 0ll);
    a.lo = lo;
}

struct TcParams {
    const __half* B;        // [ceil(N/64)][kchunks][limbs] digit-plane tiles
    const long long* dfix;  // [kchunks * 64] fixed-point diagonal, zero-padded
    const uint32_t* xs;     // [R][nw] state bits (x_i = bit i % 32 of word i / 32)
    void* hout;             // [R][npad] or null
    I128* part;             // [gridDim.x][R] or null
    int* err;
    int N, S, bits, limbs, kchunks, nw, R, npad;
    uint32_t ncols;         // tensor-memory columns allocated
};

template <bool INT8>
__device__ __forceinline__ uint32_t field_bits(long long acc, int S)
{
    if constexpr (INT8) return (uint32_t)(int32_t)acc;
    else return __float_as_uint(scaled_f32_of(acc, S));
}

template <bool INT8>
__global__ void __launch_bounds__(kThreads, kMinBlocks) recompute_tc_kernel(const __grid_constant__ TcParams p)
{
    extern __shared__ uint8_t smem_raw[];
    __shared__ int s_fail;
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int i0 = blockIdx.x * kBN;
    const int m = (warp & 3) * 32 + lane;           // TMEM lane = state of the tile
    const int cg = warp >> 2;                       // 16-column group of the epilogue
    const int r = blockIdx.y * kBM + m;

    if (i0 >= p.N) {   // padding beyond N (whole block): zero fields and partial sums
        if (cg == 0 && r < p.R) {
            if (p.hout)
                for (int e = 0; e < kBN; ++e)
                    if (i0 + e < p.npad) static_cast<uint32_t*>(p.hout)[(size_t)r * p.npad + i0 + e] = 0u;
            if (p.part) p.part[(size_t)blockIdx.x * p.R + r] = I128{0ull, 0ll};
        }
        return;
    }

    const uint32_t stage_bytes = kATile + (uint32_t)p.limbs * kBTile;
    uint8_t* sm = smem_raw + ((1024u - (tc::smem_u32(smem_raw) & 1023u)) & 1023u);
    uint64_t* full = reinterpret_cast<uint64_t*>(sm + kStages * stage_bytes);
    uint64_t* empty = full + kStages;
    uint64_t* done = empty + kStages;
    uint32_t* tslot = reinterpret_cast<uint32_t*>(done + 1);

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            tc::mbar_init(&full[s], 1 + kExpanders);   // the copier's expect_tx and every expander
            tc::mbar_init(&empty[s], 1);
        }
        tc::mbar_init(done, 1);
        tc::mbar_init_fence();
        s_fail = 0;
    }
    if (warp == 0) {
        tc::tmem_alloc(tslot, p.ncols);
        tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tbase = *tslot;
    const int nk = p.kchunks;

    if (warp == 0) {
        if (lane == 0) {   // bulk-copy issuer: the digit planes of each stage
            const __half* b_src = p.B + (size_t)blockIdx.x * nk * p.limbs * (kBN * kBK);
            const uint32_t b_bytes = (uint32_t)p.limbs * kBTile;
            for (int c = 0; c < nk; ++c) {
                const int s = c % kStages;
                const uint32_t u = (uint32_t)(c / kStages);
                if (u > 0 && !tc::mbar_wait(&empty[s], (u - 1) & 1u, kWaitLimit, kWaitNs)) {
                    s_fail = 1;
                    break;
                }
                uint8_t* st = sm + s * stage_bytes;
                tc::mbar_arrive_expect_tx(&full[s], b_bytes);
                tc::bulk_g2s(st + kATile, b_src + (size_t)c * p.limbs * (kBN * kBK), b_bytes, &full[s]);
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0) {   // MMA issuer
            constexpr uint32_t idesc = tc::idesc_f16_f32(kBM, kBN);
            for (int c = 0; c < nk; ++c) {
                const int s = c % kStages;
                const uint32_t u = (uint32_t)(c / kStages);
                if (!tc::mbar_wait(&full[s], u & 1u, kWaitLimit, kWaitNs)) {
                    s_fail = 1;
                    break;
                }
                tc::fence_after_sync();
                const uint32_t a0 = tc::smem_u32(sm + s * stage_bytes);
                const uint32_t b0 = a0 + kATile;
#pragma unroll
                for (int q = 0; q < kBK / 16; ++q) {
                    // K-step q covers core-matrix columns 2q, 2q + 1 of the stage
                    const uint64_t ad = tc::smem_desc(a0 + q * 2 * (kBM / 8) * 128, (kBM / 8) * 128, 128);
                    for (int l = 0; l < p.limbs; ++l) {
                        const uint64_t bd =
                            tc::smem_desc(b0 + l * kBTile + q * 2 * (kBN / 8) * 128, (kBN / 8) * 128, 128);
                        tc::mma_f16(tbase + (uint32_t)(l * kBN), ad, bd, idesc, (c > 0 || q > 0) ? 1u : 0u);
                    }
                }
                tc::mma_commit(&empty[s]);
            }
            tc::mma_commit(done);
        }
        __syncwarp();
    } else if (warp == 2 || warp == 3) {
        // the stage's state tile: thread e writes states e and e + 64 of the tile, 64
        // couplings each (2 state words) as eight 16-byte rows of f16 {0, 1} in the
        // canonical K-major layout; bits beyond N and states beyond R are 0
        const int e = (int)threadIdx.x - 64;
        // the two states' words of chunk c: loaded one chunk ahead, so that their latency
        // overlaps the wait for the stage and the writes of the chunk before
        auto load = [&](int c, uint32_t (&wv)[4]) {
            const int w0 = (c * kBK) >> 5;               // < nw: c < kchunks = ceil(N / 64)
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {
                const int r = blockIdx.y * kBM + e + 64 * hh;
                const uint32_t* xr = p.xs + (size_t)r * p.nw;
                wv[2 * hh] = r < p.R ? xr[w0] : 0u;
                wv[2 * hh + 1] = r < p.R && w0 + 1 < p.nw ? xr[w0 + 1] : 0u;
            }
        };
        uint32_t cur[4], nxt[4] = {0u, 0u, 0u, 0u};
        load(0, cur);
        for (int c = 0; c < nk; ++c) {
            const int s = c % kStages;
            const uint32_t u = (uint32_t)(c / kStages);
            if (c + 1 < nk) load(c + 1, nxt);
            if (u > 0 && !tc::mbar_wait(&empty[s], (u - 1) & 1u, kWaitLimit, kWaitNs)) {
                s_fail = 1;
                break;
            }
            uint8_t* st = sm + s * stage_bytes;
            const int nvalid = min(kBK, p.N - c * kBK);
            const uint64_t vmask = nvalid >= 64 ? ~0ull : ((1ull << nvalid) - 1ull);
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {
                const int row = e + 64 * hh;
                const uint64_t bits = (((uint64_t)cur[2 * hh + 1] << 32) | cur[2 * hh]) & vmask;
#pragma unroll
                for (int kc = 0; kc < 8; ++kc) {
                    const uint32_t b = (uint32_t)(bits >> (8 * kc)) & 0xFFu;
                    const uint4 v = make_uint4(half_pair(b & 3u), half_pair((b >> 2) & 3u), half_pair((b >> 4) & 3u),
                                               half_pair(b >> 6));
                    *reinterpret_cast<uint4*>(st + 2 * core_offset(kBM, row, kc * 8)) = v;
                }
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) cur[q] = nxt[q];
            fence_proxy_async_smem();
            tc::mbar_arrive(&full[s]);
        }
    }

    // epilogue: state r = TMEM lane m, variables i0 + 16 cg .. + 15
    if (!tc::mbar_wait(done, 0, kWaitLimit, kWaitNs)) s_fail = 1;
    __syncwarp();
    tc::fence_after_sync();
    const uint32_t lane_addr = tbase + ((uint32_t)((warp & 3) * 32) << 16);
    I128 esum{0ull, 0ll};
    const bool live = r < p.R;
    const bool vec = (p.npad & 3) == 0;
    uint32_t* hrow = p.hout ? static_cast<uint32_t*>(p.hout) + (size_t)r * p.npad : nullptr;
    {
        const int ib = i0 + cg * 16;
        long long acc[16];
#pragma unroll
        for (int e = 0; e < 16; e += 2) {
            const longlong2 d2 = *reinterpret_cast<const longlong2*>(p.dfix + ib + e);
            acc[e] = d2.x;
            acc[e + 1] = d2.y;
        }
        for (int l = 0; l < p.limbs; ++l) {
            uint32_t v[16];
            tc::tmem_ld16(lane_addr + (uint32_t)(l * kBN + cg * 16), v);
            const int sh = p.bits * l;
#pragma unroll
            for (int e = 0; e < 16; ++e)
                acc[e] = (long long)((unsigned long long)acc[e] +
                                     ((unsigned long long)(long long)small_int_of(__uint_as_float(v[e])) << sh));
        }
        if (live) {
            if (hrow) {
                uint32_t hb[16];
#pragma unroll
                for (int e = 0; e < 16; ++e) hb[e] = field_bits<INT8>(acc[e], p.S);  // 0 for i >= N
                if (vec && ib + 16 <= p.npad) {
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        *reinterpret_cast<uint4*>(hrow + ib + 4 * q) =
                            make_uint4(hb[4 * q], hb[4 * q + 1], hb[4 * q + 2], hb[4 * q + 3]);
                } else {
#pragma unroll
                    for (int e = 0; e < 16; ++e)
                        if (ib + e < p.npad) hrow[ib + e] = hb[e];
                }
            }
            if (p.part && ib < p.N) {
                const uint32_t xw = (p.xs[(size_t)r * p.nw + (ib >> 5)] >> (ib & 31)) & 0xFFFFu;
#pragma unroll
                for (int e = 0; e < 16; ++e)
                    if ((xw >> e) & 1u) i128_add(esum, p.dfix[ib + e] + acc[e]);
            }
        }
    }
    // partial energies of the 2 column groups, in the first stage's memory: every bulk
    // copy has landed and every MMA has read its operands once `done` has completed
    I128 (*s_part)[kBM] = reinterpret_cast<I128 (*)[kBM]>(sm);
    s_part[cg][m] = esum;

    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tbase, p.ncols);
    }
    if (threadIdx.x < kBM && p.part && blockIdx.y * kBM + threadIdx.x < p.R) {
        I128 t = s_part[0][threadIdx.x];
#pragma unroll
        for (int g = 1; g < kThreads / kBM; ++g) {
            const I128 u = s_part[g][threadIdx.x];
            const unsigned long long lo = t.lo + u.lo;
            t.hi += u.hi + (lo < t.lo ? 1ll : 0ll);
            t.lo = lo;
        }
        p.part[(size_t)blockIdx.x * p.R + blockIdx.y * kBM + threadIdx.x] = t;
    }
    if (threadIdx.x == 0 && s_fail) atomicExch(p.err, 1);
}

size_t smem_bytes(int limbs) { return 1024 + (size_t)kStages * (kATile + (size_t)limbs * kBTile) + 8 * (2 * kStages + 1) + 16; }

int ceil_log2(long long n)
{
    int L = 0;
    while ((1ll << L) < n) ++L;
    return L;
}

}  // namespace

void tc_digits(int wtype, int N, int* bits, int* limbs)
{
    if (wtype == kWInt8) {   // the couplings are balanced 8-bit digits already
        *bits = 8;
        *limbs = 1;
        return;
    }
    // |partial sum| <= 2^(b-1) * N <= 2^21
    const int b = std::min(12, 22 - ceil_log2(std::max(N, 2)));
    *bits = b;
    if (wtype == kWInt16) {  // |v| <= 2^15 - 1 needs b * limbs >= 17
        *limbs = (17 + b - 1) / b;
        return;
    }
    // |v| <= 2^(62 - L), 2^L >= N + 1
    const int L = ceil_log2((long long)N + 1);
    *limbs = (64 - L + b - 1) / b;
}

size_t tc_partial_bytes(int rows, int R)
{
    return (size_t)16 * (size_t)((rows + kBN - 1) / kBN) * (size_t)R;
}

// Bytes of the operand's three parts: digit planes, fixed-point diagonal, error flag.
static void tc_operand_parts(int wtype, int N, size_t* b_bytes, size_t* d_bytes)
{
    int bits = 0, limbs = 0;
    tc_digits(wtype, N, &bits, &limbs);
    const size_t kchunks = (size_t)(N + kBK - 1) / kBK;
    const size_t itiles = (size_t)(N + kBN - 1) / kBN;
    *b_bytes = itiles * kchunks * (size_t)limbs * kBTile;
    *d_bytes = kchunks * kBK * sizeof(long long);
}

size_t tc_operand_bytes(int wtype, int N)
{
    size_t b = 0, d = 0;
    tc_operand_parts(wtype, N, &b, &d);
    return (b + 255) / 256 * 256 + (d + 255) / 256 * 256 + 256;
}

static cudaError_t tc_operand_fill(int wtype, const void* W, const void* diag, int N, int ldw, int S, TcOperand* op,
                                   cudaStream_t st);

cudaError_t tc_operand_build_in(int wtype, const void* W, const void* diag, int N, int ldw, int S, void* mem,
                                TcOperand* op, cudaStream_t st)
{
    size_t b = 0, d = 0;
    tc_operand_parts(wtype, N, &b, &d);
    char* m = static_cast<char*>(mem);
    op->B = m;
    op->dfix = reinterpret_cast<long long*>(m + (b + 255) / 256 * 256);
    op->err = reinterpret_cast<int*>(m + (b + 255) / 256 * 256 + (d + 255) / 256 * 256);
    return tc_operand_fill(wtype, W, diag, N, ldw, S, op, st);
}

cudaError_t tc_operand_build(int wtype, const void* W, const void* diag, int N, int ldw, int S, TcOperand* op,
                             cudaStream_t st)
{
    size_t b = 0, d = 0;
    tc_operand_parts(wtype, N, &b, &d);
    cudaError_t e = dev_malloc(&op->B, b);
    if (e == cudaSuccess) e = dev_malloc(reinterpret_cast<void**>(&op->err), sizeof(int));
    if (e == cudaSuccess) e = dev_malloc(reinterpret_cast<void**>(&op->dfix), d);
    if (e != cudaSuccess) return e;
    return tc_operand_fill(wtype, W, diag, N, ldw, S, op, st);
}

// The digit planes and diagonal of W into op's buffers, and the error flag cleared.
static cudaError_t tc_operand_fill(int wtype, const void* W, const void* diag, int N, int ldw, int S, TcOperand* op,
                                   cudaStream_t st)
{
    tc_digits(wtype, N, &op->bits, &op->limbs);
    op->kchunks = (N + kBK - 1) / kBK;
    const int itiles = (N + kBN - 1) / kBN;
    cudaError_t e;
    e = cudaMemsetAsync(op->err, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    const long long total = (long long)itiles * op->kchunks * kBN * 8;
    const int tb = 256;
    const unsigned blocks = (unsigned)((total + tb - 1) / tb);
    const int nd = op->kchunks * kBK;
    __half* B = static_cast<__half*>(op->B);
    // the request loop builds operands beside running kernels: the carveout of the rest of its kernels
    prefer_shared<build_digits_kernel<int8_t>>();
    prefer_shared<build_digits_kernel<int16_t>>();
    prefer_shared<build_digits_kernel<float>>();
    prefer_shared<build_dfix_kernel<false>>();
    prefer_shared<build_dfix_kernel<true>>();
    if (wtype == kWInt8)
        build_digits_kernel<int8_t><<<blocks, tb, 0, st>>>(W, N, ldw, S, op->bits, op->limbs, op->kchunks, B, total);
    else if (wtype == kWInt16)
        build_digits_kernel<int16_t><<<blocks, tb, 0, st>>>(W, N, ldw, S, op->bits, op->limbs, op->kchunks, B, total);
    else
        build_digits_kernel<float><<<blocks, tb, 0, st>>>(W, N, ldw, S, op->bits, op->limbs, op->kchunks, B, total);
    if (wtype == kWFp32)
        build_dfix_kernel<false><<<(nd + tb - 1) / tb, tb, 0, st>>>(diag, N, S, op->dfix, nd);
    else
        build_dfix_kernel<true><<<(nd + tb - 1) / tb, tb, 0, st>>>(diag, N, S, op->dfix, nd);
    return cudaGetLastError();
}

void tc_operand_free(TcOperand* op)
{
    if (op->B) dev_free(op->B);
    if (op->err) dev_free(op->err);
    if (op->dfix) dev_free(op->dfix);
    *op = TcOperand{};
}

cudaError_t prepare_tc_kernels()
{
    prefer_shared<build_digits_kernel<int8_t>>();
    prefer_shared<build_digits_kernel<int16_t>>();
    prefer_shared<build_digits_kernel<float>>();
    prefer_shared<build_dfix_kernel<false>>();
    prefer_shared<build_dfix_kernel<true>>();
    prefer_shared<recompute_tc_kernel<false>>();
    prefer_shared<recompute_tc_kernel<true>>();
    cudaError_t e = cudaFuncSetAttribute(recompute_tc_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem_bytes(kMaxLimbs));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(recompute_tc_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem_bytes(2));
    return e;
}

cudaError_t launch_recompute_tc(bool is_int8, const TcOperand& op, const void* diag, int N, int S,
                                const uint32_t* xs, int nw, int R, void* hout, int npad, long long* E, int Estride,
                                cudaStream_t st, long long* scratch)
{
    if (R <= 0) return cudaSuccess;
    // the dynamic shared-memory limit of each kernel form, set once per device
    static std::mutex attr_mu;
    static std::set<std::pair<int, int>> attr_done;
    int dev = 0;
    cudaGetDevice(&dev);
    const size_t smem = smem_bytes(op.limbs);
    const int max_limbs = is_int8 ? 2 : kMaxLimbs;   // integer couplings: 1 (int8) or 2 (int16) planes
    if (op.limbs < 1 || op.limbs > max_limbs) return cudaErrorInvalidValue;
    {
        std::lock_guard<std::mutex> lock(attr_mu);
        if (!attr_done.count({is_int8 ? 1 : 0, dev})) {
            const int bytes = (int)smem_bytes(max_limbs);
            cudaError_t e = is_int8 ? cudaFuncSetAttribute(recompute_tc_kernel<true>,
                                                           cudaFuncAttributeMaxDynamicSharedMemorySize, bytes)
                                    : cudaFuncSetAttribute(recompute_tc_kernel<false>,
                                                           cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
            if (e != cudaSuccess) return e;
            attr_done.insert({is_int8 ? 1 : 0, dev});
        }
    }

    const int rtiles = (R + kBM - 1) / kBM;
    const int rows = hout ? std::max(npad, N) : N;
    const int itiles = (rows + kBN - 1) / kBN;
    TcParams p;
    p.B = static_cast<const __half*>(op.B);
    p.dfix = op.dfix;
    p.xs = xs;
    p.hout = hout;
    p.part = E ? reinterpret_cast<I128*>(scratch) : nullptr;
    p.err = op.err;
    p.N = N;
    p.S = S;
    p.bits = op.bits;
    p.limbs = op.limbs;
    p.kchunks = op.kchunks;
    p.nw = nw;
    p.R = R;
    p.npad = npad;
    uint32_t nc = 32;
    while (nc < (uint32_t)(op.limbs * kBN)) nc <<= 1;
    p.ncols = nc;
    dim3 grid(itiles, rtiles);
    if (is_int8)
        recompute_tc_kernel<true><<<grid, kThreads, smem, st>>>(p);
    else
        recompute_tc_kernel<false><<<grid, kThreads, smem, st>>>(p);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || !E) return e;
    return launch_energy_sum(is_int8, scratch, itiles, R, S, E, Estride, st);
}

}  // namespace da
