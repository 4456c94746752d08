// da_step.cuh -- the Digital Annealer's parallel-trial Monte Carlo step
// (Algorithm 2 of arXiv:1806.08815) for many replicas at once.
//
// One group of G warps anneals one replica.  Lane l of warp w owns the V
// consecutive variables i = w*32V + l*V + v (v < V) and keeps their effective
// fields g_i = Q_ii + sum_j W_ij x_j and bits x_i in registers for the whole
// launch.  Per step:
//   (a) every lane forms Delta E_i = (1 - 2 x_i) g_i for its V variables (all
//       N trials of the step run in parallel, Sec. II);
//   (b) Metropolis against the dynamic offset: delta = Delta E - E_off is
//       accepted when delta <= 0, else when u < exp(-beta delta).  u comes from
//       Philox block (i/4, t, replica, 0); the test is decided against a band
//       around a hardware estimate of exp and falls back to the exact
//       exponential only inside the band, so every decision equals the exact
//       one;
//   (c) each lane's acceptance bits are already in index order, so a warp
//       prefix sum of their popcounts locates the j-th accepted variable,
//       j = floor(u * count); the chosen x_k flips while every lane adds
//       +-W[k][i] (16-byte loads of row k, which equals column k, from L2) to
//       its fields.  The next step's Philox words are computed while that row
//       is in flight.  E_off returns to 0 on a flip and grows by inc otherwise.
// A G = 1 group needs no shared memory or barrier.  A G > 1 group publishes
// its lanes' acceptance and state masks in shared memory behind one named
// barrier per step; the energy of step t is booked after the barrier of step
// t + 1, while x still holds the state right after step t.
//
// Launches cover steps [t0, t1) and keep the state in global memory between
// launches (the fp32 path recomputes the fields between launches).
#pragma once
#include "da_device.cuh"
#include "da_internal.h"

namespace da {
namespace step_detail {

template <typename Tw> struct Arith;
template <> struct Arith<int8_t> {
    using H = int32_t;    // effective fields
    using E = long long;  // tracked energy
    static __device__ __forceinline__ H signed_field(H g, uint32_t x) { return x ? -g : g; }
    static __device__ __forceinline__ float delta(H dE, float Eoff) { return __fsub_rn(__int2float_rn(dE), Eoff); }
    static __device__ __forceinline__ H apply(H h, int8_t w, bool minus) { return minus ? h - (H)w : h + (H)w; }
    static __device__ __forceinline__ E load_e(long long b) { return b; }
    static __device__ __forceinline__ long long store_e(E e) { return e; }
    static __device__ __forceinline__ E book(E e, H dE) { return e + (E)dE; }
};
template <> struct Arith<float> {
    using H = float;
    using E = double;
    static __device__ __forceinline__ H signed_field(H g, uint32_t x)
    {
        return __int_as_float(__float_as_int(g) ^ (int)(x << 31));
    }
    static __device__ __forceinline__ float delta(H dE, float Eoff) { return __fsub_rn(dE, Eoff); }
    static __device__ __forceinline__ H apply(H h, float w, bool minus) { return minus ? __fsub_rn(h, w) : __fadd_rn(h, w); }
    static __device__ __forceinline__ E load_e(long long b) { return __longlong_as_double(b); }
    static __device__ __forceinline__ long long store_e(E e) { return __double_as_longlong(e); }
    static __device__ __forceinline__ E book(E e, H dE) { return __dadd_rn(e, (double)dE); }
};

__device__ __forceinline__ int warp_inclusive_scan(int v, int lane)
{
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int n = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += n;
    }
    return v;
}

// Position of the r-th (0-based) set bit of w; requires r < popc(w).
__device__ __forceinline__ int nth_set_bit(uint32_t w, int r)
{
    int pos = 0, c;
    c = __popc(w & 0xFFFFu); if (r >= c) { r -= c; pos += 16; w >>= 16; }
    c = __popc(w & 0xFFu);   if (r >= c) { r -= c; pos += 8;  w >>= 8; }
    c = __popc(w & 0xFu);    if (r >= c) { r -= c; pos += 4;  w >>= 4; }
    c = __popc(w & 0x3u);    if (r >= c) { r -= c; pos += 2;  w >>= 2; }
    c = (int)(w & 1u);       if (r >= c) { pos += 1; }
    return pos;
}

__device__ __forceinline__ void group_barrier(int id, int nthreads)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// Row k of W at the V consecutive entries of this lane (16-byte loads where
// the lane's slice allows).
template <typename Tw, int V> struct Row;
template <int V> struct Row<float, V> {
    static __device__ __forceinline__ void load(const float* p, float (&c)[V])
    {
        static_assert(V % 4 == 0, "V");
#pragma unroll
        for (int q = 0; q < V / 4; ++q) {
            const float4 f = __ldg(reinterpret_cast<const float4*>(p) + q);
            c[4 * q] = f.x; c[4 * q + 1] = f.y; c[4 * q + 2] = f.z; c[4 * q + 3] = f.w;
        }
    }
};
template <int V> struct Row<int8_t, V> {
    static __device__ __forceinline__ void unpack(uint32_t u, int8_t* c)
    {
        c[0] = (int8_t)(u & 0xFFu); c[1] = (int8_t)((u >> 8) & 0xFFu);
        c[2] = (int8_t)((u >> 16) & 0xFFu); c[3] = (int8_t)(u >> 24);
    }
    static __device__ __forceinline__ void load(const int8_t* p, int8_t (&c)[V])
    {
        if constexpr (V == 4) {
            unpack(__ldg(reinterpret_cast<const unsigned int*>(p)), c);
        } else if constexpr (V == 8) {
            const uint2 u = __ldg(reinterpret_cast<const uint2*>(p));
            unpack(u.x, c); unpack(u.y, c + 4);
        } else {
#pragma unroll
            for (int q = 0; q < V / 16; ++q) {
                const uint4 u = __ldg(reinterpret_cast<const uint4*>(p) + q);
                unpack(u.x, c + 16 * q); unpack(u.y, c + 16 * q + 4);
                unpack(u.z, c + 16 * q + 8); unpack(u.w, c + 16 * q + 12);
            }
        }
    }
};

// Replicas per block and the blocks per SM the register budget is sized for:
// at least 7 replicas per SM, so that 1024 replicas fill 152 SMs in one wave.
template <int G> struct Occupancy;
template <> struct Occupancy<1> { static constexpr int rpb = 4, min_blocks = 2; };
template <> struct Occupancy<2> { static constexpr int rpb = 2, min_blocks = 4; };
template <> struct Occupancy<4> { static constexpr int rpb = 1, min_blocks = 7; };
template <> struct Occupancy<8> { static constexpr int rpb = 1, min_blocks = 2; };

// The state words of a replica are standard bit-packed words (x_i is bit i%32
// of word i/32); a lane's V bits are one slice of word (w*32V + l*V) / 32.
template <int V>
__device__ __forceinline__ uint32_t gather_word(uint32_t bits, int lane)
{
    constexpr int P = 32 / V;  // lanes per word
    uint32_t m = (V == 32) ? bits : (bits << ((lane % P) * V));
#pragma unroll
    for (int o = 1; o < P; o <<= 1) m |= __shfl_xor_sync(0xffffffffu, m, o);
    return m;
}

template <typename Tw, int V, int G, bool FULL, bool TRACE>
__global__ void __launch_bounds__(32 * G * Occupancy<G>::rpb, Occupancy<G>::min_blocks)
    step_kernel(const __grid_constant__ StepParams p)
{
    using A = Arith<Tw>;
    using H = typename A::H;
    using E = typename A::E;
    static_assert(V % 4 == 0 && V <= 32, "V must be 4, 8, 16 or 32");
    constexpr int NQ = V / 4;                       // Philox blocks per lane per step
    constexpr uint32_t VMASK = V == 32 ? 0xffffffffu : ((1u << V) - 1u);
    constexpr int P = 32 / V;                       // lanes per state word

    extern __shared__ uint32_t smem[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int g = wib / G;                          // group (replica) within the block
    const int w = wib - g * G;                      // warp within the group
    const int rpb = blockDim.x / (32 * G);
    const int r = blockIdx.x * rpb + g;
    if (r >= p.R) return;

    uint32_t* gs = smem + g * (4 * 32 * G + 4);
    uint32_t* accs = gs;                            // [2][32G] lane acceptance masks
    uint32_t* xss = gs + 2 * 32 * G;                // [2][32G] lane state masks
    H* pub = reinterpret_cast<H*>(gs + 4 * 32 * G); // [2] Delta E of the flipped variable

    const Tw* __restrict__ Wm = static_cast<const Tw*>(p.W);
    const int base = w * 32 * V + lane * V;         // first variable of this lane
    H* hg = static_cast<H*>(p.h) + (size_t)r * p.npad + base;
    uint32_t* xg = p.x + (size_t)r * p.nw;
    uint32_t* bestg = p.bestx + (size_t)r * p.nw;
    const int word_of_lane = base >> 5;

    H h[V];
#pragma unroll
    for (int v = 0; v < V; ++v) h[v] = hg[v];
    uint32_t xm = (xg[word_of_lane] >> (base & 31)) & VMASK;
    uint32_t valid = VMASK;
    if constexpr (!FULL) valid = base >= p.N ? 0u : (p.N - base >= V ? VMASK : ((1u << (p.N - base)) - 1u));

    ReplicaScalars sc = p.sc[r];
    E Ecur = A::load_e(sc.E), Ebest = A::load_e(sc.best);
    long long flips = sc.flips;
    uint32_t m = sc.m;
    const uint32_t rep = p.rep_base + (uint32_t)r;
    const PhiloxKeys& keys = *reinterpret_cast<const PhiloxKeys*>(&p.round_key[0][0]);
    const bool per_rep = p.betas != nullptr;
    const float beta_rep = per_rep ? p.betas[p.temp_of[r]] : 0.f;
    u32x4 cr = {0, 0, 0, 0};
    long long cr_blk = -1;
    bool pending = false;

    auto snapshot = [&]() {
        const uint32_t word = gather_word<V>(xm, lane);
        if (lane % P == 0) bestg[word_of_lane] = word;
    };
    // Acceptance draws of one step: block q covers variables base + 4q .. + 3.
    auto draw_step = [&](u32x4 (&rr)[NQ], uint32_t tt) {
#pragma unroll
        for (int q = 0; q < NQ; ++q) rr[q] = philox4x32_10((uint32_t)(base >> 2) + q, tt, rep, 0u, keys);
    };
    u32x4 rr[NQ];
    if (p.t0 < p.t1) draw_step(rr, (uint32_t)p.t0);

    float beta_next = (!per_rep && p.t0 < p.t1) ? p.beta[p.t0] : beta_rep;
    for (long long t = p.t0; t < p.t1; ++t) {
        const float beta = beta_next;
        if (!per_rep && t + 1 < p.t1) beta_next = p.beta[t + 1];
        const float Eoff = __fmul_rn(__uint2float_rn(m), p.inc);

        // (a) + (b): every trial of this lane, branch-free except for the rare
        // draws that fall inside the band of the exp estimate.
        uint32_t accm = 0, band = 0;
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const H dE = A::signed_field(h[v], (xm >> v) & 1u);
            const float delta = A::delta(dE, Eoff);
            const float ax = -__fmul_rn(beta, delta);
            const uint32_t wd = pick(rr[v >> 2], v & 3);
            const float est = exp_estimate(ax);
            const float U = __uint2float_rn((wd >> 8) + 1u);
            const bool le0 = delta <= 0.0f;
            const bool need = !le0 && ax > kExpCut;
            const bool sure = U < __fmul_rn(est, kBandLo);
            const bool maybe = U < __fmul_rn(est, kBandHi);
            accm |= (uint32_t)(le0 || (need && sure)) << v;
            band |= (uint32_t)(need && !sure && maybe) << v;
        }
        if (__any_sync(0xffffffffu, band != 0u)) {
#pragma unroll
            for (int v = 0; v < V; ++v) {
                if ((band >> v) & 1u) {
                    const float delta = A::delta(A::signed_field(h[v], (xm >> v) & 1u), Eoff);
                    const float ax = -__fmul_rn(beta, delta);
                    const float u = uniform01(pick(rr[v >> 2], v & 3));
                    accm |= (uint32_t)(u < exp_neg(ax)) << v;
                }
            }
        }
        if constexpr (!FULL) accm &= valid;

        // (c) uniform choice among the accepted trials
        int k = -1, own_lane = 0, own_warp = 0, vk = 0;
        uint32_t xold = 0;
        if constexpr (G == 1) {
            const int cnt = __popc(accm);
            const int incl = warp_inclusive_scan(cnt, lane);
            const int total = __shfl_sync(0xffffffffu, incl, 31);
            if (total == 0) {
                m += 1;
            } else {
                const long long blk = t >> 2;
                if (blk != cr_blk) {
                    cr = philox4x32_10(0u, (uint32_t)(t & ~3ll), rep, 1u, keys);
                    cr_blk = blk;
                }
                const int j = (int)__umulhi(pick(cr, (int)(t & 3)), (uint32_t)total);
                const int excl = incl - cnt;
                own_lane = __ffs(__ballot_sync(0xffffffffu, j >= excl && j < incl)) - 1;
                const int pos = nth_set_bit(accm, j - excl);
                vk = __shfl_sync(0xffffffffu, pos, own_lane);
                xold = (__shfl_sync(0xffffffffu, xm, own_lane) >> vk) & 1u;
                k = own_lane * V + vk;
                m = 0;
            }
        } else {
            uint32_t* ap = accs + (t & 1) * 32 * G;
            uint32_t* xp = xss + (t & 1) * 32 * G;
            ap[w * 32 + lane] = accm;
            xp[w * 32 + lane] = xm;
            group_barrier(1 + g, 32 * G);
            if (pending) {          // book the flip of step t - 1
                Ecur = A::book(Ecur, pub[(t - 1) & 1]);
                if (Ecur < Ebest) { Ebest = Ecur; snapshot(); }
            }
            uint32_t e[G];
            int cnt = 0;
#pragma unroll
            for (int u = 0; u < G; ++u) { e[u] = ap[lane * G + u]; cnt += __popc(e[u]); }
            const int incl = warp_inclusive_scan(cnt, lane);
            const int total = __shfl_sync(0xffffffffu, incl, 31);
            if (total == 0) {
                m += 1;
            } else {
                const long long blk = t >> 2;
                if (blk != cr_blk) {
                    cr = philox4x32_10(0u, (uint32_t)(t & ~3ll), rep, 1u, keys);
                    cr_blk = blk;
                }
                const int j = (int)__umulhi(pick(cr, (int)(t & 3)), (uint32_t)total);
                const int excl = incl - cnt;
                const int L = __ffs(__ballot_sync(0xffffffffu, j >= excl && j < incl)) - 1;
                int ent = 0, pos = 0, rk = j - excl;
#pragma unroll
                for (int u = 0; u < G; ++u) {
                    const int cu = __popc(e[u]);
                    if (rk >= 0 && rk < cu) { ent = lane * G + u; pos = nth_set_bit(e[u], rk); }
                    rk -= cu;
                }
                ent = __shfl_sync(0xffffffffu, ent, L);
                vk = __shfl_sync(0xffffffffu, pos, L);
                own_warp = ent >> 5;
                own_lane = ent & 31;
                xold = (xp[ent] >> vk) & 1u;
                k = ent * V + vk;
                m = 0;
            }
        }

        if (k >= 0) {
            // Delta E_k from the owner's registers
            H gk = h[0];
#pragma unroll
            for (int v = 1; v < V; ++v)
                if (v == vk) gk = h[v];
            H dEk = 0;
            if constexpr (G == 1) {
                dEk = __shfl_sync(0xffffffffu, A::signed_field(gk, xold), own_lane);
            } else {
                if (w == own_warp && lane == own_lane) pub[t & 1] = A::signed_field(gk, xold);
            }
            Tw cv[V];
            if (FULL || base < p.N) Row<Tw, V>::load(Wm + (size_t)k * p.ldw + base, cv);
            // the next step's draws do not depend on row k: compute them while
            // its loads are in flight
            if (t + 1 < p.t1) draw_step(rr, (uint32_t)(t + 1));
            if (FULL || base < p.N) {
#pragma unroll
                for (int v = 0; v < V; ++v) h[v] = A::apply(h[v], cv[v], xold != 0u);
            }
            if (w == own_warp && lane == own_lane) xm ^= 1u << vk;
            ++flips;
            if constexpr (G == 1) {
                Ecur = A::book(Ecur, dEk);
                if (Ecur < Ebest) { Ebest = Ecur; snapshot(); }
            }
        } else if (t + 1 < p.t1) {
            draw_step(rr, (uint32_t)(t + 1));
        }
        if constexpr (G > 1) pending = k >= 0;
        if constexpr (TRACE) {
            if (w == 0 && lane == 0) p.trace[(size_t)r * p.trace_T + t] = k;
        }
    }
    if constexpr (G > 1) {
        group_barrier(1 + g, 32 * G);
        if (pending) {
            Ecur = A::book(Ecur, pub[(p.t1 - 1) & 1]);
            if (Ecur < Ebest) { Ebest = Ecur; snapshot(); }
        }
    }

#pragma unroll
    for (int v = 0; v < V; ++v) hg[v] = h[v];
    const uint32_t word = gather_word<V>(xm, lane);
    if (lane % P == 0) xg[word_of_lane] = word;
    if (w == 0 && lane == 0) {
        sc.E = A::store_e(Ecur);
        sc.best = A::store_e(Ebest);
        sc.flips = flips;
        sc.m = m;
        p.sc[r] = sc;
    }
}

template <typename Tw, int V, int G>
cudaError_t launch_vg(const StepShape& s, const StepParams& p, bool trace, cudaStream_t st)
{
    const int threads = 32 * G * s.rpb;
    const int blocks = (p.R + s.rpb - 1) / s.rpb;
    const size_t shm = G > 1 ? (size_t)s.rpb * (4 * 32 * G + 4) * sizeof(uint32_t) : 0;
    if (blocks == 0) return cudaSuccess;
    const bool full = p.N == 32 * V * G;
    if (full) {
        if (trace) step_kernel<Tw, V, G, true, true><<<blocks, threads, shm, st>>>(p);
        else step_kernel<Tw, V, G, true, false><<<blocks, threads, shm, st>>>(p);
    } else {
        if (trace) step_kernel<Tw, V, G, false, true><<<blocks, threads, shm, st>>>(p);
        else step_kernel<Tw, V, G, false, false><<<blocks, threads, shm, st>>>(p);
    }
    return cudaGetLastError();
}

template <typename Tw>
cudaError_t launch_typed(const StepShape& s, const StepParams& p, bool trace, cudaStream_t st)
{
#define DA_CASE(VV, GG) \
    if (s.V == VV && s.G == GG) return launch_vg<Tw, VV, GG>(s, p, trace, st);
    DA_CASE(4, 1) DA_CASE(8, 1) DA_CASE(16, 1) DA_CASE(32, 1)
    DA_CASE(4, 2) DA_CASE(8, 2) DA_CASE(16, 2) DA_CASE(32, 2)
    DA_CASE(4, 4) DA_CASE(8, 4) DA_CASE(16, 4)
    DA_CASE(8, 8) DA_CASE(16, 8) DA_CASE(32, 8)
#undef DA_CASE
    return cudaErrorInvalidConfiguration;
}

}  // namespace step_detail
}  // namespace da
