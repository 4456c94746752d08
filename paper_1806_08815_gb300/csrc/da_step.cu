// da_step.cu -- the Digital Annealer's parallel-trial Monte Carlo step
// (Algorithm 2 of arXiv:1806.08815) for many replicas at once.
//
// One group of G warps anneals one replica; lane l of warp w owns the
// variables i = w*32V + 32v + l (v < V), keeping their effective fields
// g_i = Q_ii + sum_j W_ij x_j and bits x_i in registers for the whole launch.
// Per step:
//   (a) every lane forms Delta E_i = (1 - 2 x_i) g_i for its V variables (all
//       N trials of the step run in parallel, Sec. II);
//   (b) Metropolis against the dynamic offset: delta = Delta E - E_off is
//       accepted when delta <= 0, else when u < exp(-beta delta); u is drawn
//       only for trials whose outcome is not already decided (Philox is
//       counter-based, so skipping a draw changes no other draw);
//   (c) the accepted trials become 32-bit ballot words in index order; a warp
//       prefix sum of their popcounts finds the j-th accepted index,
//       j = floor(u * count), and the chosen x_k flips while every lane adds
//       +-W[k][i] (one coalesced pass over column k, read through L2) to its
//       fields; the Philox words of the next step are computed while that
//       column is in flight.  E_off returns to 0 on a flip and grows by inc
//       otherwise.
// A G = 1 group needs no shared memory or barrier: the words live one per
// lane.  A G > 1 group exchanges its words through shared memory with one
// named barrier per step; the energy of step t is booked after the barrier of
// step t + 1, while x still holds the state right after step t.
//
// Launches cover steps [t0, t1) and keep the state in global memory between
// launches (the fp32 path recomputes the fields between launches).
#include "da_device.cuh"
#include "da_internal.h"

namespace da {
namespace {

template <typename Tw> struct Arith;
template <> struct Arith<int8_t> {
    using H = int32_t;    // fields and linear terms
    using E = long long;  // tracked energy
    static __device__ __forceinline__ float delta(H dE, float Eoff) { return __fsub_rn(__int2float_rn(dE), Eoff); }
    static __device__ __forceinline__ H apply(H h, int8_t w, bool minus) { return minus ? h - (H)w : h + (H)w; }
    static __device__ __forceinline__ E load_e(long long b) { return b; }
    static __device__ __forceinline__ long long store_e(E e) { return e; }
    static __device__ __forceinline__ E book(E e, H dE) { return e + (E)dE; }
};
template <> struct Arith<float> {
    using H = float;
    using E = double;
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

// Replicas per block and the blocks per SM the register budget is sized for:
// at least 7 replicas per SM, so that 1024 replicas fill 152 SMs in one wave.
template <int G> struct Occupancy;
template <> struct Occupancy<1> { static constexpr int rpb = 4, min_blocks = 2; };
template <> struct Occupancy<2> { static constexpr int rpb = 2, min_blocks = 4; };
template <> struct Occupancy<4> { static constexpr int rpb = 1, min_blocks = 7; };
template <> struct Occupancy<8> { static constexpr int rpb = 1, min_blocks = 2; };

template <typename Tw, int V, int G, bool TRACE>
__global__ void __launch_bounds__(32 * G * Occupancy<G>::rpb, Occupancy<G>::min_blocks)
    step_kernel(const __grid_constant__ StepParams p)
{
    using A = Arith<Tw>;
    using H = typename A::H;
    using E = typename A::E;
    constexpr int NWG = V * G;              // ballot words per replica
    constexpr int CW = (NWG + 31) / 32;     // words per lane during the choice
    constexpr int QS = V >= 4 ? 4 : V;      // variables of one lane per Philox block
    static_assert(V == 1 || V == 2 || V % 4 == 0, "V must be 1, 2 or a multiple of 4");

    extern __shared__ uint32_t smem[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int g = wib / G;                  // group (replica) within the block
    const int w = wib - g * G;              // warp within the group
    const int rpb = blockDim.x / (32 * G);
    const int r = blockIdx.x * rpb + g;
    if (r >= p.R) return;

    uint32_t* gs = smem + g * (4 * NWG + 4);
    uint32_t* accw = gs;                    // [2][NWG] accepted-trial words
    uint32_t* xws = gs + 2 * NWG;           // [2][NWG] state words
    H* pub = reinterpret_cast<H*>(gs + 4 * NWG);  // [2] Delta E of the flipped variable

    const Tw* __restrict__ Wm = static_cast<const Tw*>(p.W);
    const int base = w * 32 * V + lane;
    H h[V];
    uint32_t valid = 0, xm = 0;
    H* hg = static_cast<H*>(p.h) + (size_t)r * p.npad;
    uint32_t* xg = p.x + (size_t)r * p.nw;
    uint32_t* bestg = p.bestx + (size_t)r * p.nw;
#pragma unroll
    for (int v = 0; v < V; ++v) {
        const int i = base + 32 * v;
        const bool ok = i < p.N;
        h[v] = hg[i];
        valid |= (uint32_t)ok << v;
        xm |= ((xg[w * V + v] >> lane) & 1u) << v;
    }
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
    constexpr int NQ = V / QS;              // Philox blocks per lane per step

    auto snapshot = [&]() {
        uint32_t bw = 0;
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const uint32_t b = __ballot_sync(0xffffffffu, (xm >> v) & 1u);
            if (lane == v) bw = b;
        }
        if (lane < V) bestg[w * V + lane] = bw;
    };
    // The acceptance draws of one step: block q of this lane covers variables
    // i0 + 32c + lane (c < QS) with i0 = w*32V + 32*q*QS; counter word 0 is
    // 32*(i0/128) + lane, output lane (i0/32)%4 + c.
    auto draw_step = [&](u32x4 (&rr)[NQ], uint32_t tt) {
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            const int i0 = w * 32 * V + 32 * q * QS;
            rr[q] = philox4x32_10(32u * (uint32_t)(i0 >> 7) + (uint32_t)lane, tt, rep, 0u, keys);
        }
    };
    u32x4 rr[NQ];
    if (p.t0 < p.t1) draw_step(rr, (uint32_t)p.t0);

    float beta_next = (!per_rep && p.t0 < p.t1) ? p.beta[p.t0] : beta_rep;
    for (long long t = p.t0; t < p.t1; ++t) {
        const float beta = beta_next;
        if (!per_rep && t + 1 < p.t1) beta_next = p.beta[t + 1];
        const float Eoff = __fmul_rn(__uint2float_rn(m), p.inc);

        // (a) + (b): every trial of this lane, one Philox block of QS
        // variables at a time; u is compared only where delta > 0 and
        // exp(-beta delta) > 2^-24.
        uint32_t accm = 0;
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            float ax[QS];
            uint32_t nq = 0;
#pragma unroll
            for (int c = 0; c < QS; ++c) {
                const int v = q * QS + c;
                const H dE = ((xm >> v) & 1u) ? -h[v] : h[v];
                const float delta = A::delta(dE, Eoff);
                const bool ok = (valid >> v) & 1u;
                ax[c] = -__fmul_rn(beta, delta);
                const bool le0 = delta <= 0.0f;
                accm |= (uint32_t)(ok && le0) << v;
                nq |= (uint32_t)(ok && !le0 && ax[c] > kExpCut) << c;
            }
            if (__any_sync(0xffffffffu, nq != 0u)) {
                const int sub0 = (V % 4 == 0) ? 0 : (((w * 32 * V + 32 * q * QS) >> 5) & 3);
#pragma unroll
                for (int c = 0; c < QS; ++c) {
                    if ((nq >> c) & 1u)
                        accm |= (uint32_t)metropolis_accept(ax[c], pick(rr[q], sub0 + c)) << (q * QS + c);
                }
            }
        }

        // ballot words in index order: word w*V + v covers variables 32(w*V + v) + lane
        uint32_t wl[CW];
#pragma unroll
        for (int u = 0; u < CW; ++u) wl[u] = 0;
        uint32_t* aw = accw + (t & 1) * NWG;
        uint32_t* xw = xws + (t & 1) * NWG;
        if constexpr (G == 1) {
#pragma unroll
            for (int v = 0; v < V; ++v) {
                const uint32_t b = __ballot_sync(0xffffffffu, (accm >> v) & 1u);
                if (lane == v) wl[0] = b;
            }
        } else {
#pragma unroll
            for (int v = 0; v < V; ++v) {
                const uint32_t b = __ballot_sync(0xffffffffu, (accm >> v) & 1u);
                const uint32_t bx = __ballot_sync(0xffffffffu, (xm >> v) & 1u);
                if (lane == 0) { aw[w * V + v] = b; xw[w * V + v] = bx; }
            }
            group_barrier(1 + g, 32 * G);
            if (pending) {          // book the flip of step t - 1
                Ecur = A::book(Ecur, pub[(t - 1) & 1]);
                if (Ecur < Ebest) { Ebest = Ecur; snapshot(); }
            }
#pragma unroll
            for (int u = 0; u < CW; ++u) {
                const int gw = lane * CW + u;
                if (gw < NWG) wl[u] = aw[gw];
            }
        }

        // (c) uniform choice among the accepted trials
        int cnt = 0;
#pragma unroll
        for (int u = 0; u < CW; ++u) cnt += __popc(wl[u]);
        const int incl = warp_inclusive_scan(cnt, lane);
        const int total = __shfl_sync(0xffffffffu, incl, 31);
        int k = -1;
        if (total == 0) {
            m += 1;
        } else {
            const long long blk = t >> 2;
            if (blk != cr_blk) {
                cr = philox4x32_10(0u, (uint32_t)(t & ~3ll), rep, 1u, keys);
                cr_blk = blk;
            }
            const uint32_t uc = pick(cr, (int)(t & 3));
            const int j = (int)__umulhi(uc, (uint32_t)total);
            const int excl = incl - cnt;
            const uint32_t own = __ballot_sync(0xffffffffu, j >= excl && j < incl);
            const int L = __ffs(own) - 1;
            int kk = 0;
            if (lane == L) {
                int rk = j - excl;
#pragma unroll
                for (int u = 0; u < CW; ++u) {
                    const int cu = __popc(wl[u]);
                    if (rk >= 0 && rk < cu) kk = (lane * CW + u) * 32 + nth_set_bit(wl[u], rk);
                    rk -= cu;
                }
            }
            k = __shfl_sync(0xffffffffu, kk, L);
            m = 0;
        }

        if (k >= 0) {
            const int gwk = k >> 5, kb = k & 31;
            const int wk = gwk / V, vk = gwk - wk * V;
            // Delta E_k from the owner's registers
            H gk = h[0];
#pragma unroll
            for (int v = 1; v < V; ++v)
                if (v == vk) gk = h[v];
            uint32_t xold;
            H dEk = 0;
            if constexpr (G == 1) {
                xold = (__shfl_sync(0xffffffffu, xm, kb) >> vk) & 1u;
                dEk = __shfl_sync(0xffffffffu, xold ? -gk : gk, kb);
            } else {
                xold = (xw[gwk] >> kb) & 1u;
                if (w == wk && lane == kb) pub[t & 1] = xold ? -gk : gk;
            }
            const Tw* __restrict__ col = Wm + (size_t)k * p.ldw;
            Tw cv[V];
#pragma unroll
            for (int v = 0; v < V; ++v) cv[v] = ((valid >> v) & 1u) ? __ldg(col + base + 32 * v) : Tw(0);
            // the next step's draws do not depend on the column: compute them
            // while its loads are in flight
            if (t + 1 < p.t1) draw_step(rr, (uint32_t)(t + 1));
#pragma unroll
            for (int v = 0; v < V; ++v) h[v] = A::apply(h[v], cv[v], xold != 0u);
            if (w == wk && lane == kb) xm ^= 1u << vk;
            ++flips;
            if constexpr (G == 1) {
                Ecur = A::book(Ecur, dEk);
                if (Ecur < Ebest) { Ebest = Ecur; snapshot(); }
            }
        }
        else if (t + 1 < p.t1) {
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
    for (int v = 0; v < V; ++v) {
        hg[base + 32 * v] = h[v];
        const uint32_t bx = __ballot_sync(0xffffffffu, (xm >> v) & 1u);
        if (lane == 0) xg[w * V + v] = bx;
    }
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
    const size_t shm = G > 1 ? (size_t)s.rpb * (4 * V * G + 4) * sizeof(uint32_t) : 0;
    if (blocks == 0) return cudaSuccess;
    if (trace)
        step_kernel<Tw, V, G, true><<<blocks, threads, shm, st>>>(p);
    else
        step_kernel<Tw, V, G, false><<<blocks, threads, shm, st>>>(p);
    return cudaGetLastError();
}

template <typename Tw>
cudaError_t launch_typed(const StepShape& s, const StepParams& p, bool trace, cudaStream_t st)
{
#define DA_CASE(VV, GG) \
    if (s.V == VV && s.G == GG) return launch_vg<Tw, VV, GG>(s, p, trace, st);
    DA_CASE(2, 1) DA_CASE(4, 1) DA_CASE(8, 1) DA_CASE(16, 1) DA_CASE(32, 1)
    DA_CASE(4, 2) DA_CASE(8, 2) DA_CASE(16, 2) DA_CASE(32, 2)
    DA_CASE(4, 4) DA_CASE(8, 4) DA_CASE(16, 4) DA_CASE(32, 4)
    DA_CASE(4, 8) DA_CASE(8, 8) DA_CASE(16, 8) DA_CASE(32, 8)
#undef DA_CASE
    return cudaErrorInvalidConfiguration;
}

}  // namespace

bool step_shape_supported(const StepShape& s)
{
    const bool g1 = s.G == 1 && (s.V == 2 || s.V == 4 || s.V == 8 || s.V == 16 || s.V == 32);
    const bool gn = (s.G == 2 || s.G == 4 || s.G == 8) && (s.V == 4 || s.V == 8 || s.V == 16 || s.V == 32);
    const int max_rpb = s.G == 1 ? Occupancy<1>::rpb : s.G == 2 ? Occupancy<2>::rpb : 1;
    return (g1 || gn) && s.rpb >= 1 && s.rpb <= max_rpb;
}

cudaError_t launch_step(bool is_int8, const StepShape& s, const StepParams& p, bool trace, cudaStream_t st)
{
    if (!step_shape_supported(s)) return cudaErrorInvalidConfiguration;
    return is_int8 ? launch_typed<int8_t>(s, p, trace, st) : launch_typed<float>(s, p, trace, st);
}

}  // namespace da
