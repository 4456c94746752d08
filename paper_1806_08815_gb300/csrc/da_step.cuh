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
//       Philox block (i/4, t, replica, 0).  The test is made in the log
//       domain, t = delta beta log2(e) + log2(2^24 u) - 24 < 0, with a
//       hardware log2 of the draw; trials with |t| within a band of 2^-15,
//       wider than the error of that estimate, take the exact test with the
//       library's exponential instead, so every decision equals the exact one;
//   (c) each lane's acceptance bits are already in index order, so a warp
//       prefix sum of their popcounts locates the j-th accepted variable,
//       j = floor(u * count); the chosen x_k flips while every lane adds
//       +-W[k][i] (16-byte loads of row k, which equals column k, from L2; the
//       fp32 forms read a copy of W in the warp row order, where each load of a
//       warp covers 512 contiguous bytes) to its fields.  The next step's
//       Philox words are computed while that row is in flight.  E_off returns
//       to 0 on a flip and grows by inc otherwise.
// A G = 1 group needs no shared memory or barrier.  A G > 1 group publishes
// its lanes' acceptance and state masks in shared memory behind one named
// barrier per step; the energy of step t is booked after the barrier of step
// t + 1, while x still holds the state right after step t.  The best-state
// test of a launch's last step is left pending (ReplicaScalars::check) so that
// it sees the energy after any recompute between launches, as Algorithm 2's
// result is defined after each complete step.
//
// Launches cover steps [t0, t1) and keep the state in global memory between
// launches (the fp32 path recomputes the fields between launches).
#pragma once
#include "da_device.cuh"
#include "da_internal.h"
#include "da_replica.cuh"
#include "da_step_common.cuh"
#include "da_tc.cuh"

namespace da {
namespace step_detail {

// A launch whose stop flag is set (a cancelled request of the request loop)
// returns at once and leaves the replica state as it was.  One thread reads
// the flag for the block, so that every warp of the block takes the same
// branch (the G > 1 groups meet at barriers).
__device__ __forceinline__ bool launch_stopped(const StepParams& p)
{
    __shared__ int s_stop;
    if (threadIdx.x == 0) s_stop = p.stop ? *reinterpret_cast<const volatile int*>(p.stop) : 0;
    __syncthreads();
    return s_stop != 0;
}

template <typename Tw, int V, int G, bool FULL, bool TRACE>
__global__ void __launch_bounds__(32 * G * OccupancyGV<G, V>::rpb, OccupancyGV<G, V>::min_blocks)
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
    if (launch_stopped(p)) return;
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
    constexpr bool kCoal = sizeof(Tw) == 4 && V >= 8;   // fp32 forms: rows from p.Wc (step_uses_coal)
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
    bool chk = sc.check != 0;       // best-state test pending from the previous launch
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
    // Acceptance draws of one step as log2 U (lg2_draw): Philox block q covers
    // variables base + 4q .. + 3.
    // The step-invariant Philox words precomputed (as WarpReplica's PRE form) where the
    // launch bounds leave at least 128 registers a thread and V <= 16; V = 32 and the
    // 7-blocks-per-SM shapes have no room for them.
    constexpr int kRegCap = 65536 / (32 * G * OccupancyGV<G, V>::rpb * OccupancyGV<G, V>::min_blocks);
    constexpr bool kPre = V <= 16 && kRegCap >= 128;
    constexpr int NP = kPre ? NQ : 1;
    uint32_t kq1[NP], kq2[NP], kq3[NP], kq4[NP], ku0 = 0;
    if constexpr (kPre) {
        const uint64_t pb0 = (uint64_t)kPhiloxMulB * rep;
        ku0 = (uint32_t)(pb0 >> 32) ^ keys.a[0];
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            const uint64_t pa0 = (uint64_t)kPhiloxMulA * ((uint32_t)(base >> 2) + q);
            const uint64_t pb1 = (uint64_t)kPhiloxMulB * ((uint32_t)(pa0 >> 32) ^ keys.b[0]);
            const uint64_t pa2 = (uint64_t)kPhiloxMulA * ((uint32_t)(pb1 >> 32) ^ (uint32_t)pb0 ^ keys.a[1]);
            kq1[q] = (uint32_t)pa0 ^ keys.b[1];
            kq2[q] = (uint32_t)pb1 ^ keys.a[2];
            kq3[q] = (uint32_t)(pa2 >> 32) ^ keys.b[2];
            kq4[q] = (uint32_t)pa2 ^ keys.b[3];
        }
    }
    auto draw_step = [&](float (&lg)[V], uint32_t tt) {
        if constexpr (kPre) {
            const uint64_t P = (uint64_t)kPhiloxMulA * (ku0 ^ tt);
            const uint32_t hP = (uint32_t)(P >> 32), lP = (uint32_t)P;
            uint32_t c0[NQ], c1[NQ], c2[NQ], c3[NQ];
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
                const uint64_t pb = (uint64_t)kPhiloxMulB * (hP ^ kq1[q]);
                c0[q] = (uint32_t)(pb >> 32) ^ kq2[q];
                c1[q] = (uint32_t)pb;
                c2[q] = kq3[q] ^ lP;
                c3[q] = kq4[q];
            }
#pragma unroll
            for (int round = 3; round < 10; ++round) {
#pragma unroll
                for (int q = 0; q < NQ; ++q) {
                    const uint64_t pa = (uint64_t)kPhiloxMulA * c0[q];
                    const uint64_t pb = (uint64_t)kPhiloxMulB * c2[q];
                    c0[q] = (uint32_t)(pb >> 32) ^ c1[q] ^ keys.a[round];
                    // kq4 carried kb_3 into c3, so round 3 adds no key to it
                    c2[q] = (uint32_t)(pa >> 32) ^ c3[q] ^ (round == 3 ? 0u : keys.b[round]);
                    c1[q] = (uint32_t)pb;
                    c3[q] = (uint32_t)pa;
                }
            }
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
                lg[4 * q] = lg2_draw(c0[q]);
                lg[4 * q + 1] = lg2_draw(c1[q]);
                lg[4 * q + 2] = lg2_draw(c2[q]);
                lg[4 * q + 3] = lg2_draw(c3[q]);
            }
        } else {
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
                const u32x4 w4 = philox4x32_10((uint32_t)(base >> 2) + q, tt, rep, 0u, keys);
                lg[4 * q] = lg2_draw(w4.x);
                lg[4 * q + 1] = lg2_draw(w4.y);
                lg[4 * q + 2] = lg2_draw(w4.z);
                lg[4 * q + 3] = lg2_draw(w4.w);
            }
        }
    };
    float lg[V];
    if (p.t0 < p.t1) draw_step(lg, (uint32_t)p.t0);

    float beta_next = (!per_rep && p.t0 < p.t1) ? p.beta[p.t0] : beta_rep;
    for (long long t = p.t0; t < p.t1; ++t) {
        const float beta = beta_next;
        if (!per_rep && t + 1 < p.t1) beta_next = p.beta[t + 1];
        const float Eoff = __fmul_rn(__uint2float_rn(m), p.inc);

        // (a) + (b): every trial of this lane in the log domain (decide_log),
        // the rare trials near the threshold by the exact test (decide_exact).
        bool unsure;
        uint32_t accm = decide_log<A, V>(h, xm, Eoff, __fmul_rn(beta, kLog2e), lg, unsure);
        if (__any_sync(0xffffffffu, unsure))
            accm = decide_exact<A, V>(h, xm, Eoff, beta, lg, accm, base, (uint32_t)t, rep, keys);
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
                chk = true;
            }
            if (chk) {              // and test it: x is still the state after step t - 1
                chk = false;
                if (Ecur < Ebest) { Ebest = Ecur; snapshot(); }
            }
            uint32_t e[G];
            int cnt = 0;
#pragma unroll
            for (int u = 0; u < G; ++u) { e[u] = ap[lane * G + u]; cnt += __popc(e[u]); }
            const int total = (int)__reduce_add_sync(0xffffffffu, (unsigned)cnt);
            const int incl = warp_inclusive_scan(cnt, lane);
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
            const H gk = select_slot<H, V>(h, vk);
            H dEk = 0;
            if constexpr (G == 1) {
                dEk = __shfl_sync(0xffffffffu, A::signed_field(gk, xold), own_lane);
            } else {
                if (w == own_warp && lane == own_lane) pub[t & 1] = A::signed_field(gk, xold);
            }
            Tw cv[V];
            if (FULL || base < p.N) {
                if constexpr (kCoal)   // this warp's slice of the row in the warp row order (pitch npad)
                    RowCoal<Tw, V>::load(static_cast<const Tw*>(p.Wc) + (size_t)k * p.npad + w * 32 * V + 4 * lane,
                                         cv);
                else
                    Row<Tw, V>::load(Wm + (size_t)k * p.ldw + base, cv);
            }
            // the next step's draws do not depend on row k: compute them while
            // its loads are in flight
            if (t + 1 < p.t1) draw_step(lg, (uint32_t)(t + 1));
            if (FULL || base < p.N) {
                const typename A::Sign sg = A::sign(xold);
#pragma unroll
                for (int v = 0; v < V; ++v) h[v] = A::apply_signed(h[v], cv[v], sg);
            }
            if (w == own_warp && lane == own_lane) xm ^= 1u << vk;
            ++flips;
            if constexpr (G == 1) {
                Ecur = A::book(Ecur, dEk);
                if (Ecur < Ebest) { Ebest = Ecur; snapshot(); }
            }
        } else if (t + 1 < p.t1) {
            draw_step(lg, (uint32_t)(t + 1));
        }
        if constexpr (G > 1) pending = k >= 0;
        if constexpr (TRACE) {
            if (w == 0 && lane == 0) p.trace[(size_t)r * p.trace_T + t] = k;
        }
    }
    if constexpr (G > 1) {
        group_barrier(1 + g, 32 * G);
        if (pending) {              // book the last flip; its test waits for any recompute
            Ecur = A::book(Ecur, pub[(p.t1 - 1) & 1]);
            chk = true;
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
        sc.check = chk ? 1u : 0u;
        p.sc[r] = sc;
    }
}

// G = 1: one warp per replica, the body of WarpReplica.  PT: the launch anneals
// replicas at fixed per-replica temperatures (p.betas), where the best-state test
// stays before the count.  The fp32 forms at V >= 8 read their rows from p.Wc
// (the warp row order, pitch 32 V).
template <typename Tw, int V, bool FULL, bool TRACE, bool PT = false>
__global__ void __launch_bounds__(32 * Occupancy<1>::rpb, Occupancy<1>::min_blocks)
    step_kernel_g1(const __grid_constant__ StepParams p)
{
    constexpr bool kCoal = sizeof(Tw) == 4 && V >= 8;   // float and f32e
    using R_ = WarpReplica<Tw, V, false, true, !PT && V >= 8, kCoal>;
    using H = typename R_::H;
    if (launch_stopped(p)) return;
    const int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (r >= p.R) return;
    R_ rp;
    rp.init(static_cast<const Tw*>(kCoal ? p.Wc : p.W), p.N, kCoal ? 32 * V : p.ldw, p.rep_base + (uint32_t)r,
            p.bestx + (size_t)r * p.nw);
    H* hg = static_cast<H*>(p.h) + (size_t)r * p.npad + rp.base;
    uint32_t* xg = p.x + (size_t)r * p.nw;
#pragma unroll
    for (int v = 0; v < V; ++v) rp.h[v] = hg[v];
    rp.xm = (xg[rp.base >> 5] >> (rp.base & 31)) & R_::VMASK;
    ReplicaScalars sc = p.sc[r];
    rp.Ecur = Arith<Tw>::load_e(sc.E);
    rp.Ebest = Arith<Tw>::load_e(sc.best);
    rp.flips = sc.flips;
    rp.m = sc.m;
    rp.chk = sc.check != 0;
    const PhiloxKeys& keys = *reinterpret_cast<const PhiloxKeys*>(&p.round_key[0][0]);
    const bool per_rep = p.betas != nullptr;
    const float beta_rep = per_rep ? p.betas[p.temp_of[r]] : 0.f;
    rp.prep_draws(keys);
    if (p.t0 < p.t1) rp.draw_pre((uint32_t)p.t0, keys);
    float beta_next = (!per_rep && p.t0 < p.t1) ? p.beta[p.t0] : beta_rep;
    for (long long t = p.t0; t < p.t1; ++t) {
        const float beta = beta_next;
        if (!per_rep && t + 1 < p.t1) beta_next = p.beta[t + 1];
        const int k = rp.template step<FULL>(t, t + 1 < p.t1, beta, p.inc, keys);
        if constexpr (TRACE) {
            if (rp.lane == 0) p.trace[(size_t)r * p.trace_T + t] = k;
        }
    }
#pragma unroll
    for (int v = 0; v < V; ++v) hg[v] = rp.h[v];
    const uint32_t word = rp.word();
    if (rp.lane % R_::P == 0) xg[rp.base >> 5] = word;
    if (rp.lane == 0) {
        sc.E = Arith<Tw>::store_e(rp.Ecur);
        sc.best = Arith<Tw>::store_e(rp.Ebest);
        sc.flips = rp.flips;
        sc.m = rp.m;
        sc.check = rp.chk ? 1u : 0u;
        p.sc[r] = sc;
    }
}

// G = 1 with warp specialisation: block = one replica = an annealer warp
// (WarpReplica::step_log) and a producer warp that computes the acceptance
// draws of the coming steps, L = log2 U for every trial, into a ring of
// kWsRing shared-memory buffers.  The producer depends on nothing the
// annealer computes, so it runs up to kWsRing steps ahead; the annealer reads
// the next step's buffer while its row load is in flight.  Full/empty
// handshakes are mbarriers whose waits are bounded (a wait that gives up
// sets *p.err and ends the launch; the replica's results are then invalid,
// and later launches that see the flag leave at once).
constexpr int kWsRing = 4;
constexpr uint32_t kWsWaitPolls = 1u << 26;
constexpr uint64_t kWsWaitNs = 2000000000ull;

template <typename Tw, int V, bool FULL, bool TRACE>
__global__ void __launch_bounds__(64, 7) step_kernel_ws(const __grid_constant__ StepParams p)
{
    using R_ = WarpReplica<Tw, V>;
    using H = typename R_::H;
    constexpr int NQ = V / 4;
    __shared__ float4 ring[kWsRing][NQ][32];
    __shared__ uint64_t full[kWsRing], empty[kWsRing];
    __shared__ int failed;
    const int r = blockIdx.x;
    if (r >= p.R) return;   // whole block
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int b = 0; b < kWsRing; ++b) {
            tc::mbar_init(&full[b], 32);
            tc::mbar_init(&empty[b], 32);
        }
        failed = (p.err ? *reinterpret_cast<volatile int*>(p.err) : 0) |
                 (p.stop ? *reinterpret_cast<const volatile int*>(p.stop) : 0);
    }
    __syncthreads();
    if (failed) return;     // whole block
    const PhiloxKeys& keys = *reinterpret_cast<const PhiloxKeys*>(&p.round_key[0][0]);
    const uint32_t rep = p.rep_base + (uint32_t)r;
    const long long n = p.t1 - p.t0;

    if (warp == 1) {   // producer: draws of steps t0 .. t1 - 1, in order
        const uint32_t q0 = (uint32_t)(lane * V) >> 2;
        for (long long i = 0; i < n; ++i) {
            const int b = (int)(i % kWsRing);
            const uint32_t ph = (uint32_t)(i / kWsRing);
            if (ph > 0 && !tc::mbar_wait(&empty[b], (ph - 1) & 1u, kWsWaitPolls, kWsWaitNs)) {
                if (p.err) atomicExch(p.err, 2);
                break;
            }
            const uint32_t tt = (uint32_t)(p.t0 + i);
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
                const u32x4 w = philox4x32_10(q0 + q, tt, rep, 0u, keys);
                ring[b][q][lane] = make_float4(lg2_draw(w.x), lg2_draw(w.y), lg2_draw(w.z), lg2_draw(w.w));
            }
            tc::mbar_arrive(&full[b]);
        }
        return;
    }

    R_ rp;
    rp.init(static_cast<const Tw*>(p.W), p.N, p.ldw, rep, p.bestx + (size_t)r * p.nw);
    H* hg = static_cast<H*>(p.h) + (size_t)r * p.npad + rp.base;
    uint32_t* xg = p.x + (size_t)r * p.nw;
#pragma unroll
    for (int v = 0; v < V; ++v) rp.h[v] = hg[v];
    rp.xm = (xg[rp.base >> 5] >> (rp.base & 31)) & R_::VMASK;
    ReplicaScalars sc = p.sc[r];
    rp.Ecur = Arith<Tw>::load_e(sc.E);
    rp.Ebest = Arith<Tw>::load_e(sc.best);
    rp.flips = sc.flips;
    rp.m = sc.m;
    rp.chk = sc.check != 0;
    const bool per_rep = p.betas != nullptr;
    const float beta_rep = per_rep ? p.betas[p.temp_of[r]] : 0.f;

    float L[V];
    bool ok = true;
    auto fetch = [&](long long i) {   // the draws of step t0 + i, then release the buffer
        const int b = (int)(i % kWsRing);
        if (!tc::mbar_wait(&full[b], (uint32_t)(i / kWsRing) & 1u, kWsWaitPolls, kWsWaitNs)) {
            ok = false;
            return;
        }
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            const float4 f = ring[b][q][lane];
            L[4 * q] = f.x; L[4 * q + 1] = f.y; L[4 * q + 2] = f.z; L[4 * q + 3] = f.w;
        }
        tc::mbar_arrive(&empty[b]);
    };
    if (n > 0) fetch(0);
    float beta_next = (!per_rep && n > 0) ? p.beta[p.t0] : beta_rep;
    for (long long i = 0; i < n && __all_sync(0xffffffffu, ok); ++i) {
        const long long t = p.t0 + i;
        const float beta = beta_next;
        if (!per_rep && i + 1 < n) beta_next = p.beta[t + 1];
        const int k = rp.template step_log<FULL>(t, beta, p.inc, L, keys, [&] {
            if (i + 1 < n) fetch(i + 1);
        });
        if constexpr (TRACE) {
            if (lane == 0) p.trace[(size_t)r * p.trace_T + t] = k;
        }
    }
    if (!__all_sync(0xffffffffu, ok) && lane == 0 && p.err) atomicExch(p.err, 2);
#pragma unroll
    for (int v = 0; v < V; ++v) hg[v] = rp.h[v];
    const uint32_t word = rp.word();
    if (lane % R_::P == 0) xg[rp.base >> 5] = word;
    if (lane == 0) {
        sc.E = Arith<Tw>::store_e(rp.Ecur);
        sc.best = Arith<Tw>::store_e(rp.Ebest);
        sc.flips = rp.flips;
        sc.m = rp.m;
        sc.check = rp.chk ? 1u : 0u;
        p.sc[r] = sc;
    }
}

// One launch of kernel K with the on-chip memory split of prefer_shared; with
// no blocks (p.R = 0) only the attribute is set, which also loads the kernel.
template <auto K>
inline void launch_shared(int blocks, int threads, size_t shm, cudaStream_t st, const StepParams& p)
{
    prefer_shared<K>();
    if (blocks > 0) K<<<blocks, threads, shm, st>>>(p);
}

template <typename Tw, int V, int G>
cudaError_t launch_vg(const StepShape& s, const StepParams& p, bool trace, cudaStream_t st)
{
    const int threads = 32 * G * s.rpb;
    const int blocks = (p.R + s.rpb - 1) / s.rpb;
    const size_t shm = G > 1 ? (size_t)s.rpb * (4 * 32 * G + 4) * sizeof(uint32_t) : 0;
    const bool full = p.N == 32 * V * G;
    if constexpr (G == 1) {
        if (s.ws) {
            if (blocks == 0) return cudaSuccess;
            if (full) {
                if (trace) step_kernel_ws<Tw, V, true, true><<<p.R, 64, 0, st>>>(p);
                else step_kernel_ws<Tw, V, true, false><<<p.R, 64, 0, st>>>(p);
            } else {
                if (trace) step_kernel_ws<Tw, V, false, true><<<p.R, 64, 0, st>>>(p);
                else step_kernel_ws<Tw, V, false, false><<<p.R, 64, 0, st>>>(p);
            }
            return cudaGetLastError();
        }
        const bool pt = p.betas != nullptr;
        if (blocks > 0 && sizeof(Tw) == 4 && V >= 8 && p.Wc == nullptr) return cudaErrorInvalidValue;
        if (full) {
            if (trace) launch_shared<step_kernel_g1<Tw, V, true, true>>(blocks, threads, 0, st, p);
            else if (pt) launch_shared<step_kernel_g1<Tw, V, true, false, true>>(blocks, threads, 0, st, p);
            else launch_shared<step_kernel_g1<Tw, V, true, false>>(blocks, threads, 0, st, p);
        } else {
            if (trace) launch_shared<step_kernel_g1<Tw, V, false, true>>(blocks, threads, 0, st, p);
            else if (pt) launch_shared<step_kernel_g1<Tw, V, false, false, true>>(blocks, threads, 0, st, p);
            else launch_shared<step_kernel_g1<Tw, V, false, false>>(blocks, threads, 0, st, p);
        }
        return cudaGetLastError();
    }
    if (blocks > 0 && sizeof(Tw) == 4 && V >= 8 && p.Wc == nullptr) return cudaErrorInvalidValue;
    if (full) {
        if (trace) launch_shared<step_kernel<Tw, V, G, true, true>>(blocks, threads, shm, st, p);
        else launch_shared<step_kernel<Tw, V, G, true, false>>(blocks, threads, shm, st, p);
    } else {
        if (trace) launch_shared<step_kernel<Tw, V, G, false, true>>(blocks, threads, shm, st, p);
        else launch_shared<step_kernel<Tw, V, G, false, false>>(blocks, threads, shm, st, p);
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
    DA_CASE(4, 4) DA_CASE(8, 4) DA_CASE(16, 4) DA_CASE(32, 4)
    DA_CASE(8, 8) DA_CASE(16, 8) DA_CASE(32, 8)
#undef DA_CASE
    return cudaErrorInvalidConfiguration;
}

}  // namespace step_detail
}  // namespace da
