// da_replica.cuh -- one replica annealed by one warp (the G = 1 form of the
// step in da_step.cuh), packaged so that the chunked step kernel and the
// persistent batched kernel share it.
//
// Lane l owns the V consecutive variables i = l*V + v of the replica and keeps
// their effective fields g_i, bits x_i and the Philox words of the current step
// in registers.  step() performs one step of Algorithm 2 (see da_step.cuh for
// the decomposition); recompute() replaces the fp32 fields and the tracked
// energy by their exact fixed-point values (the same definition as the tiled
// recompute in da_fields.cu, evaluated by the warp itself).
#pragma once
#include "da_device.cuh"
#include "da_fixed.cuh"
#include "da_internal.h"
#include "da_step_common.cuh"

namespace da {
namespace step_detail {

// SW: the rows of W are read from a copy staged in shared memory (W points
// there) instead of from global memory.
// PRE: the step-invariant part of each Philox block is computed once per launch
// (prep_draws) and the draws of every step start from it (draw_pre); four more
// words per block live in registers, for kernels that have them to spare.
// LATE: the best-state test is made under the row load (see flush_best).
// COAL: W points at the couplings in the warp row order (row pitch ldw = 32 V;
// step_uses_coal in da_internal.h) and rows are read with RowCoal.
template <typename Tw, int V, bool SW = false, bool PRE = false, bool LATE = (V >= 8), bool COAL = false>
struct WarpReplica {
    using A = Arith<Tw>;
    using H = typename A::H;
    using E = typename A::E;
    static_assert(V % 4 == 0 && V <= 32, "V must be 4, 8, 16 or 32");
    static constexpr int NQ = V / 4;
    static constexpr uint32_t VMASK = V == 32 ? 0xffffffffu : ((1u << V) - 1u);
    static constexpr int P = 32 / V;

    H h[V];
    float lg[V];      // log2 U of this lane's draws for the current step (lg2_draw)
    u32x4 cr;
    long long cr_blk;
    uint32_t xm, valid, m;
    bool chk;         // the best-state test of the last step (or recompute) is pending
    E Ecur, Ebest;
    long long flips;
    int lane, base, N, ldw;
    int rowoff;       // this lane's first entry in a row of W: base, or 4 lane in the G = 1 order
    uint32_t rep;
    const Tw* __restrict__ W;
    uint32_t* bestg;  // best-state words of this replica
    // Step-invariant Philox words of the lane's blocks (prep_draws): kq1..kq4 per
    // block, ku0 shared by the lane's blocks.
    uint32_t kq1[PRE ? NQ : 1], kq2[PRE ? NQ : 1], kq3[PRE ? NQ : 1], kq4[PRE ? NQ : 1];
    uint32_t ku0;

    __device__ __forceinline__ void init(const Tw* W_, int N_, int ldw_, uint32_t rep_, uint32_t* bestg_)
    {
        lane = threadIdx.x & 31;
        base = lane * V;
        rowoff = COAL ? 4 * lane : base;
        N = N_;
        ldw = ldw_;
        rep = rep_;
        W = W_;
        bestg = bestg_;
        valid = base >= N ? 0u : (N - base >= V ? VMASK : ((1u << (N - base)) - 1u));
        cr = {0, 0, 0, 0};
        cr_blk = -1;
        chk = false;
    }

    // The test of Algorithm 2's result: a strictly lower tracked energy than any
    // seen makes the current state the best one.  It is made one step late (x is
    // unchanged until the next flip), and after any recompute of the step.  With
    // LATE (by default for V >= 8) it runs while the next step's row of W is in
    // flight (or once it is known that nothing flips), so that the fp64 compare
    // stays off the chain from the trials to the row load; otherwise before the
    // count.  Measured: the late test is slower at V = 4, whose short row leaves no
    // room for it, and for replicas at fixed temperatures (parallel tempering),
    // whose low-temperature steps mostly flip nothing.
    static constexpr bool kTestUnderRow = LATE;
    __device__ __forceinline__ void flush_best()
    {
        if (chk) {
            chk = false;
            if (Ecur < Ebest) {
                Ebest = Ecur;
                snapshot();
            }
        }
    }

    __device__ __forceinline__ uint32_t word() const { return gather_word<V>(xm, lane); }

    static __device__ __forceinline__ void load_row(const Tw* p, Tw (&c)[V])
    {
        static_assert(!(SW && COAL), "a staged W is in the plain order");
        if constexpr (SW) RowShared<Tw, V>::load(p, c);
        else if constexpr (COAL) RowCoal<Tw, V>::load(p, c);
        else Row<Tw, V>::load(p, c);
    }

    __device__ __forceinline__ void snapshot()
    {
        const uint32_t wv = word();
        if (lane % P == 0) bestg[base >> 5] = wv;
    }

    template <class Keys>
    __device__ __forceinline__ void draw(uint32_t tt, const Keys& keys)
    {
        // the NQ Philox4x32-10 blocks round by round, so that their independent
        // multiply-xor chains interleave
        uint32_t c0[NQ], c1[NQ], c2[NQ], c3[NQ];
#pragma unroll
        for (int q = 0; q < NQ; ++q) { c0[q] = (uint32_t)(base >> 2) + q; c1[q] = tt; c2[q] = rep; c3[q] = 0u; }
#pragma unroll
        for (int round = 0; round < 10; ++round) {
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
                const uint64_t pa = (uint64_t)kPhiloxMulA * c0[q];
                const uint64_t pb = (uint64_t)kPhiloxMulB * c2[q];
                const uint32_t n0 = (uint32_t)(pb >> 32) ^ c1[q] ^ keys.a[round];
                const uint32_t n2 = (uint32_t)(pa >> 32) ^ c3[q] ^ keys.b[round];
                c1[q] = (uint32_t)pb;
                c3[q] = (uint32_t)pa;
                c0[q] = n0;
                c2[q] = n2;
            }
        }
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            lg[4 * q] = lg2_draw(c0[q]);
            lg[4 * q + 1] = lg2_draw(c1[q]);
            lg[4 * q + 2] = lg2_draw(c2[q]);
            lg[4 * q + 3] = lg2_draw(c3[q]);
        }
    }

    // The acceptance block q of step t has counter (c0, t, rep, 0), c0 = base/4 + q.
    // Following the words of Philox4x32-10 through its first rounds (round r:
    // products pa = A c0, pb = B c2; c0 <- hi(pb) ^ c1 ^ ka_r, c1 <- lo(pb),
    // c2 <- hi(pa) ^ c3 ^ kb_r, c3 <- lo(pa)):
    //   after round 0: (u ^ t, lo(B rep), y2_q, y3_q) with u = hi(B rep) ^ ka_0,
    //     y2_q = hi(A c0) ^ kb_0, y3_q = lo(A c0): only the first word depends on t;
    //   round 1 multiplies that word (one product per lane and step, P = A (u ^ t))
    //     and y2_q (step-invariant): after it (z0_q, z1_q, hi(P) ^ y3_q ^ kb_1, lo(P))
    //     with z0_q, z1_q step-invariant;
    //   round 2 multiplies z0_q (step-invariant) and the third word (per block).
    // So a step needs one product for the lane and, per block, one product in round
    // 2 and the full rounds 3..9: the words below are the step-invariant operands
    // with their round keys folded in.  draw_pre returns philox4x32_10's words bit
    // for bit.
    template <class Keys>
    __device__ __forceinline__ void prep_draws(const Keys& keys)
    {
        static_assert(PRE, "prep_draws needs PRE");
        const uint64_t pb0 = (uint64_t)kPhiloxMulB * rep;
        ku0 = (uint32_t)(pb0 >> 32) ^ keys.a[0];
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            const uint64_t pa0 = (uint64_t)kPhiloxMulA * ((uint32_t)(base >> 2) + q);
            const uint64_t pb1 = (uint64_t)kPhiloxMulB * ((uint32_t)(pa0 >> 32) ^ keys.b[0]);
            const uint64_t pa2 = (uint64_t)kPhiloxMulA * ((uint32_t)(pb1 >> 32) ^ (uint32_t)pb0 ^ keys.a[1]);
            kq1[q] = (uint32_t)pa0 ^ keys.b[1];               // y3_q ^ kb_1
            kq2[q] = (uint32_t)pb1 ^ keys.a[2];               // z1_q ^ ka_2
            kq3[q] = (uint32_t)(pa2 >> 32) ^ keys.b[2];       // hi(A z0_q) ^ kb_2
            kq4[q] = (uint32_t)pa2 ^ keys.b[3];               // lo(A z0_q) ^ kb_3
        }
    }

    // The next step's draws in stages (PRE), so that their rounds can fill the
    // latency of the current step's warp collectives: draw_begin (the per-step
    // product and round 2), draw_round<R> (rounds 3..9), draw_end (log2 U of the
    // 4 NQ words into lg).
    uint32_t dq0[PRE ? NQ : 1], dq1[PRE ? NQ : 1], dq2[PRE ? NQ : 1], dq3[PRE ? NQ : 1];

    __device__ __forceinline__ void draw_begin(uint32_t tt)
    {
        const uint64_t P = (uint64_t)kPhiloxMulA * (ku0 ^ tt);
        const uint32_t hP = (uint32_t)(P >> 32), lP = (uint32_t)P;
#pragma unroll
        for (int q = 0; q < NQ; ++q) {            // round 2
            const uint64_t pb = (uint64_t)kPhiloxMulB * (hP ^ kq1[q]);
            dq0[q] = (uint32_t)(pb >> 32) ^ kq2[q];
            dq1[q] = (uint32_t)pb;
            dq2[q] = kq3[q] ^ lP;
            dq3[q] = kq4[q];                       // carries kb_3
        }
    }

    template <int R, class Keys>
    __device__ __forceinline__ void draw_round(const Keys& keys)
    {
        static_assert(R >= 3 && R < 10, "rounds 3..9");
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            const uint64_t pa = (uint64_t)kPhiloxMulA * dq0[q];
            const uint64_t pb = (uint64_t)kPhiloxMulB * dq2[q];
            dq0[q] = (uint32_t)(pb >> 32) ^ dq1[q] ^ keys.a[R];
            if constexpr (R == 3) dq2[q] = (uint32_t)(pa >> 32) ^ dq3[q];
            else dq2[q] = (uint32_t)(pa >> 32) ^ dq3[q] ^ keys.b[R];
            dq1[q] = (uint32_t)pb;
            dq3[q] = (uint32_t)pa;
        }
    }

    template <int R0, int R1, class Keys>
    __device__ __forceinline__ void draw_rounds(const Keys& keys)
    {
        if constexpr (R0 < R1) {
            draw_round<R0>(keys);
            draw_rounds<R0 + 1, R1>(keys);
        }
    }

    __device__ __forceinline__ void draw_end()
    {
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            lg[4 * q] = lg2_draw(dq0[q]);
            lg[4 * q + 1] = lg2_draw(dq1[q]);
            lg[4 * q + 2] = lg2_draw(dq2[q]);
            lg[4 * q + 3] = lg2_draw(dq3[q]);
        }
    }

    template <class Keys>
    __device__ __forceinline__ void draw_pre(uint32_t tt, const Keys& keys)
    {
        draw_begin(tt);
        draw_rounds<3, 10>(keys);
        draw_end();
    }

    // Work a step places in the latency of its warp collectives (choose_and_flip):
    // begin() after the count reduction is issued, at<I>() after collective I is
    // issued and before its result is used (I = 0..4: the prefix-sum shuffles;
    // 5: the owner ballot; 6: the owner's position shuffle), rest_flip() while
    // row k is in flight, rest_none() when nothing flips.
    template <class F>
    struct RestOnly {      // everything under the row load (or at once)
        F& f;
        __device__ __forceinline__ void begin() {}
        template <int I> __device__ __forceinline__ void at() {}
        __device__ __forceinline__ void rest_flip() { f(); }
        __device__ __forceinline__ void rest_none() { f(); }
    };
    template <class Keys>
    struct DrawSlots {     // the next step's draws (PRE): rounds 3-5 in the prefix
        WarpReplica& rp;   // sum, 6-7 in the choice, 8-9 and log2 under the row load
        const Keys& keys;
        uint32_t tt;
        __device__ __forceinline__ void begin() { rp.draw_begin(tt); }
        template <int I>
        __device__ __forceinline__ void at()
        {
            if constexpr (I <= 2) rp.template draw_round<3 + I>(keys);
            else if constexpr (I == 5 || I == 6) rp.template draw_round<I + 1>(keys);
        }
        __device__ __forceinline__ void rest_flip()
        {
            rp.template draw_rounds<8, 10>(keys);
            rp.draw_end();
        }
        __device__ __forceinline__ void rest_none()
        {
            rp.template draw_rounds<6, 10>(keys);
            rp.draw_end();
        }
    };

    // One step t (the draws of t are in lg).  If draw_next, the draws of t + 1
    // are computed while row k is in flight (PRE: always, spread over the
    // step's collectives as DrawSlots places them).  Returns the flipped index
    // or -1.
    template <bool FULL, class Keys>
    __device__ __forceinline__ int step(long long t, bool draw_next, float beta, float inc, const Keys& keys)
    {
        if constexpr (PRE) {
            DrawSlots<Keys> s{*this, keys, (uint32_t)(t + 1)};
            return decide_and_flip<FULL>(t, beta, inc, lg, keys, s);
        } else {
            auto f = [&] {
                if (draw_next) draw((uint32_t)(t + 1), keys);
            };
            RestOnly<decltype(f)> s{f};
            return decide_and_flip<FULL>(t, beta, inc, lg, keys, s);
        }
    }

    // One step t whose acceptance draws are L[v] = log2 U of this lane's trials
    // (lg2_draw; from draw() or from a producer warp), decided in the log domain
    // (decide_log; the rare trials near the threshold by decide_exact).
    // `overlap` runs while row k is in flight.
    template <bool FULL, class Keys, class Overlap>
    __device__ __forceinline__ int step_log(long long t, float beta, float inc, const float (&L)[V], const Keys& keys,
                                            Overlap&& overlap)
    {
        RestOnly<Overlap> s{overlap};
        return decide_and_flip<FULL>(t, beta, inc, L, keys, s);
    }

    template <bool FULL, class Keys, class Slots>
    __device__ __forceinline__ int decide_and_flip(long long t, float beta, float inc, const float (&L)[V],
                                                   const Keys& keys, Slots& slots)
    {
        const float Eoff = __fmul_rn(__uint2float_rn(m), inc);
        bool unsure;
        uint32_t accm = decide_log<A, V>(h, xm, Eoff, __fmul_rn(beta, kLog2e), L, unsure);
        if (__any_sync(0xffffffffu, unsure))
            accm = decide_exact<A, V>(h, xm, Eoff, beta, L, accm, base, (uint32_t)t, rep, keys);
        return choose_and_flip<FULL>(t, accm, keys, slots);
    }

    // Inclusive prefix sum over the lanes, level I..4, with slots.at<I>() in the
    // latency of each shuffle.
    template <int I, class Slots>
    __device__ __forceinline__ void scan_levels(int& incl, Slots& slots)
    {
        if constexpr (I < 5) {
            const int n = __shfl_up_sync(0xffffffffu, incl, 1 << I);
            slots.template at<I>();
            if (lane >= (1 << I)) incl += n;
            scan_levels<I + 1>(incl, slots);
        }
    }

    // (c) of a step with acceptance mask accm: the uniform choice among the
    // accepted trials, the best-state test left by the previous step (under the
    // row load, or first at V = 4), the flip and the field update, with `slots`
    // placed as described above.  Returns the flipped index or -1.
    template <bool FULL, class Keys, class Slots>
    __device__ __forceinline__ int choose_and_flip(long long t, uint32_t accm, const Keys& keys, Slots& slots)
    {
        if constexpr (!FULL) accm &= valid;
        if constexpr (!kTestUnderRow) flush_best();

        const int cnt = __popc(accm);
        const int total = (int)__reduce_add_sync(0xffffffffu, (unsigned)cnt);
        slots.begin();
        int incl = cnt;
        scan_levels<0>(incl, slots);
        if (total == 0) {
            m += 1;
            if constexpr (kTestUnderRow) flush_best();
            slots.rest_none();
            return -1;
        }
        const long long blk = t >> 2;
        if (blk != cr_blk) {
            cr = philox4x32_10(0u, (uint32_t)(t & ~3ll), rep, 1u, keys);
            cr_blk = blk;
        }
        const int j = (int)__umulhi(pick(cr, (int)(t & 3)), (uint32_t)total);
        const int excl = incl - cnt;
        const int own = __ffs(__ballot_sync(0xffffffffu, j >= excl && j < incl)) - 1;
        const int pos = nth_set_bit(accm, j - excl);
        slots.template at<5>();
        const int vk = __shfl_sync(0xffffffffu, pos, own);
        slots.template at<6>();
        const uint32_t xold = (__shfl_sync(0xffffffffu, xm, own) >> vk) & 1u;
        const H gk = select_slot<H, V>(h, vk);
        const H dEk = __shfl_sync(0xffffffffu, A::signed_field(gk, xold), own);
        const int k = own * V + vk;
        Tw cv[V];
        if (FULL || base < N) load_row(W + (size_t)k * ldw + rowoff, cv);
        if constexpr (kTestUnderRow) flush_best();   // x is still the state after the previous step
        slots.rest_flip();
        if (FULL || base < N) {
            const typename A::Sign sg = A::sign(xold);
#pragma unroll
            for (int v = 0; v < V; ++v) h[v] = A::apply_signed(h[v], cv[v], sg);
        }
        if (lane == own) xm ^= 1u << vk;
        ++flips;
        m = 0;
        Ecur = A::book(Ecur, dEk);
        chk = true;
        return k;
    }

    // Exact fixed-point recompute of the fp32 fields and of the tracked
    // energy (same definition as da_fields.cu): g_i = fl32(2^-S (round(d_i 2^S)
    // + sum_{x_j = 1} round(W_ij 2^S))), E = fl64(2^-(S+1) sum_{x_i = 1}
    // (round(d_i 2^S) + sum_i)).
    // shift: every coupling and linear term reaches the grid by a left shift
    // (the host checked), so fixed_of_f32_shift converts it exactly.
    // The fields of padding variables (beyond N) are set to 0, their value at the
    // start of an anneal, so that no old field stays live across the row loop.
    __device__ __forceinline__ void recompute(const float* __restrict__ diag, int S, bool shift = false)
    {
        if (shift) recompute_impl<true>(diag, S);
        else recompute_impl<false>(diag, S);
    }

    template <bool SHIFT>
    static __device__ __forceinline__ long long to_fixed(float w, int S)
    {
        if constexpr (SHIFT) return fixed_of_f32_shift(w, S);
        else return fixed_of_f32(w, S);
    }

    template <bool SHIFT>
    __device__ __forceinline__ void recompute_impl(const float* __restrict__ diag, int S)
    {
        static_assert(sizeof(Tw) == 4, "only the fp32 fields are recomputed");
        long long acc[V];
#pragma unroll
        for (int v = 0; v < V; ++v)
            acc[v] = ((valid >> v) & 1u) ? to_fixed<SHIFT>(ldx(diag + base + v), S) : 0ll;
        const uint32_t myword = word();
        const int nw = (N + 31) >> 5;
        for (int wi = 0; wi < nw; ++wi) {
            uint32_t wbits = __shfl_sync(0xffffffffu, myword, wi * P);
            while (wbits) {
                const int b = __ffs(wbits) - 1;
                wbits &= wbits - 1;
                const int j = wi * 32 + b;
                if (base < N) {
                    Tw cv[V];
                    load_row(W + (size_t)j * ldw + rowoff, cv);
#pragma unroll
                    for (int v = 0; v < V; ++v) acc[v] += to_fixed<SHIFT>(cv[v], S);
                }
            }
        }
        // energy: sum over x_i = 1 of (round(d_i 2^S) + acc_i), exact in 128 bits
        unsigned long long lo = 0;
        long long hi = 0;
#pragma unroll
        for (int v = 0; v < V; ++v) {
            if (((valid & xm) >> v) & 1u) {
                const long long t = to_fixed<SHIFT>(ldx(diag + base + v), S) + acc[v];
                const unsigned long long nlo = lo + (unsigned long long)t;
                hi += (t < 0 ? -1ll : 0ll) + (nlo < lo ? 1ll : 0ll);
                lo = nlo;
            }
            h[v] = ((valid >> v) & 1u) ? scaled_f32_of(acc[v], S) : H(0);   // padding: 0, so h is dead above
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long olo = __shfl_xor_sync(0xffffffffu, lo, o);
            const long long ohi = __shfl_xor_sync(0xffffffffu, hi, o);
            const unsigned long long nlo = lo + olo;
            hi = hi + ohi + (nlo < lo ? 1ll : 0ll);
            lo = nlo;
        }
        const long long top = (long long)((unsigned long long)hi << 32 | (lo >> 32));
        const double v = __fma_rn((double)top, 4294967296.0, (double)(uint32_t)(lo & 0xFFFFFFFFull));
        Ecur = ldexp(v, -(S + 1));
        chk = true;
    }
};

}  // namespace step_detail
}  // namespace da
