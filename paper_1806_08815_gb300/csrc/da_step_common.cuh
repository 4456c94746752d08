// da_step_common.cuh -- arithmetic and warp helpers shared by the step
// kernels (da_step.cuh, da_replica.cuh, da_batch.cu).
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
    static __device__ __forceinline__ float delta0(H dE) { return __int2float_rn(dE); }   // delta at E_off = +0
    static __device__ __forceinline__ H apply(H h, int8_t w, bool minus) { return minus ? h - (H)w : h + (H)w; }
    using Sign = int32_t;
    static __device__ __forceinline__ Sign sign(uint32_t xold) { return xold ? -1 : 1; }
    static __device__ __forceinline__ H apply_signed(H h, int8_t w, Sign s) { return h + s * (H)w; }
    static __device__ __forceinline__ E load_e(long long b) { return b; }
    static __device__ __forceinline__ long long store_e(E e) { return e; }
    static __device__ __forceinline__ E book(E e, H dE) { return e + (E)dE; }
};
// 16-bit integer couplings (the DA's fixed-point precision): as int8, wider W.
template <> struct Arith<int16_t> {
    using H = int32_t;
    using E = long long;
    static __device__ __forceinline__ H signed_field(H g, uint32_t x) { return x ? -g : g; }
    static __device__ __forceinline__ float delta(H dE, float Eoff) { return __fsub_rn(__int2float_rn(dE), Eoff); }
    static __device__ __forceinline__ float delta0(H dE) { return __int2float_rn(dE); }
    static __device__ __forceinline__ H apply(H h, int16_t w, bool minus) { return minus ? h - (H)w : h + (H)w; }
    using Sign = int32_t;
    static __device__ __forceinline__ Sign sign(uint32_t xold) { return xold ? -1 : 1; }
    static __device__ __forceinline__ H apply_signed(H h, int16_t w, Sign s) { return h + s * (H)w; }
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
    static __device__ __forceinline__ float delta0(H dE) { return dE; }   // dE - (+0) = dE, also for dE = -0
    static __device__ __forceinline__ H apply(H h, float w, bool minus) { return minus ? __fsub_rn(h, w) : __fadd_rn(h, w); }
    using Sign = float;
    static __device__ __forceinline__ Sign sign(uint32_t xold) { return xold ? -1.0f : 1.0f; }
    // h + s w with s = +-1: the product is exact, so this is the same single
    // rounding as __fadd_rn / __fsub_rn
    static __device__ __forceinline__ H apply_signed(H h, float w, Sign s) { return __fmaf_rn(s, w, h); }
    static __device__ __forceinline__ E load_e(long long b) { return __longlong_as_double(b); }
    static __device__ __forceinline__ long long store_e(E e) { return __double_as_longlong(e); }
    static __device__ __forceinline__ E book(E e, H dE) { return __dadd_rn(e, (double)dE); }
};

// Integer couplings of a DA_INT8 instance stored as fp32 (exact: |W| <= 128 and
// every |Q_ii| + sum_j |Q_ij| < 2^24, so every field and Delta E is an exact
// fp32 integer): the step runs on fp32 fields and FFMA updates, with exactly
// the values of the int8/int32 form, and books the energy in int64.
struct f32e {
    float f;
};
template <> struct Arith<f32e> {
    using H = float;
    using E = long long;
    static __device__ __forceinline__ H signed_field(H g, uint32_t x) { return Arith<float>::signed_field(g, x); }
    static __device__ __forceinline__ float delta(H dE, float Eoff) { return __fsub_rn(dE, Eoff); }
    static __device__ __forceinline__ float delta0(H dE) { return dE; }
    using Sign = float;
    static __device__ __forceinline__ Sign sign(uint32_t xold) { return xold ? -1.0f : 1.0f; }
    static __device__ __forceinline__ H apply_signed(H h, f32e w, Sign s) { return __fmaf_rn(s, w.f, h); }
    static __device__ __forceinline__ E load_e(long long b) { return b; }
    static __device__ __forceinline__ long long store_e(E e) { return e; }
    static __device__ __forceinline__ E book(E e, H dE) { return e + (E)__float2int_rn(dE); }
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

// h[vk] for a warp-uniform vk, as one switch instead of V selects.
template <typename H, int V>
__device__ __forceinline__ H select_slot(const H (&h)[V], int vk)
{
#define DA_SLOT(n) \
    case n:        \
        if constexpr (V > n) return h[n]; else return h[0];
    switch (vk) {
        DA_SLOT(0) DA_SLOT(1) DA_SLOT(2) DA_SLOT(3) DA_SLOT(4) DA_SLOT(5) DA_SLOT(6) DA_SLOT(7)
        DA_SLOT(8) DA_SLOT(9) DA_SLOT(10) DA_SLOT(11) DA_SLOT(12) DA_SLOT(13) DA_SLOT(14) DA_SLOT(15)
        DA_SLOT(16) DA_SLOT(17) DA_SLOT(18) DA_SLOT(19) DA_SLOT(20) DA_SLOT(21) DA_SLOT(22) DA_SLOT(23)
        DA_SLOT(24) DA_SLOT(25) DA_SLOT(26) DA_SLOT(27) DA_SLOT(28) DA_SLOT(29) DA_SLOT(30) DA_SLOT(31)
    default: return h[0];
    }
#undef DA_SLOT
}

__device__ __forceinline__ void group_barrier(int id, int nthreads)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// Loads of instance data through the read-only path: a kernel's inputs are
// fixed while it runs.
template <typename T>
__device__ __forceinline__ T ldx(const T* p)
{
    return __ldg(p);
}

// Row k of W at the V consecutive entries of this lane (16-byte loads where
// the lane's slice allows).  load() reads global memory through the read-only
// path; load_shared() reads a copy of W staged in shared memory (fp32 forms
// only).
template <typename Tw, int V> struct Row;
template <int V> struct Row<float, V> {
    static __device__ __forceinline__ void load(const float* p, float (&c)[V])
    {
        static_assert(V % 4 == 0, "V");
#pragma unroll
        for (int q = 0; q < V / 4; ++q) {
            const float4 f = ldx(reinterpret_cast<const float4*>(p) + q);
            c[4 * q] = f.x; c[4 * q + 1] = f.y; c[4 * q + 2] = f.z; c[4 * q + 3] = f.w;
        }
    }
};
template <int V> struct Row<f32e, V> {
    static __device__ __forceinline__ void load(const f32e* p, f32e (&c)[V])
    {
        static_assert(V % 4 == 0, "V");
#pragma unroll
        for (int q = 0; q < V / 4; ++q) {
            const float4 f = ldx(reinterpret_cast<const float4*>(p) + q);
            c[4 * q].f = f.x; c[4 * q + 1].f = f.y; c[4 * q + 2].f = f.z; c[4 * q + 3].f = f.w;
        }
    }
};

// Row k of W in the warp row order (step_uses_coal in da_internal.h): p points at
// entry 4 l of the warp's 32 V-entry slice of the row (lane l); float4 number q, at
// p + 128 q, holds the lane's slots 4 q .. 4 q + 3.  Every load instruction of the
// warp reads 512 contiguous bytes.
template <typename Tw, int V> struct RowCoal;
template <int V> struct RowCoal<float, V> {
    static __device__ __forceinline__ void load(const float* p, float (&c)[V])
    {
        static_assert(V % 4 == 0, "V");
#pragma unroll
        for (int q = 0; q < V / 4; ++q) {
            const float4 f = ldx(reinterpret_cast<const float4*>(p + 128 * q));
            c[4 * q] = f.x; c[4 * q + 1] = f.y; c[4 * q + 2] = f.z; c[4 * q + 3] = f.w;
        }
    }
};
template <int V> struct RowCoal<f32e, V> {
    static __device__ __forceinline__ void load(const f32e* p, f32e (&c)[V])
    {
        static_assert(V % 4 == 0, "V");
        const float* pf = reinterpret_cast<const float*>(p);
#pragma unroll
        for (int q = 0; q < V / 4; ++q) {
            const float4 f = ldx(reinterpret_cast<const float4*>(pf + 128 * q));
            c[4 * q].f = f.x; c[4 * q + 1].f = f.y; c[4 * q + 2].f = f.z; c[4 * q + 3].f = f.w;
        }
    }
};

// 16-byte loads from shared memory (p points into the block's staged copy).
template <typename Tw, int V> struct RowShared {
    static __device__ __forceinline__ void load(const Tw* p, Tw (&c)[V])
    {
        static_assert(sizeof(Tw) == 4 && V % 4 == 0, "fp32 forms only");
        const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
#pragma unroll
        for (int q = 0; q < V / 4; ++q) {
            float x, y, z, w;
            asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                         : "=f"(x), "=f"(y), "=f"(z), "=f"(w)
                         : "r"(a + 16u * q)
                         : "memory");
            reinterpret_cast<float*>(&c[4 * q])[0] = x;
            reinterpret_cast<float*>(&c[4 * q + 1])[0] = y;
            reinterpret_cast<float*>(&c[4 * q + 2])[0] = z;
            reinterpret_cast<float*>(&c[4 * q + 3])[0] = w;
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
            unpack(ldx(reinterpret_cast<const unsigned int*>(p)), c);
        } else if constexpr (V == 8) {
            const uint2 u = ldx(reinterpret_cast<const uint2*>(p));
            unpack(u.x, c); unpack(u.y, c + 4);
        } else {
#pragma unroll
            for (int q = 0; q < V / 16; ++q) {
                const uint4 u = ldx(reinterpret_cast<const uint4*>(p) + q);
                unpack(u.x, c + 16 * q); unpack(u.y, c + 16 * q + 4);
                unpack(u.z, c + 16 * q + 8); unpack(u.w, c + 16 * q + 12);
            }
        }
    }
};

template <int V> struct Row<int16_t, V> {
    static __device__ __forceinline__ void unpack(uint32_t u, int16_t* c)
    {
        c[0] = (int16_t)(u & 0xFFFFu);
        c[1] = (int16_t)(u >> 16);
    }
    static __device__ __forceinline__ void load(const int16_t* p, int16_t (&c)[V])
    {
        if constexpr (V == 4) {
            const uint2 u = ldx(reinterpret_cast<const uint2*>(p));
            unpack(u.x, c); unpack(u.y, c + 2);
        } else {
#pragma unroll
            for (int q = 0; q < V / 8; ++q) {
                const uint4 u = ldx(reinterpret_cast<const uint4*>(p) + q);
                unpack(u.x, c + 8 * q); unpack(u.y, c + 8 * q + 2);
                unpack(u.z, c + 8 * q + 4); unpack(u.w, c + 8 * q + 6);
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
// Per (G, V): as Occupancy<G>, except G = 4 with V = 32, whose 32 fields per lane need
// more registers than 7 blocks of 4 warps per SM leave (3 blocks: 12 warps per SM).
template <int G, int V> struct OccupancyGV {
    static constexpr int rpb = Occupancy<G>::rpb, min_blocks = Occupancy<G>::min_blocks;
};
template <> struct OccupancyGV<4, 32> { static constexpr int rpb = 1, min_blocks = 3; };

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

// Trials (a)-(b) of one lane's V variables in the log domain (lg2_draw,
// kLogBand in da_device.cuh): returns the mask of surely accepted trials and
// sets `unsure` when any trial has |t| <= kLogBand and must take the exact
// test (decide_exact).  With E_off = +0 (no offset, or no step without a flip
// since the last one) the subtraction is left out: it would return delta
// unchanged.
// The test is made on t' = s - (24 - kLogBand), s = fma(delta, c, L), instead of
// t = s - 24: wherever |t| < 12, s lies in [12, 36] and both subtractions are
// exact (Sterbenz), so t' = t + kLogBand and
//   t < -kLogBand  <=>  t' < 0      (its sign bit; t' = +0 when t = -kLogBand),
//   |t| <= kLogBand <=> 0 <= t' <= 2 kLogBand (its bits as an unsigned integer
//                       at most those of 2^-14: negative t' have bit 31 set);
// elsewhere both sides agree on a sign far from the band.  The sign bits are
// shifted into the mask and the band is one unsigned minimum per trial; pairs of
// trials share one packed fma and one packed add (each lane of a packed
// operation rounds as the scalar one).
template <typename A, int V>
__device__ __forceinline__ uint32_t decide_log(const typename A::H (&h)[V], uint32_t xm, float Eoff, float c,
                                               const float (&L)[V], bool& unsure)
{
    static_assert(V % 2 == 0, "trials are decided in pairs");
    constexpr float kShift = 24.0f - kLogBand;   // 23.999969482421875, exact in fp32
    constexpr uint32_t kBandBits = 0x38800000u;  // 2^-14 = 2 kLogBand
    const float2 cc = make_float2(c, c), sh = make_float2(-kShift, -kShift);
    uint32_t acc = 0, umin = 0xffffffffu;
    auto pair = [&](int v, float d0, float d1) {
        const float2 tp = __fadd2_rn(__ffma2_rn(make_float2(d0, d1), cc, make_float2(L[v], L[v + 1])), sh);
        const uint32_t b0 = __float_as_uint(tp.x), b1 = __float_as_uint(tp.y);
        acc = __funnelshift_l(b1, acc, 1);       // bit v + 1, then bit v
        acc = __funnelshift_l(b0, acc, 1);
        umin = min(umin, min(b0, b1));
    };
    if (Eoff == 0.0f) {
#pragma unroll
        for (int v = V - 2; v >= 0; v -= 2)
            pair(v, A::delta0(A::signed_field(h[v], (xm >> v) & 1u)),
                 A::delta0(A::signed_field(h[v + 1], (xm >> (v + 1)) & 1u)));
    } else {
#pragma unroll
        for (int v = V - 2; v >= 0; v -= 2)
            pair(v, A::delta(A::signed_field(h[v], (xm >> v) & 1u), Eoff),
                 A::delta(A::signed_field(h[v + 1], (xm >> (v + 1)) & 1u), Eoff));
    }
    unsure = umin <= kBandBits;
    return acc;
}

// The trials of this lane with |t| <= kLogBand, decided by the exact test
// delta <= 0 || u < exp_neg(-beta delta) with u from the trial's Philox word
// (recomputed: block (i/4, t, rep, 0), lane i%4 for variable i = base + v).
template <typename A, int V, class Keys>
__device__ __forceinline__ uint32_t decide_exact(const typename A::H (&h)[V], uint32_t xm, float Eoff, float beta,
                                                 const float (&L)[V], uint32_t acc, int base, uint32_t step,
                                                 uint32_t rep, const Keys& keys)
{
    const float c = __fmul_rn(beta, kLog2e);
    uint32_t band = 0;
#pragma unroll
    for (int v = 0; v < V; ++v) {
        const float t = __fsub_rn(__fmaf_rn(A::delta(A::signed_field(h[v], (xm >> v) & 1u), Eoff), c, L[v]), 24.0f);
        band |= (uint32_t)(fabsf(t) <= kLogBand) << v;
    }
    while (band) {
        const int v = __ffs(band) - 1;
        band &= band - 1;
        const float delta = A::delta(A::signed_field(select_slot<typename A::H, V>(h, v), (xm >> v) & 1u), Eoff);
        const float ax = -__fmul_rn(beta, delta);
        const uint32_t wd = pick(philox4x32_10((uint32_t)((base + v) >> 2), step, rep, 0u, keys), v & 3);
        acc |= (uint32_t)(delta <= 0.0f || uniform01(wd) < exp_neg(ax)) << v;
    }
    return acc;
}

}  // namespace step_detail
}  // namespace da
