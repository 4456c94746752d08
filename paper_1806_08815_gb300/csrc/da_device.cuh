// da_device.cuh -- device-side random numbers and the fp32 exponential used
// by every annealer kernel.
//
// Random numbers (the DA's hardware generator of Sec. II is replaced by a
// counter-based one, so that any trial's draw can be computed, or skipped,
// independently):
//   Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), key = (seed_lo, seed_hi).
//   acceptance draw of trial i at step t of replica r:
//       counter (i/4, t, r, 0), output lane i%4
//   uniform choice of step t:   counter (0, t & ~3, r, 1), output lane t%4
//   replica exchange after sweep s, pair p, ladder l:  counter (p, s, l, 2), lane 0
//   u = ((word >> 8) + 1) * 2^-24, uniform on (0, 1] with 24-bit resolution.
//
// Every fp32 operation that feeds an accept decision is written with an _rn
// intrinsic so that the compiler cannot contract it into an FMA: the
// decisions are then a function of IEEE single-precision arithmetic alone.
#pragma once
#include <cstdint>

namespace da {

struct u32x4 { uint32_t x, y, z, w; };

constexpr uint32_t kPhiloxMulA = 0xD2511F53u, kPhiloxMulB = 0xCD9E8D57u;
constexpr uint32_t kPhiloxWeylA = 0x9E3779B9u, kPhiloxWeylB = 0xBB67AE85u;

// The ten round keys of a Philox key, k + r * Weyl (r = 0..9): computed once
// per thread, so that each round costs two wide multiplies and two xors.
struct PhiloxKeys {
    uint32_t a[10], b[10];
    __device__ __forceinline__ explicit PhiloxKeys(uint64_t seed)
    {
        uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
#pragma unroll
        for (int r = 0; r < 10; ++r) {
            a[r] = k0; b[r] = k1;
            k0 += kPhiloxWeylA; k1 += kPhiloxWeylB;
        }
    }
};

__device__ __forceinline__ u32x4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                               const PhiloxKeys& k)
{
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        const uint64_t pa = (uint64_t)kPhiloxMulA * c0;
        const uint64_t pb = (uint64_t)kPhiloxMulB * c2;
        const uint32_t n0 = (uint32_t)(pb >> 32) ^ c1 ^ k.a[round];
        const uint32_t n2 = (uint32_t)(pa >> 32) ^ c3 ^ k.b[round];
        c1 = (uint32_t)pb;
        c3 = (uint32_t)pa;
        c0 = n0;
        c2 = n2;
    }
    return {c0, c1, c2, c3};
}

__device__ __forceinline__ u32x4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                               uint32_t k0, uint32_t k1)
{
    const PhiloxKeys k(((uint64_t)k1 << 32) | k0);
    return philox4x32_10(c0, c1, c2, c3, k);
}

__device__ __forceinline__ uint32_t pick(const u32x4& r, int lane)
{
    return lane == 0 ? r.x : lane == 1 ? r.y : lane == 2 ? r.z : r.w;
}

// u in (0, 1]: ((w >> 8) + 1) * 2^-24 (exact in fp32).
__device__ __forceinline__ float uniform01(uint32_t w)
{
    return __fmul_rn(__uint2float_rn((w >> 8) + 1u), 5.9604644775390625e-08f);
}

// exp(x) for x <= 0 in fp32: n = rint(x log2 e); r = x - n ln2 with ln2 split
// into a 16-bit head and a tail (Cody & Waite reduction); e^r from its Taylor
// series through r^7 by Horner's rule with fused multiply-adds; the result is
// scaled by 2^n through its exponent field.  0 for x < -86.
__device__ __forceinline__ float exp_neg(float x)
{
    if (!(x >= -86.0f)) return 0.0f;
    // rint(x log2 e) by the 1.5 * 2^23 shifter: the sum rounds to an integer
    // (ties to even) and its low mantissa bits hold n.
    const float kshift = __fadd_rn(__fmul_rn(x, 1.44269504088896341f), 12582912.0f);
    const float n = __fsub_rn(kshift, 12582912.0f);
    float r = __fmaf_rn(-n, 0.693145751953125f, x);
    r = __fmaf_rn(-n, 1.428606765330187e-06f, r);
    float p = 1.0f / 5040.0f;
    p = __fmaf_rn(p, r, 1.0f / 720.0f);
    p = __fmaf_rn(p, r, 1.0f / 120.0f);
    p = __fmaf_rn(p, r, 1.0f / 24.0f);
    p = __fmaf_rn(p, r, 1.0f / 6.0f);
    p = __fmaf_rn(p, r, 0.5f);
    p = __fmaf_rn(p, r, 1.0f);
    p = __fmaf_rn(p, r, 1.0f);
    const int ni = __float_as_int(kshift) - 0x4B400000;
    const float scale = __int_as_float((ni + 127) << 23);
    return __fmul_rn(p, scale);
}

// The Metropolis test u < exp_neg(x), x = -beta delta, as the step kernels
// make it, in the log domain: every trial's draw is kept as Lg = log2 U
// (hardware approximation, lg2_draw), U = (w >> 8) + 1 in [1, 2^24], and the
// annealer forms s = delta beta log2(e) + Lg with one fused multiply-add and
// t = s - 24 (exact wherever |t| < 12).  u < exp(-beta delta) is t < 0 up to
// the error of Lg, of exp_neg and of the roundings of beta log2(e) and of s,
// together far below 2^-15 for every argument (the tests bound each term); so
// t < -kLogBand accepts, t > kLogBand rejects, and only trials with
// |t| <= kLogBand (and delta <= 0 trials among them) take the exact test
// delta <= 0 || u < exp_neg(x).
constexpr float kLog2e = 1.44269504088896341f;
constexpr float kLogBand = 3.0517578125e-05f;   // 2^-15

__device__ __forceinline__ float lg2_draw(uint32_t w)
{
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(__uint2float_rn((w >> 8) + 1u)));
    return y;
}

// Arguments at or below this give exp_neg(x) <= 2^-24, which no u in (0, 1]
// is below: such trials are rejected without drawing u (checked
// exhaustively over all fp32 values in [-104, -16.7] by the tests).
constexpr float kExpCut = -16.7f;

}  // namespace da
