// da_tune.cpp -- host-side statistics of the benchmarking method (Sec. IV):
// the bootstrap distribution of the q-th percentile of the time to solution
// over a set of instances (Algorithm 3), and percentiles of the single-flip
// energy changes that set the temperature grid (appendix, "Parameters").
//
// The bootstrap draws every random number from Philox4x32-10 (Salmon et al.,
// SC'11) keyed by the caller's seed, block (b, j, k, 6) for resample b,
// sampled instance j and the k-th block of that pair's stream, so a result
// depends only on its inputs.  Compiled without floating-point contraction:
// the arithmetic is the IEEE double sequence written here.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <string>
#include <vector>

#include "da.h"
#include "da_internal.h"

namespace {

struct Philox {
    uint32_t k0, k1;
    void block(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t out[4]) const
    {
        uint32_t a = k0, b = k1;
        for (int r = 0; r < 10; ++r) {
            const uint64_t p0 = (uint64_t)0xD2511F53u * c0;
            const uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
            const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ a;
            const uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ b;
            c1 = (uint32_t)p1;
            c3 = (uint32_t)p0;
            c0 = n0;
            c2 = n2;
            a += 0x9E3779B9u;
            b += 0xBB67AE85u;
        }
        out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
    }
};

// The uniform stream of one (resample, instance) pair: doubles in (0, 1) with
// 53 random bits from two consecutive 32-bit words.
struct Stream {
    const Philox* ph;
    uint32_t b, j, k = 0;
    uint32_t w[4];
    int used = 4;
    uint32_t word()
    {
        if (used == 4) {
            ph->block(b, j, k++, 6u, w);
            used = 0;
        }
        return w[used++];
    }
    double uniform()
    {
        const uint64_t hi = word() >> 5, lo = word() >> 6;   // 27 + 26 bits
        return ((double)((hi << 26) | lo) + 0.5) * 0x1.0p-53;
    }
    double normal()   // Box-Muller, first variate of the pair
    {
        const double u1 = uniform(), u2 = uniform();
        return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
    }
    // Gamma(a, 1) by Marsaglia & Tsang (2000) for a >= 1; for a < 1 the draw of
    // Gamma(a + 1) is scaled by u^(1/a).  The rejection loop accepts with
    // probability above 0.95; after 1000 rejections the last candidate is
    // returned.
    double gamma(double a)
    {
        if (a < 1.0) {
            const double g = gamma(a + 1.0);
            const double u = uniform();
            return g * std::exp(std::log(u) / a);
        }
        const double d = a - 1.0 / 3.0;
        const double c = 1.0 / std::sqrt(9.0 * d);
        double v = 1.0;
        for (int it = 0; it < 1000; ++it) {
            const double x = normal();
            const double t = 1.0 + c * x;
            if (t <= 0.0) continue;
            v = t * t * t;
            const double u = uniform();
            if (std::log(u) < 0.5 * x * x + d - d * v + d * std::log(v)) return d * v;
        }
        return d * v;
    }
};

// q-th percentile (0..100) of v by linear interpolation between the order
// statistics at position (n - 1) q / 100.
double percentile(std::vector<double>& v, double q)
{
    const size_t n = v.size();
    std::sort(v.begin(), v.end());
    const double pos = (double)(n - 1) * q / 100.0;
    const size_t lo = (size_t)std::floor(pos);
    const size_t hi = std::min(lo + 1, n - 1);
    const double f = pos - (double)lo;
    return v[lo] + f * (v[hi] - v[lo]);
}

}  // namespace

extern "C" da_status da_tts_bootstrap(const int64_t* hits, const int64_t* runs, int32_t I, double tau, double q,
                                      int32_t B, uint64_t seed, double* tts_q)
{
    if (!hits || !runs || !tts_q || I < 1 || B < 1 || !(q >= 0.0 && q <= 100.0) || !(tau >= 0.0)) {
        da::set_last_error("da_tts_bootstrap: need I >= 1, B >= 1, 0 <= q <= 100, tau >= 0 and the arrays");
        return DA_EINVAL;
    }
    for (int32_t i = 0; i < I; ++i)
        if (runs[i] < 1 || hits[i] < 0 || hits[i] > runs[i]) {
            da::set_last_error("da_tts_bootstrap: need 0 <= hits <= runs and runs >= 1 for every instance");
            return DA_EINVAL;
        }
    const Philox ph{(uint32_t)seed, (uint32_t)(seed >> 32)};
    const double log_miss = std::log(1.0 - 0.99);
    std::vector<double> r99((size_t)I);
    for (int32_t b = 0; b < B; ++b) {
        for (int32_t j = 0; j < I; ++j) {
            Stream s{&ph, (uint32_t)b, (uint32_t)j};
            int64_t idx = (int64_t)(s.uniform() * (double)I);
            if (idx >= I) idx = I - 1;
            const double x = s.gamma(0.5 + (double)hits[idx]);
            const double y = s.gamma(0.5 + (double)(runs[idx] - hits[idx]));
            const double p = x / (x + y);
            double r = p >= 1.0 ? 1.0 : log_miss / std::log(1.0 - p);
            if (!(r >= 1.0)) r = 1.0;   // at least one run (p > 0.99, or p = 1)
            r99[(size_t)j] = r;
        }
        tts_q[b] = tau * percentile(r99, q);
    }
    return DA_OK;
}

extern "C" da_status da_percentiles(const double* v, int64_t n, const double* q, int32_t nq, double* out)
{
    if (!v || !q || !out || n < 1 || nq < 0) {
        da::set_last_error("da_percentiles: need n >= 1 and the arrays");
        return DA_EINVAL;
    }
    std::vector<double> w(v, v + n);
    for (int32_t k = 0; k < nq; ++k) {
        if (!(q[k] >= 0.0 && q[k] <= 100.0)) {
            da::set_last_error("da_percentiles: q outside [0, 100]");
            return DA_EINVAL;
        }
        out[k] = percentile(w, q[k]);
    }
    return DA_OK;
}
