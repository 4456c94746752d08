/*
 * da_oracle.c -- plain serial CPU reference of the Digital Annealer method
 * (arXiv:1806.08815).  TEST INFRASTRUCTURE: only the tests, the smoke check
 * and the benchmark's CPU-baseline leg load this library; it shares nothing
 * with the CUDA path.  Build: gcc -O2 -std=c11 -ffp-contract=off -fopenmp
 * -shared -fPIC (no fast-math: every fp32 operation below is one IEEE
 * rounding, which is what makes the fp32 trajectories reproducible).
 *
 * Readings of the paper used here (the paper gives no formulas for them):
 *  - Delta E of flipping x_i: (1 - 2 x_i)(Q_ii + h_i), h_i = sum_j W_ij x_j.
 *  - Metropolis with the dynamic offset (Algorithm 2): a trial with
 *    delta = Delta E - E_off is accepted when delta <= 0 (the clipped
 *    min(1, .)), otherwise when u < exp(-beta * delta) (Sec. III).
 *  - E_off = m * inc after m consecutive steps without an accepted flip; it
 *    returns to 0 after a flip (Algorithm 2).
 *  - "choose one flip uniformly at random" (Algorithm 2): j = floor(u32 * cnt
 *    / 2^32) and the j-th accepted index in increasing index order.
 *  - All runs start from x = 0, so h = 0 and E = 0 (Sec. II, DA parameters).
 *  - Random numbers: Philox4x32-10 keyed by the seed; the paper's hardware
 *    generator (Sec. II) is replaced by this counter-based one.
 * parity unpinned: none (every function here is pinned by tests/test_oracle*.py).
 */
#include "da_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* Philox4x32-10: Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as
 * easy as 1, 2, 3", SC'11.  Ten rounds of the 4x32 Philox S-box; the key is
 * bumped by the Weyl constants between rounds. */
#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)PHILOX_M0 * c0;
        uint64_t p1 = (uint64_t)PHILOX_M1 * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += PHILOX_W0;
        k1 += PHILOX_W1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static uint32_t philox_word(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, int lane)
{
    uint32_t ctr[4] = {c0, c1, c2, c3};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t out[4];
    orc_philox4x32_10(ctr, key, out);
    return out[lane];
}

/* The acceptance draw of trial i at step t: counter (i / 4, t, replica, 0),
 * output lane i % 4, so one Philox block serves four consecutive variables. */
static uint32_t draw_accept(uint64_t seed, int64_t i, uint32_t t, uint32_t rep)
{
    return philox_word(seed, (uint32_t)(i / 4), t, rep, 0u, (int)(i % 4));
}

/* The choice draw of step t: one Philox block serves four consecutive steps,
 * counter (0, t - t % 4, replica, 1), output lane t % 4. */
static uint32_t draw_choice(uint64_t seed, uint32_t t, uint32_t rep)
{
    return philox_word(seed, 0u, t & ~3u, rep, 1u, (int)(t & 3u));
}

float orc_uniform(uint32_t r)
{
    return (float)((r >> 8) + 1u) * 5.9604644775390625e-08f; /* 2^-24 */
}

/* ------------------------------------------------------------------------ */
/* exp in fp32.  x = n ln2 + r with n = rint(x / ln2) and ln2 split into a
 * short head and a tail (Cody & Waite); e^r by its Taylor series to r^7 in
 * Horner form with fused multiply-adds; then the exponent is set directly. */
float orc_expf(float x)
{
    if (!(x >= -86.0f))
        return 0.0f;
    const float log2e = 1.44269504088896341f;
    const float ln2_head = 0.693145751953125f;      /* ln 2 to 16 bits */
    const float ln2_tail = 1.428606765330187e-06f;  /* ln 2 - head     */
    float n = rintf(x * log2e);
    float r = fmaf(-n, ln2_head, x);
    r = fmaf(-n, ln2_tail, r);
    float p = 1.0f / 5040.0f;
    p = fmaf(p, r, 1.0f / 720.0f);
    p = fmaf(p, r, 1.0f / 120.0f);
    p = fmaf(p, r, 1.0f / 24.0f);
    p = fmaf(p, r, 1.0f / 6.0f);
    p = fmaf(p, r, 0.5f);
    p = fmaf(p, r, 1.0f);
    p = fmaf(p, r, 1.0f);
    int e = (int)n + 127;
    union { uint32_t u; float f; } s;
    s.u = (uint32_t)e << 23;
    return p * s.f;
}

void orc_expf_batch(const float* x, float* y, int64_t n)
{
    for (int64_t i = 0; i < n; ++i)
        y[i] = orc_expf(x[i]);
}

/* ------------------------------------------------------------------------ */
static inline int getbit(const uint32_t* x, int64_t i) { return (int)((x[i >> 5] >> (i & 31)) & 1u); }

int64_t orc_energy_int(int64_t N, const int32_t* Q, const uint32_t* x)
{
    int64_t E = 0;
    for (int64_t i = 0; i < N; ++i) {
        if (!getbit(x, i)) continue;
        E += Q[i * N + i];
        for (int64_t j = i + 1; j < N; ++j)
            if (getbit(x, j)) E += Q[i * N + j];
    }
    return E;
}

double orc_energy_f64(int64_t N, const float* Q, const uint32_t* x)
{
    double E = 0.0;
    for (int64_t i = 0; i < N; ++i) {
        if (!getbit(x, i)) continue;
        E += (double)Q[i * N + i];
        for (int64_t j = i + 1; j < N; ++j)
            if (getbit(x, j)) E += (double)Q[i * N + j];
    }
    return E;
}

/* H = -sum_{i<j} J_ij s_i s_j - sum_i hb_i s_i (Eq. 4).  With s = 2x - 1,
 * s_i s_j = 4 x_i x_j - 2 x_i - 2 x_j + 1, which gives the coefficients
 * below. */
int orc_ising_to_qubo(int64_t N, const double* J, const double* hb, double* Q, double* C)
{
    if (N < 1) return -1;
    double c = 0.0;
    for (int64_t i = 0; i < N * N; ++i) Q[i] = 0.0;
    for (int64_t i = 0; i < N; ++i) {
        Q[i * N + i] = -2.0 * hb[i];
        c += hb[i];
    }
    for (int64_t i = 0; i < N; ++i)
        for (int64_t j = i + 1; j < N; ++j) {
            double Jij = J[i * N + j];
            Q[i * N + j] = -4.0 * Jij;
            Q[i * N + i] += 2.0 * Jij;
            Q[j * N + j] += 2.0 * Jij;
            c -= Jij;
        }
    *C = c;
    return 0;
}

double orc_ising_energy(int64_t N, const double* J, const double* hb, const int8_t* s)
{
    double H = 0.0;
    for (int64_t i = 0; i < N; ++i) {
        H -= hb[i] * s[i];
        for (int64_t j = i + 1; j < N; ++j)
            H -= J[i * N + j] * s[i] * s[j];
    }
    return H;
}

int orc_brute_force_f64(int64_t N, const double* Q, double* Emin, int64_t* count, uint32_t* argmin)
{
    if (N < 1 || N > 30) return -1;
    double* h = (double*)calloc((size_t)N, sizeof(double));
    if (!h) return -2;
    uint32_t x = 0;
    double E = 0.0, best = 0.0;
    int64_t nbest = 1;
    uint32_t arg = 0;
    const uint64_t total = 1ull << N;
    for (uint64_t k = 1; k < total; ++k) {
        int i = __builtin_ctzll(k);               /* Gray code: flip bit i */
        int xi = (int)((x >> i) & 1u);
        double dE = (xi ? -1.0 : 1.0) * (Q[i * N + i] + h[i]);
        E += dE;
        x ^= 1u << i;
        double s = xi ? -1.0 : 1.0;
        for (int64_t j = 0; j < N; ++j) {
            if (j == i) continue;
            double w = (j < i) ? Q[j * N + i] : Q[i * N + j];
            h[j] += s * w;
        }
        double tol = 1e-9 * (fabs(best) + 1.0);
        if (E < best - tol) { best = E; nbest = 1; arg = x; }
        else if (fabs(E - best) <= tol) nbest++;
    }
    free(h);
    *Emin = best;
    *count = nbest;
    argmin[0] = arg;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Instance in the form the annealer reads: symmetric W and diagonal d. */
typedef struct {
    int64_t N;
    int mode;
    int64_t* Wi; int64_t* di;   /* ORC_MODE_INT */
    float* Wf; float* df;       /* ORC_MODE_F32 / ORC_MODE_F64 */
} inst_t;

static void inst_free(inst_t* I)
{
    free(I->Wi); free(I->di); free(I->Wf); free(I->df);
}

static int inst_make(inst_t* I, int64_t N, int mode, const void* Q)
{
    memset(I, 0, sizeof(*I));
    I->N = N; I->mode = mode;
    if (mode == ORC_MODE_INT) {
        const int32_t* Qi = (const int32_t*)Q;
        I->Wi = (int64_t*)calloc((size_t)(N * N), sizeof(int64_t));
        I->di = (int64_t*)calloc((size_t)N, sizeof(int64_t));
        if (!I->Wi || !I->di) { inst_free(I); return -2; }
        for (int64_t i = 0; i < N; ++i) {
            I->di[i] = Qi[i * N + i];
            for (int64_t j = i + 1; j < N; ++j) {
                I->Wi[i * N + j] = Qi[i * N + j];
                I->Wi[j * N + i] = Qi[i * N + j];
            }
        }
    } else {
        const float* Qf = (const float*)Q;
        I->Wf = (float*)calloc((size_t)(N * N), sizeof(float));
        I->df = (float*)calloc((size_t)N, sizeof(float));
        if (!I->Wf || !I->df) { inst_free(I); return -2; }
        for (int64_t i = 0; i < N; ++i) {
            I->df[i] = Qf[i * N + i];
            for (int64_t j = i + 1; j < N; ++j) {
                I->Wf[i * N + j] = Qf[i * N + j];
                I->Wf[j * N + i] = Qf[i * N + j];
            }
        }
    }
    return 0;
}

int orc_fields_int(int64_t N, const int32_t* Q, const uint32_t* x, int64_t* h)
{
    if (N < 1) return -1;
    for (int64_t i = 0; i < N; ++i) {
        int64_t s = 0;
        for (int64_t j = 0; j < N; ++j) {
            if (j == i || !getbit(x, j)) continue;
            s += (j < i) ? Q[j * N + i] : Q[i * N + j];
        }
        h[i] = s;
    }
    return 0;
}

/* Fixed-point scale of the recompute: with max(|W_ij|, |Q_ii|) < 2^e and
 * 2^L >= N + 1, S = 62 - L - e puts every |W_ij| 2^S and |Q_ii| 2^S below
 * 2^(62-L), so the sum of a linear term and N couplings cannot overflow int64. */
static int32_t fix_scale(int64_t N, const float* Wf, const float* df)
{
    float amax = 0.0f;
    for (int64_t i = 0; i < N * N; ++i) {
        float a = fabsf(Wf[i]);
        if (a > amax) amax = a;
    }
    for (int64_t i = 0; i < N; ++i) {
        float a = fabsf(df[i]);
        if (a > amax) amax = a;
    }
    if (amax == 0.0f) return 0;
    int e;
    frexpf(amax, &e);
    int L = 0;
    while ((1ll << L) < N + 1) L++;
    return 62 - L - e;
}

/* sums_i = round(Q_ii 2^S) + sum_{j: x_j = 1} round(W_ij 2^S), exactly. */
static void recompute_sums(const inst_t* I, int32_t S, const uint8_t* x, int64_t* sums)
{
    const int64_t N = I->N;
    for (int64_t i = 0; i < N; ++i) {
        int64_t s = (int64_t)llrintf(ldexpf(I->df[i], S));
        for (int64_t j = 0; j < N; ++j)
            if (x[j]) s += (int64_t)llrintf(ldexpf(I->Wf[i * N + j], S));
        sums[i] = s;
    }
}

/* The energy that goes with the recompute, E = sum_{x_i = 1} (Q_ii + g_i) / 2
 * with g_i = Q_ii + sum_j W_ij x_j, summed exactly in fixed point:
 * E 2^(S+1) = sum_{x_i = 1} (round(Q_ii 2^S) + sums_i), an integer below 2^76
 * held in __int128, then rounded once to fp64 (its top and bottom parts
 * recombined with one fused multiply-add) and scaled by 2^-(S+1). */
static double recompute_energy(const inst_t* I, int32_t S, const uint8_t* x, const int64_t* sums)
{
    __int128 acc = 0;
    for (int64_t i = 0; i < I->N; ++i) {
        if (!x[i]) continue;
        acc += (__int128)((int64_t)llrintf(ldexpf(I->df[i], S)) + sums[i]);
    }
    const int64_t top = (int64_t)(acc >> 32);
    const uint32_t bottom = (uint32_t)(acc & 0xFFFFFFFF);
    const double v = fma((double)top, 4294967296.0, (double)bottom);
    return ldexp(v, -(S + 1));
}

int orc_recompute_f32(int64_t N, const float* Q, const uint32_t* x, float* h, int64_t* sums, int32_t* S_out)
{
    if (N < 1) return -1;
    inst_t I;
    if (inst_make(&I, N, ORC_MODE_F32, Q)) return -2;
    int32_t S = fix_scale(N, I.Wf, I.df);
    uint8_t* xb = (uint8_t*)malloc((size_t)N);
    int64_t* s = (int64_t*)malloc((size_t)N * sizeof(int64_t));
    for (int64_t i = 0; i < N; ++i) xb[i] = (uint8_t)getbit(x, i);
    recompute_sums(&I, S, xb, s);
    for (int64_t i = 0; i < N; ++i) {
        if (h) h[i] = ldexpf((float)s[i], -S);
        if (sums) sums[i] = s[i];
    }
    if (S_out) *S_out = S;
    free(xb); free(s); inst_free(&I);
    return 0;
}

double orc_recompute_energy_f32(int64_t N, const float* Q, const uint32_t* x)
{
    inst_t I;
    if (N < 1 || inst_make(&I, N, ORC_MODE_F32, Q)) return NAN;
    int32_t S = fix_scale(N, I.Wf, I.df);
    uint8_t* xb = (uint8_t*)malloc((size_t)N);
    int64_t* s = (int64_t*)malloc((size_t)N * sizeof(int64_t));
    for (int64_t i = 0; i < N; ++i) xb[i] = (uint8_t)getbit(x, i);
    recompute_sums(&I, S, xb, s);
    double E = recompute_energy(&I, S, xb, s);
    free(xb); free(s); inst_free(&I);
    return E;
}

/* ------------------------------------------------------------------------ */
/* State of one replica of the annealer. */
typedef struct {
    uint8_t* x;
    int64_t* hi;   /* ORC_MODE_INT: h_i = sum_j W_ij x_j */
    float* hf;     /* ORC_MODE_F32: effective field g_i = Q_ii + sum_j W_ij x_j */
    double* hd;    /* ORC_MODE_F64: h_i */
    int64_t Ei;    /* tracked energy, ORC_MODE_INT */
    double Ed;     /* tracked energy, real modes   */
    uint32_t m;    /* steps since the last accepted flip (dynamic offset) */
    int32_t* acc;  /* accepted indices of the current step */
} rep_t;

static int rep_init(rep_t* s, const inst_t* I)
{
    memset(s, 0, sizeof(*s));
    const int64_t N = I->N;
    s->x = (uint8_t*)calloc((size_t)N, 1);
    s->acc = (int32_t*)malloc((size_t)N * sizeof(int32_t));
    if (I->mode == ORC_MODE_INT) s->hi = (int64_t*)calloc((size_t)N, sizeof(int64_t));
    else if (I->mode == ORC_MODE_F32) {
        s->hf = (float*)calloc((size_t)N, sizeof(float));
        if (s->hf) memcpy(s->hf, I->df, (size_t)N * sizeof(float));   /* x = 0: g = diag */
    }
    else s->hd = (double*)calloc((size_t)N, sizeof(double));
    if (!s->x || !s->acc || (!s->hi && !s->hf && !s->hd)) return -2;
    return 0;
}

static void rep_free(rep_t* s)
{
    free(s->x); free(s->hi); free(s->hf); free(s->hd); free(s->acc);
}

static double tracked_energy(const inst_t* I, const rep_t* s)
{
    return I->mode == ORC_MODE_INT ? (double)s->Ei : s->Ed;
}

/* Steps (a)-(b) of the DA step: every trial against E_off; fills s->acc and
 * returns how many were accepted. */
static int32_t da_trials(const inst_t* I, rep_t* s, float beta, float inc,
                         uint64_t seed, uint32_t t, uint32_t rep)
{
    const int64_t N = I->N;
    const float E_off = (float)s->m * inc;
    int32_t cnt = 0;
    for (int64_t i = 0; i < N; ++i) {
        float delta;
        if (I->mode == ORC_MODE_INT) {
            int64_t v = I->di[i] + s->hi[i];
            int64_t dE = s->x[i] ? -v : v;
            delta = (float)dE - E_off;
        } else if (I->mode == ORC_MODE_F32) {
            float v = s->hf[i];
            float dE = s->x[i] ? -v : v;
            delta = dE - E_off;
        } else {
            double v = (double)I->df[i] + s->hd[i];
            double dE = s->x[i] ? -v : v;
            double d64 = dE - (double)E_off;
            if (d64 <= 0.0) { s->acc[cnt++] = (int32_t)i; continue; }
            float a = (float)(-(double)beta * d64);
            float p = orc_expf(a);
            if (orc_uniform(draw_accept(seed, i, t, rep)) < p) s->acc[cnt++] = (int32_t)i;
            continue;
        }
        if (delta <= 0.0f) { s->acc[cnt++] = (int32_t)i; continue; }
        float a = -(beta * delta);
        float p = orc_expf(a);
        if (orc_uniform(draw_accept(seed, i, t, rep)) < p) s->acc[cnt++] = (int32_t)i;
    }
    return cnt;
}

/* Step (c): flip x_k and update every field with the column W[:, k]. */
static void da_flip(const inst_t* I, rep_t* s, int64_t k)
{
    const int64_t N = I->N;
    const int old = s->x[k];
    if (I->mode == ORC_MODE_INT) {
        int64_t v = I->di[k] + s->hi[k];
        s->Ei += old ? -v : v;
        const int64_t sg = old ? -1 : 1;
        for (int64_t j = 0; j < N; ++j) s->hi[j] += sg * I->Wi[k * N + j];
    } else if (I->mode == ORC_MODE_F32) {
        float v = s->hf[k];
        float dE = old ? -v : v;
        s->Ed += (double)dE;
        const float sg = old ? -1.0f : 1.0f;
        for (int64_t j = 0; j < N; ++j) s->hf[j] = s->hf[j] + sg * I->Wf[k * N + j];
    } else {
        double v = (double)I->df[k] + s->hd[k];
        s->Ed += old ? -v : v;
        const double sg = old ? -1.0 : 1.0;
        for (int64_t j = 0; j < N; ++j) s->hd[j] += sg * (double)I->Wf[k * N + j];
    }
    s->x[k] = (uint8_t)(old ^ 1);
}

/* One complete step of Algorithm 2.  Returns the flipped index or -1. */
static int64_t da_step(const inst_t* I, rep_t* s, float beta, float inc,
                       uint64_t seed, uint32_t t, uint32_t rep, int32_t* n_acc)
{
    int32_t cnt = da_trials(I, s, beta, inc, seed, t, rep);
    if (n_acc) *n_acc = cnt;
    if (cnt == 0) {
        s->m += 1;
        return -1;
    }
    uint32_t u = draw_choice(seed, t, rep);
    uint32_t j = (uint32_t)(((uint64_t)u * (uint64_t)cnt) >> 32);
    int64_t k = s->acc[j];
    da_flip(I, s, k);
    s->m = 0;
    return k;
}

static void pack_bits(const uint8_t* x, int64_t N, uint32_t* out)
{
    int64_t words = (N + 31) / 32;
    for (int64_t w = 0; w < words; ++w) out[w] = 0;
    for (int64_t i = 0; i < N; ++i)
        if (x[i]) out[i >> 5] |= 1u << (i & 31);
}

/* Exact recompute of the effective fields, each rounded once to fp32. */
static void periodic_recompute(const inst_t* I, rep_t* s, int32_t S, int64_t* sums)
{
    recompute_sums(I, S, s->x, sums);
    for (int64_t i = 0; i < I->N; ++i) s->hf[i] = ldexpf((float)sums[i], -S);
    s->Ed = recompute_energy(I, S, s->x, sums);
}

int orc_da_anneal(int64_t N, int mode, const void* Q,
                  const float* beta, int64_t T, float inc, int32_t R,
                  uint64_t seed, uint32_t replica_base, int64_t recompute_every,
                  double* E_final, double* E_best, uint32_t* x_final, uint32_t* x_best,
                  int64_t* flips, int32_t* trace, int32_t* accepted, int nthreads)
{
    if (N < 1 || T < 0 || R < 0 || !Q || (T > 0 && !beta)) return -1;
    if (mode < ORC_MODE_INT || mode > ORC_MODE_F64) return -1;
    inst_t I;
    if (inst_make(&I, N, mode, Q)) return -2;
    const int32_t S = (mode == ORC_MODE_F32) ? fix_scale(N, I.Wf, I.df) : 0;
    const int64_t words = (N + 31) / 32;
    int err = 0;
#ifdef _OPENMP
    if (nthreads < 1) nthreads = 1;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
#endif
    for (int32_t r = 0; r < R; ++r) {
        rep_t s;
        uint8_t* best = (uint8_t*)calloc((size_t)N, 1);
        int64_t* sums = (int64_t*)malloc((size_t)N * sizeof(int64_t));
        if (rep_init(&s, &I) || !best || !sums) {
#ifdef _OPENMP
#pragma omp atomic write
#endif
            err = -2;
            rep_free(&s); free(best); free(sums);
            continue;
        }
        const uint32_t rep = replica_base + (uint32_t)r;
        double Ebest = 0.0;
        int64_t nflip = 0;
        for (int64_t t = 0; t < T; ++t) {
            int32_t na = 0;
            int64_t k = da_step(&I, &s, beta[t], inc, seed, (uint32_t)t, rep, &na);
            if (trace) trace[(int64_t)r * T + t] = (int32_t)k;
            if (accepted) accepted[(int64_t)r * T + t] = na;
            if (k >= 0) nflip++;
            if (mode == ORC_MODE_F32 && recompute_every > 0 && (t + 1) % recompute_every == 0)
                periodic_recompute(&I, &s, S, sums);
            double E = tracked_energy(&I, &s);
            if (E < Ebest) {
                Ebest = E;
                memcpy(best, s.x, (size_t)N);
            }
        }
        if (E_final) E_final[r] = tracked_energy(&I, &s);
        if (E_best) E_best[r] = Ebest;
        if (x_final) pack_bits(s.x, N, x_final + (int64_t)r * words);
        if (x_best) pack_bits(best, N, x_best + (int64_t)r * words);
        if (flips) flips[r] = nflip;
        rep_free(&s); free(best); free(sums);
    }
    inst_free(&I);
    return err;
}

int orc_da_one_step(int64_t N, int mode, const void* Q, const uint32_t* x, uint32_t m,
                    float beta, float inc, uint64_t seed, uint32_t t, uint32_t replica,
                    int32_t* n_accepted)
{
    if (N < 1 || !Q || !x) return -2;
    inst_t I;
    if (inst_make(&I, N, mode, Q)) return -2;
    rep_t s;
    if (rep_init(&s, &I)) { rep_free(&s); inst_free(&I); return -2; }
    for (int64_t i = 0; i < N; ++i) s.x[i] = (uint8_t)getbit(x, i);
    if (mode == ORC_MODE_F32) memcpy(s.hf, I.df, (size_t)N * sizeof(float));
    /* fields of the given state, summed in index order */
    for (int64_t i = 0; i < N; ++i)
        for (int64_t j = 0; j < N; ++j) {
            if (!s.x[j]) continue;
            if (mode == ORC_MODE_INT) s.hi[i] += I.Wi[i * N + j];
            else if (mode == ORC_MODE_F32) s.hf[i] = s.hf[i] + I.Wf[i * N + j];
            else s.hd[i] += (double)I.Wf[i * N + j];
        }
    s.m = m;
    int64_t k = da_step(&I, &s, beta, inc, seed, t, replica, n_accepted);
    rep_free(&s); inst_free(&I);
    return (int)k;
}

/* ------------------------------------------------------------------------ */
/* Algorithm 1: R runs, each from a random state; temperature t is one sweep
 * over the variables in index order, proposing single flips. */
int orc_sa_anneal(int64_t N, const float* Q, const float* beta, int64_t T, int32_t R,
                  uint64_t seed, double* E_best, uint32_t* x_best, int nthreads)
{
    if (N < 1 || T < 0 || R < 0 || !Q) return -1;
    inst_t I;
    if (inst_make(&I, N, ORC_MODE_F64, Q)) return -2;
    const int64_t words = (N + 31) / 32;
    int err = 0;
#ifdef _OPENMP
    if (nthreads < 1) nthreads = 1;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
#endif
    for (int32_t r = 0; r < R; ++r) {
        uint8_t* x = (uint8_t*)calloc((size_t)N, 1);
        uint8_t* best = (uint8_t*)calloc((size_t)N, 1);
        double* h = (double*)calloc((size_t)N, sizeof(double));
        if (!x || !best || !h) {
#ifdef _OPENMP
#pragma omp atomic write
#endif
            err = -2;
            free(x); free(best); free(h);
            continue;
        }
        for (int64_t i = 0; i < N; ++i)
            x[i] = (uint8_t)(philox_word(seed, (uint32_t)(i / 4), 0u, (uint32_t)r, 4u, (int)(i % 4)) >> 31);
        double E = 0.0;
        for (int64_t i = 0; i < N; ++i) {
            if (!x[i]) continue;
            E += (double)I.df[i];
            for (int64_t j = 0; j < N; ++j) {
                if (!x[j]) continue;
                h[i] += (double)I.Wf[i * N + j];
                if (j > i) E += (double)I.Wf[i * N + j];
            }
        }
        for (int64_t i = 0; i < N; ++i) {
            if (x[i]) continue;
            for (int64_t j = 0; j < N; ++j)
                if (x[j]) h[i] += (double)I.Wf[i * N + j];
        }
        double Ebest = E;
        memcpy(best, x, (size_t)N);
        for (int64_t t = 0; t < T; ++t) {
            for (int64_t i = 0; i < N; ++i) {
                double v = (double)I.df[i] + h[i];
                double dE = x[i] ? -v : v;
                int acc = dE <= 0.0;
                if (!acc) {
                    float a = (float)(-(double)beta[t] * dE);
                    uint32_t rw = philox_word(seed, (uint32_t)(i / 4), (uint32_t)t, (uint32_t)r, 5u, (int)(i % 4));
                    acc = orc_uniform(rw) < orc_expf(a);
                }
                if (!acc) continue;
                const double sg = x[i] ? -1.0 : 1.0;
                for (int64_t j = 0; j < N; ++j) h[j] += sg * (double)I.Wf[i * N + j];
                x[i] ^= 1;
                E += dE;
                if (E < Ebest) { Ebest = E; memcpy(best, x, (size_t)N); }
            }
        }
        if (x_best) pack_bits(best, N, x_best + (int64_t)r * words);
        if (E_best) {
            uint32_t* packed = (uint32_t*)calloc((size_t)words, sizeof(uint32_t));
            pack_bits(best, N, packed);
            E_best[r] = orc_energy_f64(N, Q, packed);
            free(packed);
        }
        free(x); free(best); free(h);
    }
    inst_free(&I);
    return err;
}

/* ------------------------------------------------------------------------ */
/* PTDA: the DA step inside every replica, replica exchange between
 * neighbouring temperatures after every sweep of N steps (Sec. II, PTDA;
 * the exchange rule is the Metropolis swap of Algorithm 4). */
/* Adaptive ladder of the PTDA (Sec. II: the temperatures follow the adaptive
 * scheme of Hukushima et al.; the highest and lowest are fixed and the
 * intermediate ones are moved so that every neighbouring pair is exchanged with
 * the same probability).  The paper gives the objective, not an update rule;
 * this one is a damped proportional feedback on the gaps: with a_p the
 * accepted and n the proposed exchanges of pair (p, p+1) over the last window,
 * each gap beta_{p+1} - beta_p is multiplied by w_p^(1/8), w_p = (a_p + 1) /
 * (n + 2) the pair's smoothed acceptance (the eighth root taken as three
 * square roots), and the gaps are rescaled to the fixed span
 * beta_{K-1} - beta_0.  Pairs accepted more often than the others are pulled
 * apart, pairs accepted less often are pushed together, equal acceptances
 * leave the ladder unchanged; the damping keeps the iteration stable for
 * acceptances down to about 1e-3, where an undamped update overshoots.
 * fp64 arithmetic in this order, rounded to fp32. */
static double gap_weight(int64_t accepted, int64_t proposals)
{
    const double w = ((double)accepted + 1.0) / ((double)proposals + 2.0);
    return sqrt(sqrt(sqrt(w)));
}

void orc_pt_adapt(int32_t K, const float* betas, const int64_t* accepted, int64_t proposals, float* out)
{
    for (int32_t k = 0; k < K; ++k) out[k] = betas[k];
    if (K < 3 || proposals < 1) return;
    double total = 0.0;
    for (int32_t p = 0; p + 1 < K; ++p) {
        const double gap = (double)betas[p + 1] - (double)betas[p];
        total = total + gap * gap_weight(accepted[p], proposals);
    }
    if (!(total > 0.0)) return;
    const double span = (double)betas[K - 1] - (double)betas[0];
    double b = (double)betas[0];
    for (int32_t p = 0; p + 2 < K; ++p) {
        const double gap = (double)betas[p + 1] - (double)betas[p];
        b = b + (gap * gap_weight(accepted[p], proposals)) * span / total;
        out[p + 1] = (float)b;
    }
}

/* One ladder of the PTDA for sweeps [s0, s1) at the ladder `b`. */
static void ptda_window(const inst_t* I, rep_t* reps, uint8_t* best, double* Ebest, int32_t* tof, int32_t* at,
                        int64_t* cnt, const float* b, int32_t K, int32_t l, int64_t s0, int64_t s1, int64_t sweeps,
                        float inc, uint64_t seed, uint8_t* swap_trace)
{
    const int64_t N = I->N;
    for (int64_t sw = s0; sw < s1; ++sw) {
        for (int32_t k = 0; k < K; ++k) {
            const float beta = b[tof[k]];
            const uint32_t rep = (uint32_t)(l * K + k);
            for (int64_t q = 0; q < N; ++q) {
                const uint32_t t = (uint32_t)(sw * N + q);
                da_step(I, &reps[k], beta, inc, seed, t, rep, NULL);
                double E = tracked_energy(I, &reps[k]);
                if (E < Ebest[k]) { Ebest[k] = E; memcpy(best + (int64_t)k * N, reps[k].x, (size_t)N); }
            }
        }
        for (int32_t p = 0; p + 1 < K; ++p) {
            const int32_t a = at[p], c = at[p + 1];
            const double arg = ((double)b[p] - (double)b[p + 1]) *
                               (tracked_energy(I, &reps[a]) - tracked_energy(I, &reps[c]));
            int acc = arg >= 0.0;
            if (!acc) {
                uint32_t rw = philox_word(seed, (uint32_t)p, (uint32_t)sw, (uint32_t)l, 2u, 0);
                acc = orc_uniform(rw) < orc_expf((float)arg);
            }
            if (swap_trace) swap_trace[((int64_t)l * sweeps + sw) * (K - 1) + p] = (uint8_t)acc;
            if (acc) {
                at[p] = c; at[p + 1] = a;
                tof[a] = p + 1; tof[c] = p;
                cnt[p]++;
            }
        }
    }
}

int orc_ptda_adaptive(int64_t N, int mode, const void* Q, const float* betas_in, int32_t K,
                      int64_t sweeps, float inc, int32_t L, uint64_t seed, int64_t adapt_every,
                      int64_t adapt_sweeps, float* betas_out,
                      double* E_final, double* E_best, uint32_t* x_best, int32_t* temp_of,
                      int64_t* swaps, uint8_t* swap_trace, int nthreads)
{
    if (N < 1 || K < 1 || sweeps < 0 || L < 0 || !Q || !betas_in || adapt_every < 0) return -1;
    if (mode != ORC_MODE_INT && mode != ORC_MODE_F32) return -1;
    inst_t I;
    if (inst_make(&I, N, mode, Q)) return -2;
    const int64_t words = (N + 31) / 32;
    const int64_t LK = (int64_t)L * K;
    const int32_t P = K > 1 ? K - 1 : 0;
    rep_t* reps = (rep_t*)calloc((size_t)(LK > 0 ? LK : 1), sizeof(rep_t));
    uint8_t* best = (uint8_t*)calloc((size_t)(LK * N > 0 ? LK * N : 1), 1);
    double* Ebest = (double*)calloc((size_t)(LK > 0 ? LK : 1), sizeof(double));
    int32_t* tof = (int32_t*)malloc((size_t)(LK > 0 ? LK : 1) * sizeof(int32_t));
    int32_t* at = (int32_t*)malloc((size_t)(LK > 0 ? LK : 1) * sizeof(int32_t));
    int64_t* cnt = (int64_t*)calloc((size_t)((int64_t)L * P > 0 ? (int64_t)L * P : 1), sizeof(int64_t));
    int64_t* seen = (int64_t*)calloc((size_t)(P > 0 ? P : 1), sizeof(int64_t));
    int64_t* win = (int64_t*)calloc((size_t)(P > 0 ? P : 1), sizeof(int64_t));
    float* b = (float*)malloc((size_t)K * sizeof(float));
    float* nb = (float*)malloc((size_t)K * sizeof(float));
    int err = (!reps || !best || !Ebest || !tof || !at || !cnt || !seen || !win || !b || !nb) ? -2 : 0;
    for (int64_t r = 0; r < LK && !err; ++r) err = rep_init(&reps[r], &I) != 0 ? -2 : 0;
    if (!err) {
        for (int32_t k = 0; k < K; ++k) b[k] = betas_in[k];
        for (int64_t r = 0; r < LK; ++r) { tof[r] = (int32_t)(r % K); at[r] = (int32_t)(r % K); }
        int64_t sw = 0;
        while (sw < sweeps) {
            const int adapting = adapt_every > 0 && sw < adapt_sweeps;
            int64_t end = sweeps;
            if (adapting && (sw / adapt_every + 1) * adapt_every < end) end = (sw / adapt_every + 1) * adapt_every;
#ifdef _OPENMP
            if (nthreads < 1) nthreads = 1;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
#endif
            for (int32_t l = 0; l < L; ++l)
                ptda_window(&I, reps + (int64_t)l * K, best + (int64_t)l * K * N, Ebest + (int64_t)l * K,
                            tof + (int64_t)l * K, at + (int64_t)l * K, cnt + (int64_t)l * P, b, K, l, sw, end,
                            sweeps, inc, seed, swap_trace);
            if (adapting && end % adapt_every == 0 && end <= adapt_sweeps) {
                for (int32_t p = 0; p < P; ++p) {
                    int64_t tot = 0;
                    for (int32_t l = 0; l < L; ++l) tot += cnt[(int64_t)l * P + p];
                    win[p] = tot - seen[p];
                    seen[p] = tot;
                }
                orc_pt_adapt(K, b, win, (int64_t)L * adapt_every, nb);
                for (int32_t k = 0; k < K; ++k) b[k] = nb[k];
            }
            sw = end;
        }
        for (int64_t o = 0; o < LK; ++o) {
            if (E_final) E_final[o] = tracked_energy(&I, &reps[o]);
            if (E_best) E_best[o] = Ebest[o];
            if (x_best) pack_bits(best + o * N, N, x_best + o * words);
            if (temp_of) temp_of[o] = tof[o];
        }
        if (swaps) for (int64_t o = 0; o < (int64_t)L * P; ++o) swaps[o] = cnt[o];
        if (betas_out) for (int32_t k = 0; k < K; ++k) betas_out[k] = b[k];
    }
    if (reps) for (int64_t r = 0; r < LK; ++r) rep_free(&reps[r]);
    free(reps); free(best); free(Ebest); free(tof); free(at); free(cnt); free(seen); free(win); free(b); free(nb);
    inst_free(&I);
    return err;
}

int orc_ptda(int64_t N, int mode, const void* Q, const float* betas, int32_t K,
             int64_t sweeps, float inc, int32_t L, uint64_t seed,
             double* E_final, double* E_best, uint32_t* x_best, int32_t* temp_of,
             int64_t* swaps, uint8_t* swap_trace, int nthreads)
{
    return orc_ptda_adaptive(N, mode, Q, betas, K, sweeps, inc, L, seed, 0, 0, NULL, E_final, E_best, x_best,
                             temp_of, swaps, swap_trace, nthreads);
}

/* ------------------------------------------------------------------------ */
/* Time to solution over a set of instances (Sec. IV, Algorithm 3).  Random
 * numbers: Philox blocks (b, j, k, 6) of the seed for resample b, sampled
 * instance j, k-th block of that pair; uniforms in (0, 1) from 53 bits of two
 * consecutive words; normals by Box-Muller (first variate); Gamma(a) by
 * Marsaglia & Tsang for a >= 1 and Gamma(a + 1) u^(1/a) for a < 1; Beta(a, b)
 * = X / (X + Y) from two Gamma draws; the posterior of an instance with y hits
 * in r runs is Beta(0.5 + y, 0.5 + r - y) (Jeffreys prior). */
typedef struct { uint64_t seed; uint32_t b, j, k; uint32_t w[4]; int used; } ustream_t;

static uint32_t us_word(ustream_t* s)
{
    if (s->used == 4) {
        const uint32_t ctr[4] = {s->b, s->j, s->k++, 6u};
        const uint32_t key[2] = {(uint32_t)s->seed, (uint32_t)(s->seed >> 32)};
        orc_philox4x32_10(ctr, key, s->w);
        s->used = 0;
    }
    return s->w[s->used++];
}

static double us_uniform(ustream_t* s)
{
    const uint64_t hi = us_word(s) >> 5;
    const uint64_t lo = us_word(s) >> 6;
    return ((double)((hi << 26) | lo) + 0.5) * 0x1.0p-53;
}

static double us_normal(ustream_t* s)
{
    const double u1 = us_uniform(s);
    const double u2 = us_uniform(s);
    return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
}

static double us_gamma(ustream_t* s, double a)
{
    if (a < 1.0) {
        const double g = us_gamma(s, a + 1.0);
        const double u = us_uniform(s);
        return g * exp(log(u) / a);
    }
    const double d = a - 1.0 / 3.0;
    const double c = 1.0 / sqrt(9.0 * d);
    double v = 1.0;
    for (int it = 0; it < 1000; ++it) {
        const double x = us_normal(s);
        const double t = 1.0 + c * x;
        if (t <= 0.0) continue;
        v = t * t * t;
        const double u = us_uniform(s);
        if (log(u) < 0.5 * x * x + d - d * v + d * log(v)) return d * v;
    }
    return d * v;
}

void orc_beta_samples(double a, double b, int64_t n, uint64_t seed, double* out)
{
    for (int64_t i = 0; i < n; ++i) {
        ustream_t s = {seed, (uint32_t)(i >> 32), (uint32_t)i, 0u, {0, 0, 0, 0}, 4};
        const double x = us_gamma(&s, a);
        const double y = us_gamma(&s, b);
        out[i] = x / (x + y);
    }
}

static int cmp_double(const void* a, const void* b)
{
    const double x = *(const double*)a, y = *(const double*)b;
    return (x > y) - (x < y);
}

/* q-th percentile (0..100), linear interpolation at position (n - 1) q / 100 of
 * the sorted values (sorts v). */
double orc_percentile(double* v, int64_t n, double q)
{
    qsort(v, (size_t)n, sizeof(double), cmp_double);
    const double pos = (double)(n - 1) * q / 100.0;
    int64_t lo = (int64_t)floor(pos);
    int64_t hi = lo + 1 < n ? lo + 1 : n - 1;
    const double f = pos - (double)lo;
    return v[lo] + f * (v[hi] - v[lo]);
}

int orc_tts_bootstrap(const int64_t* hits, const int64_t* runs, int32_t I, double tau, double q, int32_t B,
                      uint64_t seed, double* tts_q)
{
    if (I < 1 || B < 1) return -1;
    double* r99 = (double*)malloc((size_t)I * sizeof(double));
    if (!r99) return -2;
    const double log_miss = log(1.0 - 0.99);
    for (int32_t b = 0; b < B; ++b) {
        for (int32_t j = 0; j < I; ++j) {
            ustream_t s = {seed, (uint32_t)b, (uint32_t)j, 0u, {0, 0, 0, 0}, 4};
            int64_t idx = (int64_t)(us_uniform(&s) * (double)I);
            if (idx >= I) idx = I - 1;
            const double x = us_gamma(&s, 0.5 + (double)hits[idx]);
            const double y = us_gamma(&s, 0.5 + (double)(runs[idx] - hits[idx]));
            const double p = x / (x + y);
            double r = p >= 1.0 ? 1.0 : log_miss / log(1.0 - p);
            if (!(r >= 1.0)) r = 1.0;
            r99[j] = r;
        }
        tts_q[b] = tau * orc_percentile(r99, I, q);
    }
    free(r99);
    return 0;
}

/* The DA's fixed-point scaling (Sec. III, "Benchmarking Problems"): one factor
 * s = min(coupler_max / max_{i<j} |Q_ij|, bias_max / max_i |Q_ii|) (terms with
 * a zero maximum left out, s = 1 for Q = 0), Qint = nearest integer to s Q
 * (ties to even) on and above the diagonal, 0 below. */
int orc_quantize(int64_t N, const float* Q, int32_t coupler_max, int32_t bias_max, int32_t* Qint, double* scale)
{
    double qmax = 0.0, dmax = 0.0;
    for (int64_t i = 0; i < N; ++i)
        for (int64_t j = i; j < N; ++j) {
            const double v = fabs((double)Q[i * N + j]);
            if (i == j) { if (v > dmax) dmax = v; }
            else if (v > qmax) qmax = v;
        }
    double s = 0.0;
    if (qmax > 0.0) s = (double)coupler_max / qmax;
    if (dmax > 0.0) {
        const double sd = (double)bias_max / dmax;
        if (!(s > 0.0) || sd < s) s = sd;
    }
    if (!(s > 0.0)) s = 1.0;
    for (int64_t i = 0; i < N; ++i)
        for (int64_t j = 0; j < N; ++j)
            Qint[i * N + j] = j < i ? 0 : (int32_t)nearbyint(s * (double)Q[i * N + j]);
    *scale = s;
    return 0;
}
