/*
 * da_oracle.h -- plain, slow, serial CPU reference for the Digital Annealer
 * (Aramon et al., "Physics-Inspired Optimization for Quadratic Unconstrained
 * Problems Using a Digital Annealer", arXiv:1806.08815).
 *
 * TEST INFRASTRUCTURE ONLY.  This library exists to check the CUDA path.  It
 * shares no code, header, constant or helper with the product library
 * (paper_1806_08815_gb300/csrc).  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may load it.
 *
 * Conventions (identical to the product ABI so the two can be compared):
 *   - A QUBO instance is an N x N row-major matrix Q whose upper triangle
 *     (i <= j) is read: Q[i][i] are the linear terms, Q[i][j] (i < j) the
 *     couplings.  E(x) = sum_i Q_ii x_i + sum_{i<j} Q_ij x_i x_j
 *     (Sec. "Benchmarking Problems", QUBO form of Eq. 4).
 *   - W is the symmetric off-diagonal coupling matrix (W_ij = W_ji = Q_ij for
 *     i < j, W_ii = 0); the local field of variable i is h_i = sum_j W_ij x_j.
 *   - A state is bit-packed: bit (i % 32) of word (i / 32) is x_i.
 *
 * Every function returns 0 on success and a negative value on bad arguments.
 */
#ifndef DA_ORACLE_H
#define DA_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Arithmetic of the field vector h (and the energy tracked step by step). */
enum {
    ORC_MODE_INT = 0, /* integer couplings: int64 h, int64 E (exact)          */
    ORC_MODE_F32 = 1, /* real couplings: fp32 effective fields Q_ii + h_i (one
                         rounding per update), fp64 E accumulated from fp32
                         Delta E, fp32 decisions                               */
    ORC_MODE_F64 = 2  /* real couplings: fp64 h and E (statistical reference) */
};

/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): one block of 4 words. */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* exp(x) in fp32 by Cody-Waite reduction and a degree-7 Taylor polynomial.
 * Returns 0 for x < -86. */
float orc_expf(float x);
void orc_expf_batch(const float* x, float* y, int64_t n);

/* Uniform u in (0, 1]: ((r >> 8) + 1) * 2^-24. */
float orc_uniform(uint32_t r);

/* Exact QUBO energies from the upper triangle of Q. */
int64_t orc_energy_int(int64_t N, const int32_t* Q, const uint32_t* x);
double  orc_energy_f64(int64_t N, const float* Q, const uint32_t* x);

/* Ising -> QUBO with s = 2x - 1: H(s) = E(x) + C.  J is N x N, upper triangle
 * (i < j) read; hb[N] are the biases of Eq. 4.  Q receives N x N (upper
 * triangle written, lower triangle zeroed). */
int orc_ising_to_qubo(int64_t N, const double* J, const double* hb, double* Q, double* C);
double orc_ising_energy(int64_t N, const double* J, const double* hb, const int8_t* s);

/* Minimum of E over all 2^N states (N <= 30) by Gray-code enumeration.
 * Returns the minimum, the number of minimising states and one of them. */
int orc_brute_force_f64(int64_t N, const double* Q, double* Emin, int64_t* count, uint32_t* argmin);

/* Local fields h = W x of a bit-packed state. */
int orc_fields_int(int64_t N, const int32_t* Q, const uint32_t* x, int64_t* h);
/* The periodic recompute of the fp32 path's effective fields
 * g_i = Q_ii + sum_j W_ij x_j as an exact fixed-point sum: Q_ii and the W_ij
 * are put on the grid 2^-S (S from max(|W|, |Q_ii|) and N, see the .c file),
 * summed exactly in int64, and rounded once to fp32.  sums[N] (may be NULL)
 * receives the exact integer sums, *S_out the scale. */
int orc_recompute_f32(int64_t N, const float* Q, const uint32_t* x, float* h, int64_t* sums, int32_t* S_out);
/* The energy that accompanies the recompute: sum_i x_i (Q_ii + g_i) / 2 summed
 * exactly on the fixed-point grid and rounded once to fp64. */
double orc_recompute_energy_f32(int64_t N, const float* Q, const uint32_t* x);

/* The Digital Annealer (Algorithm 2) run R times from x = 0.
 *   Q        N x N upper-triangular QUBO: int32_t* when mode == ORC_MODE_INT,
 *            float* otherwise.
 *   beta[T]  inverse temperature of each step (updated every iteration).
 *   inc      offset increase rate; E_off = m * inc after m steps without an
 *            accepted flip (0 turns the dynamic offset off).
 *   seed     Philox key; replica r draws with counter replica id
 *            replica_base + r.
 *   recompute_every  (ORC_MODE_F32 only) period of the fixed-point field
 *            recompute, 0 = never.
 * Outputs (each may be NULL): E_final[R], E_best[R] (tracked energies),
 * x_final/x_best[R * ceil(N/32)], flips[R], trace[R * T] (the flipped
 * variable of every step, -1 when none was accepted), accepted[R * T]
 * (number of accepted trials of every step).  nthreads > 1 runs replicas on
 * OpenMP threads (results do not depend on it). */
int orc_da_anneal(int64_t N, int mode, const void* Q,
                  const float* beta, int64_t T, float inc, int32_t R,
                  uint64_t seed, uint32_t replica_base, int64_t recompute_every,
                  double* E_final, double* E_best, uint32_t* x_final, uint32_t* x_best,
                  int64_t* flips, int32_t* trace, int32_t* accepted, int nthreads);

/* One DA step from a given state for the transition-distribution tests.
 * x (bit-packed) and the offset count m are read, nothing is modified.
 * Returns the flipped index or -1, and writes the accept count. */
int orc_da_one_step(int64_t N, int mode, const void* Q, const uint32_t* x, uint32_t m,
                    float beta, float inc, uint64_t seed, uint32_t t, uint32_t replica,
                    int32_t* n_accepted);

/* Simulated annealing (Algorithm 1), one Metropolis sweep per temperature, R
 * runs from Philox-random initial states; fp64 fields.  Returns the best
 * energy of each run and its state. */
int orc_sa_anneal(int64_t N, const float* Q, const float* beta, int64_t T, int32_t R,
                  uint64_t seed, double* E_best, uint32_t* x_best, int nthreads);

/* Parallel tempering with the DA step (PTDA).  L independent ladders of K
 * replicas; replica k starts at temperature index k (betas ascending) from
 * x = 0.  A sweep is N DA steps of every replica, followed by replica-exchange
 * proposals between temperature indices (0,1), (1,2), ..., (K-2,K-1) in that
 * order.  Outputs (each may be NULL): E_final[L*K], E_best[L*K],
 * x_best[L*K*words], temp_of[L*K] (final temperature index of each replica),
 * swaps[L*(K-1)] (accepted exchanges per pair), swap_trace[L*sweeps*(K-1)]
 * (1 if the exchange of pair k after a sweep was accepted). */
int orc_ptda(int64_t N, int mode, const void* Q, const float* betas, int32_t K,
             int64_t sweeps, float inc, int32_t L, uint64_t seed,
             double* E_final, double* E_best, uint32_t* x_best, int32_t* temp_of,
             int64_t* swaps, uint8_t* swap_trace, int nthreads);

/* The PTDA with its adaptive ladder: as orc_ptda, and after every
 * adapt_every sweeps up to sweep adapt_sweeps the ladder is updated by
 * orc_pt_adapt from the exchanges accepted in that window over all ladders
 * (proposals = L * adapt_every per pair); betas_out[K] (may be NULL) gets the
 * final ladder.  adapt_every = 0 is orc_ptda. */
int orc_ptda_adaptive(int64_t N, int mode, const void* Q, const float* betas_in, int32_t K,
                      int64_t sweeps, float inc, int32_t L, uint64_t seed, int64_t adapt_every,
                      int64_t adapt_sweeps, float* betas_out,
                      double* E_final, double* E_best, uint32_t* x_best, int32_t* temp_of,
                      int64_t* swaps, uint8_t* swap_trace, int nthreads);

/* The adaptive ladder update (proportional feedback on the gaps towards equal
 * exchange acceptance, ends fixed): out[K] from betas[K], accepted[K-1]
 * exchanges of each pair out of `proposals`. */
void orc_pt_adapt(int32_t K, const float* betas, const int64_t* accepted, int64_t proposals, float* out);

/* Time to solution over instances (Sec. IV, Algorithm 3): B bootstrap
 * resamples of the I instances (with replacement); for each sampled instance a
 * success probability from its posterior Beta(0.5 + y, 0.5 + r - y) (hits y of
 * runs r), R99 = log(0.01) / log(1 - p) (at least 1); tts_q[b] = tau times the
 * q-th percentile of the R99 values of resample b. */
int orc_tts_bootstrap(const int64_t* hits, const int64_t* runs, int32_t I, double tau, double q, int32_t B,
                      uint64_t seed, double* tts_q);
/* n draws of Beta(a, b) from the sampler of orc_tts_bootstrap (draw i uses the
 * Philox stream (i >> 32, i & 0xffffffff, k, 6)). */
void orc_beta_samples(double a, double b, int64_t n, uint64_t seed, double* out);
/* q-th percentile by linear interpolation of the sorted values (sorts v). */
double orc_percentile(double* v, int64_t n, double q);

/* The DA's fixed-point scaling of a real QUBO: one factor
 * s = min(coupler_max / max_{i<j} |Q_ij|, bias_max / max_i |Q_ii|), Qint the
 * nearest integers (ties to even) to s Q on and above the diagonal. */
int orc_quantize(int64_t N, const float* Q, int32_t coupler_max, int32_t bias_max, int32_t* Qint, double* scale);

#ifdef __cplusplus
}
#endif
#endif
