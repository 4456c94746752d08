/*
 * da.h -- C ABI of a GB300 (sm_103a) library for the Digital Annealer's
 * method: the parallel-trial Monte Carlo step on a dense QUBO with a dynamic
 * offset, run over many replicas, and its parallel-tempering variant (PTDA).
 *
 * Paper: M. Aramon, G. Rosenberg, E. Valiante, T. Miyazawa, H. Tamura,
 * H. G. Katzgraber, "Physics-Inspired Optimization for Quadratic
 * Unconstrained Problems Using a Digital Annealer", arXiv:1806.08815.
 *
 * General conventions
 *  - Every entry point returns a da_status and never aborts.  On failure a
 *    description is available from da_last_error() (per calling thread).
 *  - "host" pointers are ordinary CPU memory owned by the caller; the library
 *    copies what it needs before returning (or, for the *_async calls, before
 *    the queued work reads it).  "device" pointers are CUDA global memory of
 *    the current device, owned by the caller.  The library owns all other
 *    device memory it uses (its context's copies of the instance and its
 *    workspace) and frees it in da_destroy.
 *  - A QUBO is an N x N row-major matrix Q of which only the upper triangle
 *    (i <= j) is read: Q_ii are the linear terms and Q_ij (i < j) the
 *    couplings of E(x) = sum_i Q_ii x_i + sum_{i<j} Q_ij x_i x_j over
 *    x in {0,1}^N ("Benchmarking Problems": the QUBO form the DA optimises,
 *    obtained from Eq. 4 with s = 2x - 1).
 *  - A state is bit-packed in 32-bit words: x_i is bit (i % 32) of word
 *    (i / 32); a state of N variables takes da_words(N) = ceil(N / 32) words.
 *  - Calls on one da_ctx are serialised by the context (thread-safe); the
 *    *_async calls only order work on the caller's stream, so concurrent
 *    async calls on one context must use one stream.
 *  - No CPU fallback: without a usable CUDA device every call that computes
 *    returns DA_ECUDA.
 */
#ifndef DA_H
#define DA_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct da_ctx da_ctx;

typedef enum da_dtype {
    DA_INT8 = 0,  /* integer couplings (e.g. bimodal +-1 -> +-4): int8 W, int32 fields, exact */
    DA_FP32 = 1,  /* real couplings (e.g. Gaussian): fp32 W and fields, fp64 energies */
    DA_INT16 = 2  /* the DA's fixed-point precision (Sec. III "Benchmarking Problems": 16-bit
                     couplers, 26-bit biases): int16 W, int32 fields, exact integer energies
                     (real couplings enter through da_quantize) */
} da_dtype;

typedef enum da_status {
    DA_OK = 0,
    DA_EINVAL = 1,    /* an argument is out of range; nothing was done */
    DA_ENOMEM = 2,    /* a device or host allocation failed */
    DA_EBUDGET = 3,   /* the request can never fit the device-memory budget */
    DA_EBUSY = 4,     /* the context is in use by an incompatible call */
    DA_ETIMEOUT = 5,  /* a bounded wait ran out */
    DA_ECUDA = 6,     /* a CUDA call failed (no device, launch error, ...) */
    DA_ENOTREADY = 7, /* asynchronous work has not finished yet */
    DA_ECANCELED = 8  /* the request was cancelled (da_cancel) */
} da_status;

/* Results of da_anneal, one entry per replica r (host arrays, caller-allocated;
 * every pointer may be NULL to skip that output). */
typedef struct da_result {
    double* final_E;    /* [R] exact energy of the final state (int64 sum for DA_INT8;
                           exact fixed-point fields then fp64 for DA_FP32) */
    double* best_E;     /* [R] exact energy of the lowest-energy state the run visited */
    uint32_t* final_x;  /* [R * da_words(N)] final state */
    uint32_t* best_x;   /* [R * da_words(N)] best state */
    double* max_drift;  /* [R] |tracked energy - exact energy| of the final state
                           (the fp32 accumulation error; 0 for DA_INT8) */
    int64_t* flips;     /* [R] number of accepted (applied) flips */
    int32_t* trace;     /* [R * steps] index flipped at every step, -1 if none was
                           accepted (debug output; slows the run) */
    double elapsed_s;   /* written by the call: device time of the anneal */
} da_result;

/* Device-side results of da_anneal_async (device arrays, caller-allocated,
 * each may be NULL).  Same meaning as in da_result. */
typedef struct da_dev_result {
    double* final_E;
    double* best_E;
    uint32_t* final_x;
    uint32_t* best_x;
    double* max_drift;
    int64_t* flips;
    int32_t* trace;
} da_dev_result;

/* Results of da_pt: L ladders of K replicas; replica k of ladder l is entry
 * l*K + k.  Host arrays, caller-allocated, each may be NULL. */
typedef struct da_pt_result {
    double* final_E;     /* [L*K] exact energy of each replica's final state */
    double* best_E;      /* [L*K] exact energy of each replica's best state */
    uint32_t* best_x;    /* [L*K*da_words(N)] */
    int32_t* temp_of;    /* [L*K] final temperature index of each replica */
    int64_t* swaps;      /* [L*(K-1)] accepted exchanges of each neighbouring pair */
    uint8_t* swap_trace; /* [L*sweeps*(K-1)] 1 where the exchange of pair p after a
                            sweep was accepted (debug output) */
    double elapsed_s;    /* written by the call: device time */
} da_pt_result;

/* Library version (major * 10000 + minor * 100 + patch). */
int da_version(void);

/* Words of a bit-packed state of N variables: ceil(N / 32). */
int64_t da_words(int64_t N);

/* Description of the last failure on the calling thread ("" if none).  The
 * string stays valid until the next call on this thread. */
const char* da_last_error(void);

/* Create a context holding one QUBO instance on the current CUDA device.
 *   Q      host, N x N row-major (int32_t for DA_INT8 and DA_INT16, float for
 *          DA_FP32); the upper triangle is checked on the host, then the
 *          array goes to the device once (a transient N*N*4-byte copy) where
 *          W and diag are built from it; the caller keeps Q.
 *   N      1 <= N <= 8192 (the next-generation DA size named in Sec. II).
 *   dtype  DA_INT8 requires every coupling in [-128, 127] and every
 *          |Q_ii| + sum_j |Q_ij| < 2^24 (so that every Delta E is exact in
 *          fp32); DA_INT16 requires every coupling in [-32767, 32767] and every
 *          |Q_ii| + sum_j |Q_ij| < 2^31 (fields and energies stay exact; a
 *          Delta E beyond 2^24 enters the acceptance test rounded to fp32, as
 *          every Delta E does); DA_FP32 requires finite values.
 *          DA_INT16 contexts serve da_anneal, da_anneal_async, da_pt,
 *          da_pt_adaptive, da_batch_anneal, da_energy, da_field_recompute and
 *          da_move_energy_percentiles, and da_submit takes DA_INT16 jobs (the
 *          plain and allocation-free forms take DA_INT8 / DA_FP32 and DA_INT8).
 * The library stores W (symmetric, zero diagonal) and diag(Q) in device
 * memory.  Errors: DA_EINVAL (bad N, dtype, range), DA_ENOMEM, DA_ECUDA. */
da_status da_create(const void* Q, int64_t N, da_dtype dtype, da_ctx** out);

/* The DA's scaling of real coefficients to its fixed-point precision (Sec. III,
 * "Benchmarking Problems": the coefficients are scaled up to the hardware's
 * limits, 2^15 - 1 for the quadratic and 2^25 - 1 for the linear ones, and
 * rounded to the nearest integers).  One factor for the whole instance:
 * scale = min(coupler_max / max_{i<j} |Q_ij|, bias_max / max_i |Q_ii|) (a
 * term whose maximum is 0 is left out; scale = 1 for Q = 0);
 * Qint[i][j] = round(scale Q[i][j]) to nearest, ties to even, upper triangle
 * with diagonal (the lower triangle is set to 0).  Q, Qint: host N x N
 * row-major.  The quantized problem's energies are scale times the original
 * ones up to the rounding; a DA_INT16 context takes Qint with the anneal's
 * beta divided by scale.  Errors: DA_EINVAL (non-finite entries, N < 1, limits
 * < 1 or above 2^30). */
da_status da_quantize(const float* Q, int64_t N, int32_t coupler_max, int32_t bias_max, int32_t* Qint,
                      double* scale);

/* Release a context and its device memory (NULL is ignored). */
void da_destroy(da_ctx* ctx);

/* N and dtype of a context. */
da_status da_ctx_info(const da_ctx* ctx, int64_t* N, da_dtype* dtype);

/* Fix the launch shape of the step kernel for this context instead of the
 * automatic choice: a group of G warps per replica, V variables per lane
 * (32 * V * G >= N), rpb replicas per thread block.  Supported: G = 1 or 2
 * with V in {4, 8, 16, 32}; G = 4 with V in {4, 8, 16}; G = 8 with V in
 * {8, 16, 32}; rpb <= 4 (G = 1), <= 2 (G = 2), = 1 (G = 4, 8).  V = 0
 * restores the automatic choice.  Results do
 * not depend on the shape (the random numbers are keyed by variable index,
 * step and replica).  Errors: DA_EINVAL. */
da_status da_set_launch_shape(da_ctx* ctx, int32_t V, int32_t G, int32_t rpb);

/* Autotune the step kernel's launch shape for this context's instance and R
 * replicas: every supported shape that covers N (for each G in 1, 2, 4, 8 the
 * narrowest lane width V, every allowed rpb, and for G = 1 the producer-warp
 * form) runs probe_steps steps from x = 0 with beta = 0 (every step flips), the
 * fastest (CUDA events, best of two runs) is written to *V, *G, *rpb,
 * *draw_warp (each may be NULL) and kept in a process-wide cache keyed by
 * (device, coupling type, N, R) that every context's later anneals use unless
 * a shape was fixed with da_set_launch_shape.  Results of an anneal do not
 * depend on the shape.  Blocking; uses the context's workspace.  Errors:
 * DA_EINVAL, DA_ENOMEM, DA_ECUDA. */
da_status da_tune_shape(da_ctx* ctx, int32_t replicas, int64_t probe_steps, int32_t* V, int32_t* G, int32_t* rpb,
                        int32_t* draw_warp);

/* For shapes with G = 1 (the automatic choice up to N = 1024): on = 1 runs
 * each replica as an annealer warp plus a producer warp that computes the
 * acceptance draws of the coming steps (Philox words as log2 u) into shared
 * memory, one replica per block, rpb ignored; on = 0 (the default) lets the
 * annealer warp draw for itself while its row load is in flight.  Results
 * are identical either way (each trial's decision equals the exact Metropolis
 * test of Sec. II with the same u).  Errors: DA_EINVAL. */
da_status da_set_draw_warp(da_ctx* ctx, int32_t on);

/* Run the Digital Annealer (Algorithm 2) R times from x = 0 (all runs start
 * from one state, Sec. II) for `steps` iterations, blocking until done.
 *   beta_schedule  host, [steps] inverse temperature of every step (the
 *                  temperature is updated every iteration, "DA parameters");
 *                  every entry finite and >= 0 (DA_EINVAL otherwise).
 *   offset_inc     dynamic-offset increase rate: after m steps without an
 *                  accepted flip the trials use Delta E - m * offset_inc;
 *                  0 switches the offset off (as in the paper's runs).
 *   replicas       R >= 1 independent runs.
 *   seed           Philox key; run r draws its numbers with replica id r, so
 *                  results do not depend on R, on the launch shape or on the
 *                  device.
 *   recompute_every  DA_FP32 only: recompute the fields exactly every this many
 *                  steps to bound the fp32 drift (0 = never).  Ignored for
 *                  DA_INT8 and DA_INT16, whose fields are exact.
 * Errors: DA_EINVAL, DA_ENOMEM, DA_ECUDA, DA_ETIMEOUT (a bounded wait inside a
 * pipelined kernel gave up; the results are invalid). */
da_status da_anneal(da_ctx* ctx, const float* beta_schedule, int64_t steps, float offset_inc,
                    int32_t replicas, uint64_t seed, int64_t recompute_every, da_result* out);

/* The state of R replicas between two segments of an anneal (host arrays,
 * caller-allocated; written by da_anneal_segment, read back by the next one).
 * The paper has no counterpart (its runs go from x = 0 to the end); it makes a
 * long anneal resumable. */
typedef struct da_checkpoint {
    uint32_t* x;       /* [R * da_words(N)] current states */
    uint32_t* best_x;  /* [R * da_words(N)] lowest-energy states seen */
    void* fields;      /* [R * N] effective fields g_i = Q_ii + sum_j W_ij x_j as the anneal
                          holds them: int32_t for DA_INT8 and DA_INT16, float for DA_FP32
                          (with its fp32 rounding since the last recompute) */
    int64_t* scalars;  /* [R * 4] per replica: tracked energy, best tracked energy (int64
                          for integer couplings, fp64 bit patterns for DA_FP32), accepted
                          flips, steps without an accepted flip (E_off = that count * inc) */
} da_checkpoint;

/* Steps [t0, t1) of an anneal of `total_steps` steps (Algorithm 2), from the
 * checkpoint `in` (NULL: from x = 0, then t0 must be 0), leaving the state after
 * step t1 in `out` (may be NULL) and, in `res` (may be NULL; no trace), the
 * results the anneal would report if it ended after step t1.  The random
 * numbers are keyed by the absolute step and the fp32 recompute falls on
 * absolute multiples of recompute_every, so running [0, T) in segments gives
 * exactly the results of da_anneal over [0, T) with the same arguments.
 *   beta  host, [total_steps] the whole schedule (entries [0, t1) are read).
 * `in` must come from da_anneal_segment on a context with the same instance
 * and the same replica count.  Blocking.  Errors: DA_EINVAL (0 <= t0 <= t1 <=
 * total_steps < 2^32 violated, in == NULL with t0 > 0, a trace requested, ...),
 * DA_ENOMEM, DA_ECUDA, DA_ETIMEOUT. */
da_status da_anneal_segment(da_ctx* ctx, const float* beta, int64_t total_steps, int64_t t0, int64_t t1,
                            float offset_inc, int32_t replicas, uint64_t seed, int64_t recompute_every,
                            const da_checkpoint* in, da_checkpoint* out, da_result* res);

/* As da_anneal, with the schedule and every output in device memory, queued
 * on `stream` (a cudaStream_t; NULL = the legacy default stream) and
 * returning without waiting.  The device schedule is not inspected: its
 * entries must be finite and >= 0 (other values give undefined results).
 * The context's workspace is reused: calls on one context must be ordered on
 * one stream.  A bounded wait that gave up in a queued call is reported
 * (DA_ETIMEOUT) by the next blocking call on the context. */
da_status da_anneal_async(da_ctx* ctx, const float* beta_schedule_dev, int64_t steps, float offset_inc,
                          int32_t replicas, uint64_t seed, int64_t recompute_every,
                          const da_dev_result* out, void* stream);

/* The plain GPU form of the same anneal, kept as the baseline the library's
 * kernels are measured against: one kernel launch per DA step (Algorithm 2),
 * one thread block per replica, one thread per variable, fp32 fields and
 * state in global memory between launches, no field recompute.  It draws the
 * same random numbers, so its trajectories equal da_anneal's with
 * recompute_every = 0.  N <= 1024.  Same arguments and results as da_anneal.
 * Errors: DA_EINVAL, DA_ENOMEM, DA_ECUDA. */
da_status da_anneal_plain(da_ctx* ctx, const float* beta_schedule, int64_t steps, float offset_inc,
                          int32_t replicas, uint64_t seed, da_result* out);

/* One instance's share of a batched launch (see da_batch_anneal). */
typedef struct da_batch_item {
    da_ctx* ctx;                /* the instance (N <= 1024) */
    const float* beta;          /* host, [steps] schedule */
    int64_t steps;
    float offset_inc;
    int32_t replicas;
    uint64_t seed;
    int64_t recompute_every;    /* DA_FP32 only, 0 = never */
    da_result* out;             /* host results, as for da_anneal (may be NULL) */
} da_batch_item;

/* Anneal many instances of different sizes and coupling types together: every
 * replica of every item is one work unit, and warps of one persistent kernel per
 * (coupling type, size class) pull units from a device queue until none are left;
 * all launches and the exact final evaluation form one CUDA graph.  Each item's
 * results are identical to da_anneal on that item alone (the random numbers are
 * keyed by the item's seed and replica index).  Each class's configuration is
 * chosen by an autotuner that times short probes (1024 steps) of the class's own
 * units once per process, device and class: warps per block (1, 2, 4), and,
 * where the class's largest instance fits (N x 32V x 4 bytes <= 227 KB, V <= 8),
 * W staged in shared memory, where each block takes a group of replicas of one
 * instance (2, 4, 8 or 16, one per warp), copies that instance's W once and
 * reads every row from there instead of from L2 (taken only when its probe is
 * more than 3 % faster than the best L2 one).  *elapsed_s receives the
 * device time of the graph.  Errors: DA_EINVAL (bad item, N > 1024), DA_ENOMEM,
 * DA_ECUDA. */
da_status da_batch_anneal(const da_batch_item* items, int32_t n, double* elapsed_s);

/* The configuration the last da_batch_anneal on the calling thread used for
 * each class, with the tuner's probe times, as text (at most len - 1 bytes and
 * a terminating 0 written to buf).  Errors: DA_EINVAL. */
da_status da_batch_describe(char* buf, int64_t len);

/* Override the tuner of da_batch_anneal for the calls that follow, process
 * wide (for tests and measurements): staging -1 = the tuner's choice, 0 = rows
 * of W from L2, 1 = W staged in shared memory where the class allows it (else
 * L2), 2 = rows of W from L2 in the one-warp row order (a copy of the fp32
 * couplings whose rows are permuted so that every 16-byte load of a warp reads
 * 512 contiguous bytes) where the class allows it (fp32 and int8 instances of
 * more than 128 variables; else plain L2); warps_per_block 0 = the tuner's
 * choice, else 1, 2 or 4 (2, 4, 8 or 16 when staged).  da_batch_force(-1, 0)
 * restores the tuner.  Errors: DA_EINVAL. */
da_status da_batch_force(int32_t staging, int32_t warps_per_block);

/* ---- Request loop (continuous batching) ------------------------------------
 * A server runs each admitted request on a CUDA stream of its own: requests that
 * arrive while others are on the GPU are admitted as soon as device memory
 * (within the server's budget) and a request slot are free, and their kernels
 * start at once beside those already in flight.  Admission queues all of a
 * request's work (upload, instance build, the anneal in chunks, the exact final
 * evaluation) without waiting for the GPU.  A request's results are identical
 * to da_anneal on the same instance, schedule and seed (recompute_every applies
 * to DA_FP32, as in da_anneal). */
typedef struct da_server da_server;
typedef struct da_req da_req;

typedef struct da_job {
    const void* Q;            /* host, N x N upper-triangular QUBO (as da_create);
                                 Q and beta must stay valid until da_poll returns
                                 DA_OK or an error for this request */
    int64_t N;                /* 1 <= N <= 8192 */
    da_dtype dtype;
    const float* beta;        /* host, [steps] */
    int64_t steps;
    float offset_inc;
    int32_t replicas;         /* 1 <= replicas <= 65536 */
    uint64_t seed;
    int64_t recompute_every;
} da_job;

/* Start a server on the current device.  hbm_budget_bytes bounds the device
 * memory of admitted requests (instance, schedule, state, results, and the
 * transient copy of Q until the instance is built from it);
 * max_requests bounds how many are admitted at once.  Requests are admitted in
 * arrival order; admission also waits while the running requests' step
 * launches hold 8 warps per SM (replicas x warps per replica), beyond which
 * a further request would only share SMs with them; a request is admitted
 * alone whatever its size.  Creating a server loads and configures every
 * kernel it launches.  Errors: DA_EINVAL, DA_ENOMEM, DA_ECUDA. */
da_status da_server_create(int64_t hbm_budget_bytes, int32_t max_requests, da_server** out);

/* Queue a request; returns at once.  The instance is checked on the host here
 * (as da_create); its device layout is built at admission from a transient
 * device copy of Q (N*N*4 bytes, charged to the budget from admission until
 * the build is done).  The request loop is the one entry point that takes a
 * server instead of a context: a request carries its own instance, which the
 * server builds on its own stream, so that no context (and no host
 * synchronisation of one) stands between requests.
 * Errors: DA_EINVAL; DA_EBUDGET if the request alone
 * exceeds the budget (it could never be admitted); DA_EBUSY while the server is
 * shutting down.  A request whose device allocation fails at admission
 * finishes with DA_ENOMEM (reported by da_poll); the server goes on with the
 * others. */
da_status da_submit(da_server* srv, const da_job* job, da_req** out);

/* Wait up to timeout_us microseconds for a request.  DA_OK: results written to
 * out (host arrays as for da_anneal; out->elapsed_s = submit-to-completion
 * latency in seconds).  DA_ENOTREADY (timeout_us = 0) or DA_ETIMEOUT if it has
 * not finished; the request's own error if it failed. */
da_status da_poll(da_req* req, int32_t timeout_us, da_result* out);

/* Release a request handle (after its last poll). */
void da_req_free(da_req* req);

/* Cancel a request.  A queued request leaves the queue at once; a running one
 * stops at the start of its next step launch (launches already running finish
 * their chunk), then its memory returns to the budget.  da_poll then returns
 * DA_ECANCELED.  Cancelling a finished request changes nothing.
 * Errors: DA_EINVAL (null request). */
da_status da_cancel(da_req* req);

/* Requests of at most max_n variables (0 <= max_n <= 1024) submitted from now
 * on run resident: the whole anneal is one launch in which each replica's warp
 * keeps its state in registers from the first step to the last (fp32 fields
 * recomputed exactly by the warp itself every recompute_every steps; a
 * cancelled request leaves at its next multiple of 1024 steps).  Larger
 * requests, and all of them with max_n = 0, run as chunked step launches.
 * Results are the same either way.  Errors: DA_EINVAL. */
da_status da_server_resident(da_server* srv, int32_t max_n);

/* Requests completed, kernels queued so far (all requests), device bytes in use. */
da_status da_server_stats(da_server* srv, int64_t* completed, int64_t* kernel_launches, int64_t* bytes_in_use);

/* Wait for every submitted request to finish, then free the server.  A da_req
 * refers to its server: poll every request for the last time before
 * da_server_destroy (da_poll and da_cancel on a request of a destroyed server
 * are undefined); da_req_free may follow at any time. */
void da_server_destroy(da_server* srv);

/* Parallel tempering with the DA step (PTDA, Sec. II and Algorithm 4): L
 * independent ladders of K replicas at inverse temperatures betas[0..K-1]
 * (host, ascending), replica k starting at index k from x = 0.  A sweep is N DA
 * steps of every replica; after each sweep the pairs (0,1), (1,2), ...,
 * (K-2,K-1) propose, in order, to swap their temperatures with probability
 * min(1, exp((beta_p - beta_{p+1})(E_p - E_{p+1}))).  Blocking.
 * Errors: DA_EINVAL (K < 1, betas not ascending, ...), DA_ENOMEM, DA_ECUDA. */
da_status da_pt(da_ctx* ctx, const float* betas, int32_t K, int64_t sweeps, int32_t ladders,
                float offset_inc, uint64_t seed, da_pt_result* out);

/* PTDA with the adaptive ladder (Sec. II: the temperatures follow an
 * adaptive scheme in which the highest and lowest temperatures are fixed and
 * the intermediate ones are adjusted towards equal exchange probabilities of
 * neighbouring pairs).  As da_pt, and after every adapt_every sweeps up to
 * sweep adapt_sweeps the ladder is updated from the exchanges accepted in that
 * window over all ladders: each gap beta_{p+1} - beta_p is multiplied by
 * w_p^(1/8), w_p = (a_p + 1) / (L adapt_every + 2) the pair's smoothed
 * acceptance, and the gaps are rescaled to the fixed span beta_{K-1} - beta_0
 * (fp64, rounded to fp32); the updated ladder applies from the next sweep.  betas[K] (host, ascending) is
 * the initial ladder on entry and the final ladder on return.
 * Errors: DA_EINVAL (adapt_every < 1, as da_pt otherwise), DA_ENOMEM, DA_ECUDA. */
da_status da_pt_adaptive(da_ctx* ctx, float* betas, int32_t K, int64_t sweeps, int32_t ladders,
                         float offset_inc, uint64_t seed, int64_t adapt_every, int64_t adapt_sweeps,
                         da_pt_result* out);

/* The temperature grid's input (appendix, "Parameters": the low and high
 * temperatures are searched near the 5th-10th and 80th-85th percentiles of
 * the distribution of the energy changes of proposed moves): over the R host
 * states x[R * da_words(N)], every single-flip move that raises the energy,
 * Delta E_i = (1 - 2 x_i) g_i > 0 with the exactly recomputed fields; out[k] =
 * q[k]-th percentile (0..100) of those Delta E.  Errors: DA_EINVAL (no move
 * raises the energy, q outside [0, 100]), DA_ENOMEM, DA_ECUDA. */
da_status da_move_energy_percentiles(da_ctx* ctx, const uint32_t* x, int32_t R, const double* q, int32_t nq,
                                     double* out);

/* Exact energies of R bit-packed host states x[R * da_words(N)] into E[R]
 * (host).  Errors: DA_EINVAL, DA_ENOMEM, DA_ECUDA. */
da_status da_energy(da_ctx* ctx, const uint32_t* x, int32_t R, double* E);

/* The field recompute of R host states: h[R * N] (host; int32_t for DA_INT8,
 * float for DA_FP32), exactly as used between steps.  Errors as da_energy. */
da_status da_field_recompute(da_ctx* ctx, const uint32_t* x, int32_t R, void* h);

/* Per-launch timing of the step kernel: while enabled, every step-kernel
 * launch of this context is bracketed by CUDA events on the stream it runs
 * on.  da_profile_read waits for the recorded launches, returns their count
 * and summed device time, and starts a new count.  Enabling resets the
 * count.  Errors: DA_EINVAL, DA_ECUDA. */
da_status da_profile_enable(da_ctx* ctx, int32_t on);
da_status da_profile_read(da_ctx* ctx, int64_t* launches, double* total_ms);

/* An integer anneal that allocates nothing.  Some callers cannot allocate
 * device memory at the moment they want to anneal: a service that reserves
 * the GPU's memory up front and forbids later allocations, code inside
 * another framework's allocator-free region, or a program about to capture
 * its work into a CUDA graph.  This entry point runs the same anneal as
 * da_anneal_async on a DA_INT8 instance, with every intermediate buffer in one
 * fixed 16 MiB device array that the library defines (each device that loads
 * the library holds it until the process exits); it calls no cudaMalloc,
 * cudaFree or other allocating routine.  The paper has no counterpart: this
 * is a property of the library, not of the method.
 *   W      device, int8, N x ldw row-major, 16-byte aligned (rows are read
 *          with 16-byte loads): the symmetric couplings W_ij = Q_ij (i < j)
 *          mirrored, zero diagonal; entries in columns N..ldw-1 are read but
 *          only affect padding.  da_static_pitch(N) <= ldw <= INT_MAX, a
 *          multiple of 16.
 *   diag   device, int32, the N linear terms Q_ii (4-byte aligned).
 *   N      1 <= N <= 1024.
 *   beta   device, [steps] schedule (4-byte aligned); other arguments as in
 *          da_anneal_async.
 *   out    device result arrays (each may be NULL), each aligned to its
 *          element size.
 * A misaligned pointer or a pitch out of range returns DA_EINVAL before
 * anything is queued.  Sizes beyond the array (roughly replicas * N > 3.4e6 at
 * N = 1024) return DA_EINVAL.  The first call on a device looks up the array's
 * device address (cudaGetSymbolAddress) and caches it with the current CUDA
 * context (it is looked up again when the context changes); make that first
 * call before any stream capture.  A context destroyed by cudaDeviceReset may
 * be re-created under the same handle with the array elsewhere, so do not call
 * this entry point again after a device reset.  Every call reuses the same
 * array, so calls that overlap on the GPU (different streams, or different host
 * threads without ordering) race; order them on one stream.  The call
 * re-initialises the parts it needs, so results do not depend on earlier
 * calls.  Errors: DA_EINVAL, DA_ECUDA. */
da_status da_anneal_static(const int8_t* W, const int32_t* diag, int64_t N, int64_t ldw, const float* beta,
                           int64_t steps, float offset_inc, int32_t replicas, uint64_t seed,
                           const da_dev_result* out, void* stream);
/* The smallest row pitch da_anneal_static accepts for N variables (0 if N is
 * out of range). */
int64_t da_static_pitch(int64_t N);

/* Failure injection for tests of the error paths (host side; nothing is
 * faulted on the device): the library's next `after` device allocations (of
 * contexts, workspaces, tensor-core operands, batched launches and admitted
 * requests) succeed and the `count` after them fail as if the device were out
 * of memory, without being attempted.  count = 0 disarms.
 * da_diag_live_allocations: device allocations of the library that are live
 * now and their bytes, and how many failures were injected so far.
 * Errors: DA_EINVAL (negative arguments). */
da_status da_diag_fail_alloc(int32_t after, int32_t count);
da_status da_diag_live_allocations(int64_t* count, int64_t* bytes, int64_t* injected_failures);

/* Read bandwidth of the device buffer buf[bytes] (device, 16-byte aligned,
 * bytes a multiple of 16): one untimed pass, then `passes` timed passes of
 * 16-byte loads that bypass L1; *seconds = device time of the timed passes.
 * bytes * passes / *seconds is the L2 read bandwidth for a buffer that fits
 * L2 (the step kernel reads its rows of W from there) and the HBM read
 * bandwidth for a larger one; the roofline of the step kernel is stated
 * against it.  Errors: DA_EINVAL, DA_ECUDA. */
da_status da_diag_read_bandwidth(const void* buf, int64_t bytes, int32_t passes, double* seconds);

/* Diagnostics: run the device's own fp32 exponential (used for every
 * Metropolis decision) on n host values x[n] -> y[n], and its Philox4x32-10
 * (Salmon et al., SC'11) on n host records ctr_key[6n] = (c0, c1, c2, c3, k0,
 * k1) -> out[4n].  For testing the device arithmetic against independent
 * implementations.  Errors: DA_EINVAL, DA_ECUDA. */
da_status da_diag_expf(const float* x, float* y, int64_t n);
da_status da_diag_philox(const uint32_t* ctr_key, uint32_t* out, int64_t n);
/* Time to solution over a set of instances (Sec. IV, Algorithm 3), host
 * computation: B bootstrap resamples of the I instances (with replacement);
 * for each sampled instance a success probability p from its posterior
 * Beta(0.5 + hits, 0.5 + runs - hits) (Jeffreys prior), R99 = log(0.01) /
 * log(1 - p) (at least one run); tts_q[b] = tau times the q-th percentile
 * (0..100, linear interpolation between order statistics) of the R99 values
 * of resample b.  tau: time per run.  Random numbers: Philox4x32-10 of seed,
 * block (b, j, k, 6) for sampled instance j; Gamma draws by Marsaglia & Tsang,
 * normals by Box-Muller.  hits[I], runs[I], tts_q[B] host arrays.
 * Errors: DA_EINVAL (I < 1, B < 1, q outside [0, 100], hits > runs, ...). */
da_status da_tts_bootstrap(const int64_t* hits, const int64_t* runs, int32_t I, double tau, double q,
                           int32_t B, uint64_t seed, double* tts_q);

/* out[k] = q[k]-th percentile (0..100) of v[n], linear interpolation between
 * order statistics at position (n - 1) q / 100.  Host.  Errors: DA_EINVAL. */
da_status da_percentiles(const double* v, int64_t n, const double* q, int32_t nq, double* out);

/* The log-domain decision of the step kernels: da_diag_log_uniform returns
 * L[i] = log2 U (the hardware approximation the kernels keep for every draw)
 * for U = (w[i] >> 8) + 1, i.e. u = U 2^-24; da_diag_accept_log
 * returns, per trial (delta[i], beta[i], w[i]), bit 0 = the kernel's accept
 * decision and bit 1 = set when the trial fell in the band and was decided by
 * the exact test delta <= 0 || u < exp_neg(-fl(beta delta)). */
da_status da_diag_log_uniform(const uint32_t* w, float* L, int64_t n);
da_status da_diag_accept_log(const float* delta, const float* beta, const uint32_t* w, uint8_t* out, int64_t n);
/* The bounded wait used by every pipelined kernel (tensor-core recompute,
 * producer-warp step): out3[0] = 1 if a wait on an mbarrier that received its
 * arrival succeeded, out3[1] = 0 if a wait on an mbarrier that never receives
 * one gave up, out3[2] = nanoseconds that wait took (about ns, 1 <= ns <= 1e9).
 * No kernel hangs on a lost arrival: it records the failure and returns.
 * Errors: DA_EINVAL, DA_ECUDA. */
da_status da_diag_bounded_wait(int64_t ns, int64_t* out3);
/* The fixed-point conversions of the exact recompute (da_field_recompute) as
 * the kernels evaluate them, in integer arithmetic (got), beside the same
 * conversions through the 64-bit conversion instructions (ref):
 * da_diag_fixed:  got[i], ref[i] = round(w[i] 2^S[i]) to nearest, ties to even
 *                 (defined for |w[i] 2^S[i]| < 2^63);
 * da_diag_scaled: got[i], ref[i] = fl32(v[i]) 2^-S[i] (fl32 = round to nearest
 *                 even).  Host arrays of n entries.  Errors: DA_EINVAL, DA_ECUDA. */
da_status da_diag_fixed(const float* w, const int32_t* S, int64_t* got, int64_t* ref, int64_t n);
da_status da_diag_scaled(const int64_t* v, const int32_t* S, float* got, float* ref, int64_t n);

#ifdef __cplusplus
}
#endif
#endif /* DA_H */
