// da_internal.h -- structures shared by the library's kernels and its runtime
// (not part of the public ABI in include/da.h).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include <string>

struct da_ctx;

namespace da {

// Coupling types, with the values of da_dtype in include/da.h; kWInt8AsF32:
// int8 couplings held as exact fp32 for the step kernel (int32-exact fields in
// fp32, int64 energies), the form DA_INT8 contexts anneal with.
constexpr int kWInt8 = 0, kWFp32 = 1, kWInt16 = 2, kWInt8AsF32 = 3;

// Per-replica scalars kept in global memory between kernel launches.
// E and best hold int64 energies (int8 instances) or fp64 bit patterns (fp32).
struct alignas(32) ReplicaScalars {
    long long E;       // tracked energy after the last completed step
    long long best;    // lowest tracked energy seen
    long long flips;   // accepted flips
    uint32_t m;        // consecutive steps without an accepted flip (E_off = m * inc)
    uint32_t check;    // 1: the best-state test of the last step is still to be made
};

// Launch shape of the parallel-trial step: a group of G warps per replica,
// V variables per lane, so one replica spans Npad = 32 * V * G variables;
// lane l of warp w owns i = w*32V + 32v + l (v < V).
struct StepShape {
    int V = 0;
    int G = 0;
    int rpb = 0;  // replicas (groups) per block
    bool ws = false;  // G = 1 only: one replica per block, with a producer warp for its draws
    int npad() const { return 32 * V * G; }
    int nwords() const { return V * G; }
};

struct StepParams {
    const void* W = nullptr;      // [N][ldw] symmetric, zero diagonal (int8 or fp32)
    const void* Wc = nullptr;     // the same couplings in the warp row order, row pitch npad
                                  // (coal_W_bytes); required where step_uses_coal, unused otherwise
    const void* diag = nullptr;   // [N] int32 or fp32
    int N = 0;
    int ldw = 0;
    int R = 0;                    // replicas handled by this launch
    int npad = 0, nw = 0;
    void* h = nullptr;            // [R][npad] int32 / fp32 fields
    uint32_t* x = nullptr;        // [R][nw] state words
    uint32_t* bestx = nullptr;    // [R][nw] best-state words
    ReplicaScalars* sc = nullptr; // [R]
    const float* beta = nullptr;  // schedule, indexed by the global step t
    const float* betas = nullptr; // PT: beta of replica r is betas[temp_of[r]]
    const int* temp_of = nullptr;
    float inc = 0.f;
    uint64_t seed = 0;
    uint32_t round_key[2][10] = {};  // Philox round keys of seed (set by set_seed)
    uint32_t rep_base = 0;        // Philox replica id of replica r is rep_base + r
    long long t0 = 0, t1 = 0;     // steps [t0, t1)
    int* trace = nullptr;         // optional [R][trace_T]
    long long trace_T = 0;
    int* err = nullptr;           // device flag, set to 2 when a bounded wait gives up
    const int* stop = nullptr;    // optional flag (host-mapped): a launch that finds it
                                  // set returns at once (a cancelled request)
};

// Philox4x32-10 round keys k + r * Weyl (r = 0..9) of a seed.
inline void set_seed(StepParams& p, uint64_t seed)
{
    p.seed = seed;
    uint32_t a = (uint32_t)seed, b = (uint32_t)(seed >> 32);
    for (int r = 0; r < 10; ++r) {
        p.round_key[0][r] = a;
        p.round_key[1][r] = b;
        a += 0x9E3779B9u;
        b += 0xBB67AE85u;
    }
}

// Start state x = 0 of R replicas: fields g = diag (the effective field of
// x = 0), words and scalars zero (da_fields.cu).  float_fields: an integer
// diagonal written as fp32 fields (for kWInt8AsF32).
cudaError_t launch_init_state(bool is_int8, const void* diag, int N, int R, void* g, int npad, cudaStream_t st,
                              bool float_fields = false);

// The best-state test left pending by the last step of an anneal (made after
// any recompute of that step): if E < best, best = E and the state words are
// copied to the best-state words (da_fields.cu).
cudaError_t launch_best_fixup(int R, ReplicaScalars* sc, bool is_int8, const uint32_t* x, uint32_t* bestx, int nw,
                              cudaStream_t st);

// Step kernel launcher (da_step.cu).  is_int8 selects int8 W / int32 fields.
// wtype: the da_dtype of W (DA_INT8, DA_FP32, DA_INT16).
cudaError_t launch_step(int wtype, const StepShape& s, const StepParams& p, bool trace, cudaStream_t st);

// The step kernel (no producer warp) of the fp32 coupling forms (fp32, and int8
// held as exact fp32) at V >= 8 variables per lane reads its rows of W from a copy
// in another order, "the warp row order": in the 32 V entries of warp w's slice of
// a row, variable i = w 32 V + l V + v (lane l, slot v) sits at entry
// w 32 V + 128 (v / 4) + 4 l + v % 4, so that float4 number q of lane l (entries
// w 32 V + 128 q + 4 l .. + 3) holds the lane's slots 4 q .. 4 q + 3 and each
// 16-byte load instruction of the warp reads 512 contiguous bytes (in the plain
// order every lane's 16 bytes fall in a different 128-byte line).  Entries of
// padding variables (i >= N) are 0.  The copy is [N][32 V G] floats (the shape's
// padded width), 16-byte aligned (da_fields.cu).
bool step_uses_coal(int wtype, const StepShape& s);
size_t coal_W_bytes(int N, const StepShape& s);
cudaError_t launch_coalesce_W(const float* W, int N, int ldw, int V, int G, float* Wc, cudaStream_t st);
bool step_shape_supported(const StepShape& s);

// Field recompute and energies (da_fields.cu).
// Exact effective fields g = diag + W x of R bit-packed states xs[R][nw]
// (words of 32 variables): int8: in int32.  fp32: every W_ij and diag_i is
// put on the grid 2^-S, summed exactly in int64, and rounded once to fp32.
// hout[R][npad] (npad >= N) receives the fields (0 beyond N).  If
// E != nullptr, also writes the energy sum_{x_i=1} (d_i + g_i) / 2 (int64 or
// fp64 bit pattern) to E[r*Estride]; scratch must then hold
// 16 * ceil(max(npad, N) / 64) * R bytes.
cudaError_t launch_recompute(bool is_int8, const void* W, const void* diag, int N, int ldw, int S,
                             const uint32_t* xs, int nw, int R, void* hout, int npad,
                             long long* E, int Estride, cudaStream_t st, long long* scratch);

// The same for couplings of type wtype (kWInt8, kWFp32 or kWInt16; the integer
// types give int32 fields and int64 energies).
cudaError_t launch_recompute_w(int wtype, const void* W, const void* diag, int N, int ldw, int S,
                               const uint32_t* xs, int nw, int R, void* hout, int npad,
                               long long* E, int Estride, cudaStream_t st, long long* scratch);

// E[r * Estride] from the 128-bit partial sums part[tiles][R] of a recompute:
// the energy sum / 2^(S+1) (int64, or the fp64 bit pattern of its single
// rounding for fp32) (da_fields.cu).
cudaError_t launch_energy_sum(bool is_int8, const long long* part, int tiles, int R, int S, long long* E, int Estride,
                              cudaStream_t st);

// Tensor-core form of the same recompute (da_mma.cu), bit-identical to
// launch_recompute.  The operand holds the instance's couplings on the
// fixed-point grid (the int8 couplings themselves) split into `limbs`
// balanced digits of `bits` bits, each exact in f16, laid out for the tensor
// cores; `err` is a device flag set to 1 if a bounded wait inside the kernel
// gave up (the results of that call are then invalid).
struct TcOperand {
    void* B = nullptr;
    long long* dfix = nullptr;  // the diagonal on the same grid
    int* err = nullptr;
    int bits = 0, limbs = 0, kchunks = 0;
};
void tc_digits(int wtype, int N, int* bits, int* limbs);
cudaError_t tc_operand_build(int wtype, const void* W, const void* diag, int N, int ldw, int S, TcOperand* op,
                             cudaStream_t st);
void tc_operand_free(TcOperand* op);   // for operands from tc_operand_build
// The same operand built in caller-provided device memory (tc_operand_bytes(wtype,
// N) bytes, 256-byte aligned), nothing allocated; the caller frees mem.
size_t tc_operand_bytes(int wtype, int N);
cudaError_t tc_operand_build_in(int wtype, const void* W, const void* diag, int N, int ldw, int S, void* mem,
                                TcOperand* op, cudaStream_t st);
// Bytes of launch_recompute_tc's scratch for R states and `rows` = max(npad, N)
// field columns (hout given) or N (none): one 128-bit partial energy per state and
// 64-column tile.
size_t tc_partial_bytes(int rows, int R);
// Arguments as launch_recompute (is_int8: integer couplings of either width,
// int32 fields); with E, scratch must hold tc_partial_bytes(rows, R) bytes.
cudaError_t launch_recompute_tc(bool is_int8, const TcOperand& op, const void* diag, int N, int S,
                                const uint32_t* xs, int nw, int R, void* hout, int npad, long long* E, int Estride,
                                cudaStream_t st, long long* scratch);

// PT exchange (da_pt.cu).
cudaError_t launch_pt_exchange(bool is_int8, const float* betas, int K, int L,
                               const ReplicaScalars* sc, int* temp_of, int* rep_at,
                               long long* swaps, uint8_t* swap_trace, long long sweep, long long sweeps,
                               uint64_t seed, cudaStream_t st);

// Adaptive PTDA ladder update (da_pt.cu): betas[K] (device) from the exchange
// counts swaps[L][K-1] accumulated since the counts in seen[K-1] (updated),
// with `proposals` proposals per pair in the window.
cudaError_t launch_pt_adapt(float* betas, int K, int L, const long long* swaps, long long* seen, long long proposals,
                            cudaStream_t st);

// The plain one-launch-per-step form of the DA step (da_plain.cu), N <= 1024:
// ws holds plain_workspace_bytes(N, R); words_out [2R][ceil(N/32)] receives the
// final and best states, eex [2R] their exact energies (part: recompute
// scratch), tracked_E / flips [R] (host) the tracked energies and flip counts.
cudaError_t plain_anneal(const void* W, const void* diag, bool int8, int N, int ldw, int S, const float* beta_dev,
                         long long T, float inc, int R, uint64_t seed, void* ws, int* trace, uint32_t* words_out,
                         long long* eex, long long* part, double* tracked_E, int64_t* flips, cudaStream_t st);
size_t plain_workspace_bytes(int N, int R);

// An instance in the library's device layout: W symmetric with zero
// diagonal (element type of the da_dtype `dtype`), row pitch ldw, 8192 zero
// entries of slack (instance_W_bytes); diag (n x 4 bytes, int32 or fp32);
// fixed-point scale S (fp32).  build_instance (da_api.cu) checks the upper
// triangle of Q on the host and sets ldw and S; launch_expand_instance
// (da_fields.cu) writes W (unless null), the optional fp32 copy Wf of integer
// couplings and diag from a device copy of Q (int32 entries for the integer dtypes, fp32
// otherwise).
struct HostInstance {
    int ldw = 0, S = 0;
    bool exact_shift = false;   // fp32: every nonzero entry reaches the grid 2^-S by a left shift
};
size_t instance_W_bytes(int n, int dtype);
// Zeroes `bytes` bytes at p (device, 16-byte aligned) with a kernel of this
// library, so that zeroing takes the same on-chip memory split as the rest.
cudaError_t launch_zero(void* p, size_t bytes, cudaStream_t st);
// Sets the on-chip memory split (prefer_shared) of every step-kernel instance
// of coupling type wtype (da_step.cu), and of the instance build, state and
// recompute kernels (da_fields.cu), which also loads them: a kernel loaded on
// first use while other kernels run may wait for them.
cudaError_t prepare_step(int wtype);
cudaError_t prepare_field_kernels();
cudaError_t prepare_tc_kernels();   // da_mma.cu: the tensor-core recompute and its operand build

// An SM runs blocks of several kernels at once only under one split of its
// on-chip memory between L1 and shared memory.  Kernels that run beside the
// kernels of other requests ask for the split with the most shared memory, so
// that none of them holds its SMs in a split the others cannot use.  Called
// before a launch; the attribute is set once per kernel.
template <auto K>
inline void prefer_shared()
{
    static const bool once = [] {
        if (cudaFuncSetAttribute(reinterpret_cast<const void*>(K), cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared) != cudaSuccess)
            cudaGetLastError();
        return true;
    }();
    (void)once;
}
cudaError_t launch_expand_instance(const void* Q, int n, int ldw, int dtype, void* W, float* Wf, void* diag,
                                   cudaStream_t st);
bool build_instance(const void* Q, int n, int dtype, HostInstance& out, std::string& why);

// The default launch shape of the step kernel for N variables and R replicas.
StepShape default_shape(int N, int R);

// True when every entry of a host schedule is finite and >= 0 (the kernels'
// fast Metropolis test relies on beta >= 0).
inline bool schedule_ok(const float* beta, long long n)
{
    for (long long t = 0; t < n; ++t)
        if (!(beta[t] >= 0.f) || beta[t] == __builtin_huge_valf()) return false;
    return true;
}

// The library's device allocations (da_alloc.cu): cudaMalloc / cudaFree and
// cudaMallocFromPoolAsync / cudaFreeAsync with a count of live allocations,
// and the host-side failure injection of da_diag_fail_alloc.
cudaError_t dev_malloc(void** p, size_t bytes);
cudaError_t dev_free(void* p);
cudaError_t pool_malloc_async(void** p, size_t bytes, cudaMemPool_t pool, cudaStream_t st);
cudaError_t pool_free_async(void* p, cudaStream_t st);

// One instance of a batched launch as its kernel sees it (da_batch.cu); the
// request loop uses one item for a request that runs resident.
struct BatchItemDev {
    const void* W;          // couplings in the step kernel's form
    const void* Wc;         // the same in the warp row order (pitch 32 V; step_uses_coal), or null
    const void* diag;
    const float* beta;
    uint32_t* xs;           // [2R][nw]: final states, then best states
    ReplicaScalars* sc;     // [R]
    int* trace;             // [R][T] or null
    long long T;
    long long recompute_every;
    long long unit0;        // first unit of this item in its class
    uint64_t seed;
    int N, ldw, S, R;
    float inc;
    int exact_shift;        // fp32: the recompute may convert with shifts alone (HostInstance)
    const int* stop;        // optional (host-mapped): set, the anneal leaves at its next multiple of 1024 steps
};

// A whole anneal of R replicas of one item by one launch of the batched
// kernel (da_batch.cu): one warp per replica keeps its state in registers from
// the first step to the last (fp32 fields recomputed by the warp itself every
// recompute_every steps); writes xs and sc as the chunked launches do.
// wk: the step coupling form (kWInt8AsF32, kWFp32, kWInt16), V: lanes' width.
cudaError_t launch_resident_anneal(int wk, int V, const BatchItemDev* item_dev, unsigned long long* head_dev, int R,
                                   cudaStream_t st);
cudaError_t prepare_resident_kernels();

// The carveout of prefer_shared for a kernel given by address.
inline void prefer_shared_fn(const void* k)
{
    if (cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared) !=
        cudaSuccess)
        cudaGetLastError();
}

// Error text returned by da_last_error() on the calling thread (da_api.cu).
void set_last_error(const std::string& msg);

// Device copies of a context's instance: W (row pitch ldw), diag, and the
// fixed-point scale S of its fp32 recompute (da_api.cu).
// Wstep (may be null): the couplings in the step kernel's form (DA_INT8: exact
// fp32, kWInt8AsF32; otherwise W).
void ctx_device_view(const da_ctx* c, const void** W, const void** diag, int32_t* ldw, int32_t* S,
                     const void** Wstep = nullptr);
// The context's couplings in the one-warp row order for V variables per lane
// (built on first use), or null when they cannot be made (da_last_error says why).
const void* ctx_coal_W(da_ctx* c, int V);
// The context's tensor-core operand of W (built by da_create).
const TcOperand& ctx_tc_operand(const da_ctx* c);
// Whether the context's fp32 instance reaches its fixed-point grid by shifts alone.
bool ctx_exact_shift(const da_ctx* c);

// Fixed-point scale of the fp32 recompute for amax = max(|W_ij|, |diag_i|)
// and N variables (N + 1 terms per sum).
int fix_scale(float amax, int N);

}  // namespace da
