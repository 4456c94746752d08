// da_api.cu -- the C ABI of include/da.h: instance contexts, the blocking and
// asynchronous anneal, PTDA, exact energies and the field recompute.
//
// Runtime layout in HBM (per call, in the context's workspace):
//   h      [R][npad]   int32 / fp32 fields between step launches
//   xs     [2R][nw]    current states, then best states (adjacent, so the
//                      final exact evaluation treats them as 2R states)
//   sc     [R]         ReplicaScalars (tracked E, best E, flips, offset count)
//   sums   [N/64][2R] 128-bit partial energies of the exact recompute
//   E_ex   [2R]        exact energies of the final and best states
// The instance itself (symmetric W with row pitch ldw, and diag) lives in the
// context for its whole life.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "da.h"
#include "da_internal.h"

using da::ReplicaScalars;
using da::StepParams;
using da::StepShape;

namespace {

thread_local std::string g_err;

da_status fail(da_status s, const std::string& msg)
{
    g_err = msg;
    return s;
}

#define DA_CU(call)                                                                                    \
    do {                                                                                               \
        cudaError_t e_ = (call);                                                                       \
        if (e_ != cudaSuccess) return fail(DA_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

}  // namespace

struct da_ctx {
    int N = 0;
    da_dtype dtype = DA_INT8;
    int ldw = 0;
    int S = 0;  // fixed-point scale of the fp32 recompute
    bool exact_shift = false;  // fp32: every entry reaches the grid by a left shift
    int device = 0;
    void* W = nullptr;
    void* Wf = nullptr;  // DA_INT8: the couplings as exact fp32, for the step kernel
    void* Wc[6][4] = {};  // the step couplings in the warp row order, by (log2 V, log2 G) (step_uses_coal)
    void* diag = nullptr;
    da::TcOperand tc;  // digit planes of W for the tensor-core recompute
    void* ws = nullptr;
    size_t ws_bytes = 0;
    cudaStream_t stream = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    StepShape forced;  // V = 0: automatic
    bool draw_warp = false;  // G = 1 shapes: a producer warp computes the acceptance draws
    // optional per-launch timing of the step kernel (da_profile_*)
    bool prof = false;
    std::vector<cudaEvent_t> prof_ev;  // pairs around step launches
    size_t prof_used = 0;
    std::mutex mu;
};

namespace {

// Integer couplings (DA_INT8, DA_INT16): exact fields, exact int64 energies.
bool is_int(const da_ctx* c) { return c->dtype != DA_FP32; }

// The step kernel's coupling form: DA_INT8 contexts anneal on their couplings
// held as exact fp32 (the same values, FFMA updates, int64 energies).
int step_wtype(const da_ctx* c) { return c->dtype == DA_INT8 ? da::kWInt8AsF32 : (int)c->dtype; }
const void* step_W(const da_ctx* c) { return c->dtype == DA_INT8 ? c->Wf : c->W; }

// Default launch shape: one warp per replica up to N = 1024 (V <= 32
// variables per lane).  Beyond, the fewest warps per replica that cover N
// with V <= 32 (G = 2, 4 or 8), doubled while the launch has fewer than 1024
// warps (few replicas: more warps per replica keep the SMs busy); V the
// smallest supported width for that G.  Register budgets keep every choice in
// one wave for the replica counts that select it.
StepShape auto_shape(int N, int R)
{
    StepShape s;
    if (N <= 1024) {
        int V = 4;
        while (32 * V < N) V *= 2;
        s.V = V; s.G = 1; s.rpb = 4;
        return s;
    }
    auto width = [N](int G) {
        int V = G == 8 ? 8 : 4;
        while (32 * V * G < N) V *= 2;
        return V;
    };
    int G = 2;
    while (32 * 32 * G < N) G *= 2;
    while (G < 8 && (long long)R * G < 1024) G *= 2;
    s.G = G;
    s.V = width(G);
    s.rpb = G == 2 ? 2 : 1;
    return s;
}

// Launch shapes chosen by da_tune_shape, per (device, step coupling form, N,
// replicas), for every context of the process.
std::mutex g_shape_mu;
std::map<std::tuple<int, int, int, int>, StepShape> g_shape_cache;

StepShape shape_for(const da_ctx* c, int R)
{
    if (c->forced.V > 0) {
        StepShape s = c->forced;
        s.ws = s.ws || (s.G == 1 && c->draw_warp);
        return s;
    }
    {
        std::lock_guard<std::mutex> lk(g_shape_mu);
        auto f = g_shape_cache.find(std::make_tuple(c->device, step_wtype(c), c->N, R));
        if (f != g_shape_cache.end()) return f->second;
    }
    StepShape s = auto_shape(c->N, R);
    s.ws = s.G == 1 && c->draw_warp;
    return s;
}

da_status ensure_ws(da_ctx* c, size_t bytes)
{
    if (bytes <= c->ws_bytes) return DA_OK;
    if (c->ws) {
        cudaStreamSynchronize(c->stream);
        da::dev_free(c->ws);
        c->ws = nullptr;
        c->ws_bytes = 0;
    }
    cudaError_t e = da::dev_malloc(&c->ws, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(DA_ENOMEM, std::string("workspace of ") + std::to_string(bytes) + " bytes: " + cudaGetErrorString(e));
    }
    c->ws_bytes = bytes;
    return DA_OK;
}

// Workspace carve-up for one anneal-like call.
struct Layout {
    size_t h, xs, sc, sums, eex, beta, res, trace, pt, total;
};

Layout plan(const da_ctx* c, const StepShape& s, int R, long long T, bool with_beta, bool with_trace, size_t pt_bytes)
{
    Layout L{};
    size_t o = 0;
    auto take = [&](size_t bytes) { size_t at = o; o = align_up(o + bytes, 256); return at; };
    L.h = take((size_t)R * s.npad() * 4);
    L.xs = take((size_t)2 * R * s.nwords() * 4);
    L.sc = take((size_t)R * sizeof(ReplicaScalars));
    L.sums = take(da::tc_partial_bytes(std::max(s.npad(), c->N), 2 * R));
    L.eex = take((size_t)2 * R * 8);
    L.beta = take(with_beta ? (size_t)T * 4 : 0);
    L.res = take((size_t)4 * R * 8);
    L.trace = take(with_trace ? (size_t)R * T * 4 : 0);
    L.pt = take(pt_bytes);
    L.total = o;
    return L;
}

__global__ void finalize_kernel(bool int8, int R, const ReplicaScalars* sc, const long long* eex, double* final_E,
                                double* best_E, double* drift, int64_t* flips)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    double ef, eb, tracked;
    if (int8) {
        ef = (double)eex[r];
        eb = (double)eex[R + r];
        tracked = (double)sc[r].E;
    } else {
        ef = __longlong_as_double(eex[r]);
        eb = __longlong_as_double(eex[R + r]);
        tracked = __longlong_as_double(sc[r].E);
    }
    if (final_E) final_E[r] = ef;
    if (best_E) best_E[r] = eb;
    if (drift) drift[r] = fabs(tracked - ef);
    if (flips) flips[r] = sc[r].flips;
}

struct RunBuffers {
    char* base;
    Layout L;
    StepShape s;
    int R;
    void* h() const { return base + L.h; }
    uint32_t* x() const { return reinterpret_cast<uint32_t*>(base + L.xs); }
    uint32_t* bestx() const { return x() + (size_t)R * s.nwords(); }
    ReplicaScalars* sc() const { return reinterpret_cast<ReplicaScalars*>(base + L.sc); }
    long long* sums() const { return reinterpret_cast<long long*>(base + L.sums); }
    long long* eex() const { return reinterpret_cast<long long*>(base + L.eex); }
};

int log2_of(int v) { return 31 - __builtin_clz((unsigned)v); }

// The copy of the step couplings in the warp row order for shape s, built on the
// context's stream (and waited for) the first time a launch of that shape needs it.
void*& coal_slot(da_ctx* c, const StepShape& s) { return c->Wc[log2_of(s.V)][log2_of(s.G)]; }

da_status ensure_coal(da_ctx* c, const StepShape& s)
{
    if (!da::step_uses_coal(step_wtype(c), s) || coal_slot(c, s)) return DA_OK;
    void* p = nullptr;
    cudaError_t e = da::dev_malloc(&p, da::coal_W_bytes(c->N, s));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(DA_ENOMEM, std::string("row-ordered couplings: ") + cudaGetErrorString(e));
    }
    e = da::launch_coalesce_W(static_cast<const float*>(step_W(c)), c->N, c->ldw, s.V, s.G, static_cast<float*>(p),
                              c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        da::dev_free(p);
        return fail(DA_ECUDA, std::string("row-ordered couplings: ") + cudaGetErrorString(e));
    }
    coal_slot(c, s) = p;
    return DA_OK;
}

StepParams base_params(const da_ctx* c, const RunBuffers& b)
{
    StepParams p;
    p.W = step_W(c);
    p.Wc = da::step_uses_coal(step_wtype(c), b.s) ? c->Wc[log2_of(b.s.V)][log2_of(b.s.G)] : nullptr;
    p.diag = c->diag;
    p.N = c->N;
    p.ldw = c->ldw;
    p.R = b.R;
    p.npad = b.s.npad();
    p.nw = b.s.nwords();
    p.h = b.h();
    p.x = b.x();
    p.bestx = b.bestx();
    p.sc = b.sc();
    p.err = c->tc.err;
    return p;
}

// The start state of every replica: x = 0, so the effective fields are the
// linear terms and E = 0 (all runs start from the same state, Sec. II).
da_status reset_state(const da_ctx* c, const RunBuffers& b, cudaStream_t st)
{
    DA_CU(da::launch_init_state(is_int(c), c->diag, c->N, b.R, b.h(), b.s.npad(), st, c->dtype == DA_INT8));
    DA_CU(cudaMemsetAsync(b.x(), 0, (size_t)2 * b.R * b.s.nwords() * 4, st));
    DA_CU(cudaMemsetAsync(b.sc(), 0, (size_t)b.R * sizeof(ReplicaScalars), st));
    return DA_OK;
}

// Exact energies of the final and best states into eex[0..2R).
da_status evaluate(const da_ctx* c, const RunBuffers& b, cudaStream_t st)
{
    DA_CU(da::launch_recompute_tc(is_int(c), c->tc, c->diag, c->N, c->S, b.x(), b.s.nwords(), 2 * b.R, nullptr,
                                  b.s.npad(), b.eex(), 1, st, b.sums()));
    return DA_OK;
}

// After a call's stream work has completed: a bounded wait inside a kernel
// (the tensor-core recompute's pipeline, the step's producer/annealer
// handshake) that gave up invalidates the call's results.
da_status check_kernel_flag(da_ctx* c)
{
    int flag = 0;
    DA_CU(cudaMemcpy(&flag, c->tc.err, sizeof(int), cudaMemcpyDeviceToHost));
    if (flag) {
        DA_CU(cudaMemset(c->tc.err, 0, sizeof(int)));
        return fail(DA_ETIMEOUT, flag == 2 ? "step kernel: a bounded wait on the draw ring gave up"
                                           : "tensor-core recompute: a bounded wait on a pipeline barrier gave up");
    }
    return DA_OK;
}

// Next free pair of profiling events (created on first use).
da_status prof_pair(da_ctx* c, cudaEvent_t* a, cudaEvent_t* b)
{
    while (c->prof_used + 2 > c->prof_ev.size()) {
        cudaEvent_t e;
        DA_CU(cudaEventCreate(&e));
        c->prof_ev.push_back(e);
    }
    *a = c->prof_ev[c->prof_used];
    *b = c->prof_ev[c->prof_used + 1];
    c->prof_used += 2;
    return DA_OK;
}

// The anneal loop proper: steps [t_begin, T) in launches that end at every
// recompute point (fp32, absolute multiples of recompute_every) or every 2^14
// steps; beta_dev is indexed by the absolute step.
da_status run_anneal(da_ctx* c, const RunBuffers& b, const float* beta_dev, long long t_begin, long long T, float inc,
                     uint64_t seed, long long recompute_every, int* trace_dev, cudaStream_t st)
{
    if (da_status e = ensure_coal(c, b.s)) return e;
    StepParams p = base_params(c, b);
    p.beta = beta_dev;
    p.inc = inc;
    da::set_seed(p, seed);
    p.rep_base = 0;
    p.trace = trace_dev;
    p.trace_T = T;
    const bool rec = !is_int(c) && recompute_every > 0;
    for (long long t0 = t_begin; t0 < T; t0 = p.t1) {
        p.t0 = t0;
        p.t1 = std::min(T, t0 + (1ll << 14));
        if (rec) p.t1 = std::min(p.t1, (t0 / recompute_every + 1) * recompute_every);
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        if (c->prof) {
            if (da_status e = prof_pair(c, &e0, &e1)) return e;
            DA_CU(cudaEventRecord(e0, st));
        }
        DA_CU(da::launch_step(step_wtype(c), b.s, p, trace_dev != nullptr, st));
        if (e1) DA_CU(cudaEventRecord(e1, st));
        if (rec && p.t1 % recompute_every == 0) {
            DA_CU(da::launch_recompute_tc(false, c->tc, c->diag, c->N, c->S, b.x(), b.s.nwords(), b.R, b.h(),
                                          b.s.npad(), reinterpret_cast<long long*>(b.sc()),
                                          (int)(sizeof(ReplicaScalars) / 8), st, b.sums()));
        }
    }
    DA_CU(da::launch_best_fixup(b.R, b.sc(), is_int(c), b.x(), b.bestx(), b.s.nwords(), st));
    return DA_OK;
}

da_status check_ctx(const da_ctx* c)
{
    if (!c) return fail(DA_EINVAL, "null context");
    return DA_OK;
}

struct CtxLock {
    da_ctx* c;
    explicit CtxLock(da_ctx* cc) : c(cc)
    {
        c->mu.lock();
        cudaSetDevice(c->device);
    }
    ~CtxLock() { c->mu.unlock(); }
};

}  // namespace

namespace da {
// Integer couplings: range of every coupling (upper triangle) and
// |Q_ii| + sum_j |Q_ij| below row_limit; the rows are read in order.
static bool check_integer(const int32_t* q, int n, int32_t lo, int32_t hi, long long row_limit, const char* name,
                          std::string& why)
{
    std::vector<long long> rowabs(n, 0);
    for (int i = 0; i < n; ++i) {
        rowabs[i] += std::llabs((long long)q[(size_t)i * n + i]);
        for (int j = i + 1; j < n; ++j) {
            const int32_t v = q[(size_t)i * n + j];
            if (v < lo || v > hi) {
                why = std::string(name) + " coupling Q[" + std::to_string(i) + "][" + std::to_string(j) + "] = " +
                      std::to_string(v) + " outside [" + std::to_string(lo) + ", " + std::to_string(hi) + "]";
                return false;
            }
            rowabs[i] += std::abs(v);
            rowabs[j] += std::abs(v);
        }
    }
    for (int i = 0; i < n; ++i)
        if (rowabs[i] >= row_limit) {
            why = std::string(name) + " row " + std::to_string(i) + ": |Q_ii| + sum |Q_ij| too large for exact fields";
            return false;
        }
    return true;
}

bool build_instance(const void* Q, int n, int dtype, HostInstance& out, std::string& why)
{
    out.ldw = (int)align_up((size_t)n, 128);
    out.S = 0;
    if (dtype == DA_INT8) {
        if (!check_integer(static_cast<const int32_t*>(Q), n, -128, 127, 1ll << 24, "DA_INT8", why)) return false;
    } else if (dtype == DA_INT16) {
        if (!check_integer(static_cast<const int32_t*>(Q), n, -32767, 32767, 1ll << 31, "DA_INT16", why)) return false;
    } else {
        const float* q = static_cast<const float*>(Q);
        float amax = 0.f;
        for (int i = 0; i < n; ++i)
            for (int j = i; j < n; ++j) {
                const float v = q[(size_t)i * n + j];
                if (!std::isfinite(v)) {
                    why = "non-finite Q entry";
                    return false;
                }
                amax = std::max(amax, std::fabs(v));
            }
        out.S = fix_scale(amax, n);
        // every nonzero entry a normal number whose grid value round(v 2^S) needs no
        // rounding (a left shift of its significand): the warp-level recompute then
        // converts with a shift alone
        out.exact_shift = true;
        for (int i = 0; i < n && out.exact_shift; ++i)
            for (int j = i; j < n; ++j) {
                uint32_t b;
                std::memcpy(&b, q + (size_t)i * n + j, 4);
                const int E = (int)((b >> 23) & 0xFFu);
                if ((b & 0x7FFFFFFFu) != 0 && (E == 0 || E - 150 + out.S < 0)) {
                    out.exact_shift = false;
                    break;
                }
            }
    }
    return true;
}

size_t instance_W_bytes(int n, int dtype)
{
    const size_t esz = dtype == DA_INT8 ? 1 : dtype == DA_INT16 ? 2 : 4;
    // 8192 zero entries after the last row: a lane whose slice straddles N
    // reads up to the launch width (at most 8192) past the row start
    return ((size_t)n * align_up((size_t)n, 128) + 8192) * esz;
}

StepShape default_shape(int N, int R) { return auto_shape(N, R); }

void set_last_error(const std::string& msg) { g_err = msg; }
const TcOperand& ctx_tc_operand(const da_ctx* c) { return c->tc; }
bool ctx_exact_shift(const da_ctx* c) { return c->exact_shift; }

const void* ctx_coal_W(da_ctx* c, int V)
{
    StepShape s;
    s.V = V;
    s.G = 1;
    s.rpb = 1;
    if (!step_uses_coal(step_wtype(c), s) || ensure_coal(c, s) != DA_OK) return nullptr;
    return coal_slot(c, s);
}

void ctx_device_view(const da_ctx* c, const void** W, const void** diag, int32_t* ldw, int32_t* S, const void** Wstep)
{
    *W = c->W;
    if (Wstep) *Wstep = step_W(c);
    *diag = c->diag;
    *ldw = c->ldw;
    *S = c->S;
}
}  // namespace da

extern "C" {

int da_version(void) { return 100; }

int64_t da_words(int64_t N) { return N <= 0 ? 0 : (N + 31) / 32; }

const char* da_last_error(void) { return g_err.c_str(); }

da_status da_create(const void* Q, int64_t N, da_dtype dtype, da_ctx** out)
{
    g_err.clear();
    if (!out) return fail(DA_EINVAL, "out is null");
    *out = nullptr;
    if (!Q) return fail(DA_EINVAL, "Q is null");
    if (N < 1 || N > 8192) return fail(DA_EINVAL, "N must be in [1, 8192]");
    if (dtype != DA_INT8 && dtype != DA_FP32 && dtype != DA_INT16) return fail(DA_EINVAL, "unknown dtype");
    const int n = (int)N;
    da::HostInstance hin;
    std::string why;
    if (!da::build_instance(Q, n, (int)dtype, hin, why)) return fail(DA_EINVAL, why);
    const int ldw = hin.ldw;
    int dev = 0;
    DA_CU(cudaGetDevice(&dev));
    da_ctx* c = new (std::nothrow) da_ctx;
    if (!c) return fail(DA_ENOMEM, "host allocation");
    c->N = n;
    c->dtype = dtype;
    c->ldw = ldw;
    c->device = dev;
    c->S = hin.S;
    c->exact_shift = hin.exact_shift;
    auto bail = [&](da_status s, const std::string& m) {
        da_destroy(c);
        return fail(s, m);
    };
    cudaError_t e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&c->ev0);
    if (e == cudaSuccess) e = cudaEventCreate(&c->ev1);
    if (e != cudaSuccess) return bail(DA_ECUDA, std::string("stream/event: ") + cudaGetErrorString(e));
    // DA_INT8 also keeps its couplings as exact fp32, same pitch and slack
    const size_t qbytes = (size_t)n * n * 4;
    void* qd = nullptr;
    e = da::dev_malloc(&c->W, da::instance_W_bytes(n, (int)dtype));
    if (e == cudaSuccess) e = da::dev_malloc(&c->diag, (size_t)n * 4);
    if (e == cudaSuccess && dtype == DA_INT8) e = da::dev_malloc(&c->Wf, da::instance_W_bytes(n, DA_FP32));
    if (e == cudaSuccess) e = da::dev_malloc(&qd, qbytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (qd) da::dev_free(qd);
        return bail(DA_ENOMEM, std::string("instance: ") + cudaGetErrorString(e));
    }
    e = cudaMemcpyAsync(qd, Q, qbytes, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
        e = da::launch_expand_instance(qd, n, ldw, (int)dtype, c->W, static_cast<float*>(c->Wf), c->diag, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    const cudaError_t ef = da::dev_free(qd);
    if (e == cudaSuccess) e = ef;
    if (e != cudaSuccess) return bail(DA_ECUDA, std::string("instance upload: ") + cudaGetErrorString(e));
    e = da::tc_operand_build((int)dtype, c->W, c->diag, n, ldw, c->S, &c->tc, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return bail(e == cudaErrorMemoryAllocation ? DA_ENOMEM : DA_ECUDA,
                    std::string("tensor-core operand: ") + cudaGetErrorString(e));
    }
    // the row-ordered couplings of the default one-warp shape, so that an anneal in that
    // shape waits for nothing
    if (n <= 1024)
        if (da_status st = ensure_coal(c, auto_shape(n, 1024))) return bail(st, std::string(g_err));
    *out = c;
    return DA_OK;
}

da_status da_quantize(const float* Q, int64_t N, int32_t coupler_max, int32_t bias_max, int32_t* Qint,
                      double* scale)
{
    g_err.clear();
    if (!Q || !Qint || !scale || N < 1) return fail(DA_EINVAL, "need Q, Qint, scale and N >= 1");
    if (coupler_max < 1 || bias_max < 1 || coupler_max > (1 << 30) || bias_max > (1 << 30))
        return fail(DA_EINVAL, "limits must be in [1, 2^30]");
    const int64_t n = N;
    double qmax = 0.0, dmax = 0.0;
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = i; j < n; ++j) {
            const double v = Q[i * n + j];
            if (!std::isfinite(v)) return fail(DA_EINVAL, "non-finite Q entry");
            if (i == j) dmax = std::max(dmax, std::fabs(v));
            else qmax = std::max(qmax, std::fabs(v));
        }
    double s = 0.0;
    if (qmax > 0.0) s = (double)coupler_max / qmax;
    if (dmax > 0.0) s = s > 0.0 ? std::min(s, (double)bias_max / dmax) : (double)bias_max / dmax;
    if (!(s > 0.0)) s = 1.0;
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = 0; j < n; ++j) Qint[i * n + j] = j < i ? 0 : (int32_t)std::nearbyint(s * (double)Q[i * n + j]);
    *scale = s;
    return DA_OK;
}

void da_destroy(da_ctx* c)
{
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    if (c->W) da::dev_free(c->W);
    if (c->Wf) da::dev_free(c->Wf);
    for (auto& row : c->Wc)
        for (void* w : row)
            if (w) da::dev_free(w);
    if (c->diag) da::dev_free(c->diag);
    da::tc_operand_free(&c->tc);
    if (c->ws) da::dev_free(c->ws);
    for (cudaEvent_t e : c->prof_ev) cudaEventDestroy(e);
    if (c->ev0) cudaEventDestroy(c->ev0);
    if (c->ev1) cudaEventDestroy(c->ev1);
    if (c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

da_status da_ctx_info(const da_ctx* c, int64_t* N, da_dtype* dtype)
{
    if (da_status s = check_ctx(c)) return s;
    if (N) *N = c->N;
    if (dtype) *dtype = c->dtype;
    return DA_OK;
}

da_status da_set_draw_warp(da_ctx* c, int32_t on)
{
    if (da_status s = check_ctx(c)) return s;
    if (on != 0 && on != 1) return fail(DA_EINVAL, "on must be 0 or 1");
    c->draw_warp = on != 0;
    return DA_OK;
}

da_status da_set_launch_shape(da_ctx* c, int32_t V, int32_t G, int32_t rpb)
{
    if (da_status s = check_ctx(c)) return s;
    if (V == 0) {
        c->forced = StepShape{};
        return DA_OK;
    }
    StepShape s;
    s.V = V;
    s.G = G;
    s.rpb = rpb;
    if (!da::step_shape_supported(s)) return fail(DA_EINVAL, "unsupported launch shape");
    if (s.npad() < c->N) return fail(DA_EINVAL, "launch shape covers fewer than N variables");
    c->forced = s;
    return DA_OK;
}

static da_status anneal_common(da_ctx* c, const float* beta, bool beta_on_host, int64_t steps, float inc,
                               int32_t R, uint64_t seed, int64_t recompute_every, bool want_trace,
                               cudaStream_t st, RunBuffers* out_b)
{
    if (steps < 0) return fail(DA_EINVAL, "steps < 0");
    if (steps > 0 && !beta) return fail(DA_EINVAL, "beta schedule is null");
    if (R < 1) return fail(DA_EINVAL, "replicas < 1");
    if (steps >= (1ll << 32)) return fail(DA_EINVAL, "steps >= 2^32");
    if (!(inc >= 0.f) || !std::isfinite(inc)) return fail(DA_EINVAL, "offset_inc must be finite and >= 0");
    if (recompute_every < 0) return fail(DA_EINVAL, "recompute_every < 0");
    if (beta_on_host && !da::schedule_ok(beta, steps)) return fail(DA_EINVAL, "beta must be finite and >= 0");
    const StepShape s = shape_for(c, R);
    if (s.npad() < c->N) return fail(DA_EINVAL, "launch shape too small for N");
    const Layout L = plan(c, s, R, steps, beta_on_host, want_trace, 0);
    if (da_status e = ensure_ws(c, L.total)) return e;
    RunBuffers b{static_cast<char*>(c->ws), L, s, R};
    const float* beta_dev = beta;
    if (beta_on_host && steps > 0) {
        DA_CU(cudaMemcpyAsync(b.base + L.beta, beta, (size_t)steps * 4, cudaMemcpyHostToDevice, st));
        beta_dev = reinterpret_cast<const float*>(b.base + L.beta);
    }
    if (da_status e = reset_state(c, b, st)) return e;
    int* trace_dev = want_trace ? reinterpret_cast<int*>(b.base + L.trace) : nullptr;
    if (da_status e = run_anneal(c, b, beta_dev, 0, steps, inc, seed, recompute_every, trace_dev, st)) return e;
    if (da_status e = evaluate(c, b, st)) return e;
    *out_b = b;
    return DA_OK;
}

da_status da_anneal(da_ctx* c, const float* beta, int64_t steps, float inc, int32_t R, uint64_t seed,
                    int64_t recompute_every, da_result* out)
{
    g_err.clear();
    if (da_status s = check_ctx(c)) return s;
    CtxLock lock(c);
    const bool want_trace = out && out->trace;
    cudaStream_t st = c->stream;
    DA_CU(cudaEventRecord(c->ev0, st));
    RunBuffers b{};
    if (da_status e = anneal_common(c, beta, true, steps, inc, R, seed, recompute_every, want_trace, st, &b)) return e;
    double* res = reinterpret_cast<double*>(b.base + b.L.res);
    finalize_kernel<<<(R + 127) / 128, 128, 0, st>>>(is_int(c), R, b.sc(), b.eex(), res, res + R, res + 2 * R,
                                                     reinterpret_cast<int64_t*>(res + 3 * R));
    DA_CU(cudaGetLastError());
    DA_CU(cudaEventRecord(c->ev1, st));
    if (!out) {
        DA_CU(cudaStreamSynchronize(st));
        return check_kernel_flag(c);
    }
    const size_t words = (size_t)da_words(c->N);
    std::vector<double> hres((size_t)4 * R);
    DA_CU(cudaMemcpyAsync(hres.data(), res, hres.size() * 8, cudaMemcpyDeviceToHost, st));
    if (out->final_x)
        DA_CU(cudaMemcpy2DAsync(out->final_x, words * 4, b.x(), (size_t)b.s.nwords() * 4, words * 4, R,
                                cudaMemcpyDeviceToHost, st));
    if (out->best_x)
        DA_CU(cudaMemcpy2DAsync(out->best_x, words * 4, b.bestx(), (size_t)b.s.nwords() * 4, words * 4, R,
                                cudaMemcpyDeviceToHost, st));
    if (want_trace && steps > 0)
        DA_CU(cudaMemcpyAsync(out->trace, b.base + b.L.trace, (size_t)R * steps * 4, cudaMemcpyDeviceToHost, st));
    DA_CU(cudaStreamSynchronize(st));
    if (da_status e = check_kernel_flag(c)) return e;
    float ms = 0.f;
    DA_CU(cudaEventElapsedTime(&ms, c->ev0, c->ev1));
    out->elapsed_s = ms * 1e-3;
    for (int r = 0; r < R; ++r) {
        if (out->final_E) out->final_E[r] = hres[r];
        if (out->best_E) out->best_E[r] = hres[R + r];
        if (out->max_drift) out->max_drift[r] = hres[2 * R + r];
        if (out->flips) out->flips[r] = reinterpret_cast<const int64_t*>(hres.data() + 3 * R)[r];
    }
    return DA_OK;
}

da_status da_anneal_async(da_ctx* c, const float* beta_dev, int64_t steps, float inc, int32_t R, uint64_t seed,
                          int64_t recompute_every, const da_dev_result* out, void* stream)
{
    g_err.clear();
    if (da_status s = check_ctx(c)) return s;
    CtxLock lock(c);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const bool want_trace = out && out->trace;
    RunBuffers b{};
    if (da_status e = anneal_common(c, beta_dev, false, steps, inc, R, seed, recompute_every, want_trace, st, &b))
        return e;
    if (!out) return DA_OK;
    finalize_kernel<<<(R + 127) / 128, 128, 0, st>>>(is_int(c), R, b.sc(), b.eex(), out->final_E, out->best_E,
                                                     out->max_drift, out->flips);
    DA_CU(cudaGetLastError());
    const size_t words = (size_t)da_words(c->N);
    if (out->final_x)
        DA_CU(cudaMemcpy2DAsync(out->final_x, words * 4, b.x(), (size_t)b.s.nwords() * 4, words * 4, R,
                                cudaMemcpyDeviceToDevice, st));
    if (out->best_x)
        DA_CU(cudaMemcpy2DAsync(out->best_x, words * 4, b.bestx(), (size_t)b.s.nwords() * 4, words * 4, R,
                                cudaMemcpyDeviceToDevice, st));
    if (want_trace && steps > 0)
        DA_CU(cudaMemcpyAsync(out->trace, b.base + b.L.trace, (size_t)R * steps * 4, cudaMemcpyDeviceToDevice, st));
    return DA_OK;
}

static da_status pt_common(da_ctx* c, const float* betas, float* betas_final, int32_t K, int64_t sweeps, int32_t L,
                           float inc, uint64_t seed, int64_t adapt_every, int64_t adapt_sweeps, da_pt_result* out)
{
    if (da_status s = check_ctx(c)) return s;
    if (adapt_every < 0 || adapt_sweeps < 0) return fail(DA_EINVAL, "adapt_every and adapt_sweeps must be >= 0");
    if (!betas || K < 1 || K > 4096) return fail(DA_EINVAL, "need 1 <= K <= 4096 and betas");
    if (L < 1 || sweeps < 0) return fail(DA_EINVAL, "need ladders >= 1 and sweeps >= 0");
    if ((long long)L * K > (1 << 24)) return fail(DA_EINVAL, "too many replicas");
    if ((double)sweeps * c->N >= 4294967296.0) return fail(DA_EINVAL, "sweeps * N >= 2^32");
    if (!(inc >= 0.f) || !std::isfinite(inc)) return fail(DA_EINVAL, "offset_inc must be finite and >= 0");
    for (int k = 0; k < K; ++k) {
        if (!da::schedule_ok(betas + k, 1)) return fail(DA_EINVAL, "betas must be finite and >= 0");
        if (k > 0 && betas[k] < betas[k - 1]) return fail(DA_EINVAL, "betas must be ascending");
    }
    CtxLock lock(c);
    cudaStream_t st = c->stream;
    const int R = L * K;
    const StepShape s = shape_for(c, R);
    if (s.npad() < c->N) return fail(DA_EINVAL, "launch shape too small for N");
    const bool want_trace = out && out->swap_trace && K > 1;
    const size_t n_sw = (size_t)L * std::max(K - 1, 0);
    const size_t pt_bytes = align_up((size_t)K * 4, 256) + align_up((size_t)R * 4, 256) * 2 +
                            align_up(n_sw * 8, 256) + align_up((size_t)K * 8, 256) +
                            (want_trace ? n_sw * (size_t)sweeps : 0);
    const Layout Ly = plan(c, s, R, 0, false, false, pt_bytes);
    if (da_status e = ensure_ws(c, Ly.total)) return e;
    RunBuffers b{static_cast<char*>(c->ws), Ly, s, R};
    char* pb = b.base + Ly.pt;
    float* betas_dev = reinterpret_cast<float*>(pb);
    int* temp_of = reinterpret_cast<int*>(pb + align_up((size_t)K * 4, 256));
    int* rep_at = temp_of + align_up((size_t)R * 4, 256) / 4;
    long long* swaps = reinterpret_cast<long long*>(reinterpret_cast<char*>(rep_at) + align_up((size_t)R * 4, 256));
    long long* seen = reinterpret_cast<long long*>(reinterpret_cast<char*>(swaps) + align_up(n_sw * 8, 256));
    uint8_t* strace = want_trace ? reinterpret_cast<uint8_t*>(seen) + align_up((size_t)K * 8, 256) : nullptr;
    std::vector<int> init((size_t)R);
    for (int l = 0; l < L; ++l)
        for (int k = 0; k < K; ++k) init[(size_t)l * K + k] = k;
    DA_CU(cudaEventRecord(c->ev0, st));
    DA_CU(cudaMemcpyAsync(betas_dev, betas, (size_t)K * 4, cudaMemcpyHostToDevice, st));
    DA_CU(cudaMemcpyAsync(temp_of, init.data(), (size_t)R * 4, cudaMemcpyHostToDevice, st));
    DA_CU(cudaMemcpyAsync(rep_at, init.data(), (size_t)R * 4, cudaMemcpyHostToDevice, st));
    if (n_sw) DA_CU(cudaMemsetAsync(swaps, 0, n_sw * 8, st));
    DA_CU(cudaMemsetAsync(seen, 0, (size_t)K * 8, st));
    if (da_status e = reset_state(c, b, st)) return e;
    if (da_status e = ensure_coal(c, b.s)) return e;
    StepParams p = base_params(c, b);
    p.betas = betas_dev;
    p.temp_of = temp_of;
    p.inc = inc;
    da::set_seed(p, seed);
    for (long long sw = 0; sw < sweeps; ++sw) {
        p.t0 = sw * c->N;
        p.t1 = p.t0 + c->N;
        DA_CU(da::launch_step(step_wtype(c), s, p, false, st));
        DA_CU(da::launch_pt_exchange(is_int(c), betas_dev, K, L, b.sc(), temp_of, rep_at, swaps, strace, sw, sweeps,
                                     seed, st));
        if (adapt_every > 0 && (sw + 1) % adapt_every == 0 && sw + 1 <= adapt_sweeps)
            DA_CU(da::launch_pt_adapt(betas_dev, K, L, swaps, seen, (long long)L * adapt_every, st));
    }
    DA_CU(da::launch_best_fixup(R, b.sc(), is_int(c), b.x(), b.bestx(), s.nwords(), st));
    if (da_status e = evaluate(c, b, st)) return e;
    DA_CU(cudaEventRecord(c->ev1, st));
    std::vector<long long> eex((size_t)2 * R);
    DA_CU(cudaMemcpyAsync(eex.data(), b.eex(), eex.size() * 8, cudaMemcpyDeviceToHost, st));
    const size_t words = (size_t)da_words(c->N);
    if (out && out->best_x)
        DA_CU(cudaMemcpy2DAsync(out->best_x, words * 4, b.bestx(), (size_t)s.nwords() * 4, words * 4, R,
                                cudaMemcpyDeviceToHost, st));
    if (out && out->temp_of) DA_CU(cudaMemcpyAsync(out->temp_of, temp_of, (size_t)R * 4, cudaMemcpyDeviceToHost, st));
    if (out && out->swaps && n_sw)
        DA_CU(cudaMemcpyAsync(out->swaps, swaps, n_sw * 8, cudaMemcpyDeviceToHost, st));
    if (betas_final) DA_CU(cudaMemcpyAsync(betas_final, betas_dev, (size_t)K * 4, cudaMemcpyDeviceToHost, st));
    if (want_trace && sweeps > 0)
        DA_CU(cudaMemcpyAsync(out->swap_trace, strace, n_sw * (size_t)sweeps, cudaMemcpyDeviceToHost, st));
    DA_CU(cudaStreamSynchronize(st));
    if (da_status e = check_kernel_flag(c)) return e;
    if (!out) return DA_OK;
    float ms = 0.f;
    DA_CU(cudaEventElapsedTime(&ms, c->ev0, c->ev1));
    out->elapsed_s = ms * 1e-3;
    for (int r = 0; r < R; ++r) {
        const double ef = is_int(c) ? (double)eex[r] : reinterpret_cast<const double*>(eex.data())[r];
        const double eb = is_int(c) ? (double)eex[R + r] : reinterpret_cast<const double*>(eex.data())[R + r];
        if (out->final_E) out->final_E[r] = ef;
        if (out->best_E) out->best_E[r] = eb;
    }
    return DA_OK;
}

da_status da_pt(da_ctx* c, const float* betas, int32_t K, int64_t sweeps, int32_t L, float inc, uint64_t seed,
                da_pt_result* out)
{
    g_err.clear();
    return pt_common(c, betas, nullptr, K, sweeps, L, inc, seed, 0, 0, out);
}

da_status da_pt_adaptive(da_ctx* c, float* betas, int32_t K, int64_t sweeps, int32_t L, float inc, uint64_t seed,
                         int64_t adapt_every, int64_t adapt_sweeps, da_pt_result* out)
{
    g_err.clear();
    if (adapt_every < 1) return fail(DA_EINVAL, "adapt_every must be >= 1");
    return pt_common(c, betas, betas, K, sweeps, L, inc, seed, adapt_every, adapt_sweeps, out);
}

static da_status states_common(da_ctx* c, const uint32_t* x, int32_t R, void* h, double* E)
{
    if (da_status s = check_ctx(c)) return s;
    if (!x || R < 1) return fail(DA_EINVAL, "need states and R >= 1");
    CtxLock lock(c);
    cudaStream_t st = c->stream;
    const size_t words = (size_t)da_words(c->N);
    const size_t xb = align_up((size_t)R * words * 4, 256);
    const size_t hb = align_up((size_t)R * c->N * 4, 256);
    const size_t sb = align_up(da::tc_partial_bytes(c->N, R), 256);
    const size_t eb = align_up((size_t)R * 8, 256);
    if (da_status e = ensure_ws(c, xb + hb + sb + eb)) return e;
    char* base = static_cast<char*>(c->ws);
    uint32_t* xd = reinterpret_cast<uint32_t*>(base);
    void* hd = base + xb;
    long long* sums = reinterpret_cast<long long*>(base + xb + hb);
    long long* ed = reinterpret_cast<long long*>(base + xb + hb + sb);
    DA_CU(cudaMemcpyAsync(xd, x, (size_t)R * words * 4, cudaMemcpyHostToDevice, st));
    DA_CU(da::launch_recompute_tc(is_int(c), c->tc, c->diag, c->N, c->S, xd, (int)words, R, h ? hd : nullptr, c->N,
                                  E ? ed : nullptr, 1, st, sums));
    std::vector<long long> eh(E ? (size_t)R : 0);
    if (h) DA_CU(cudaMemcpyAsync(h, hd, (size_t)R * c->N * 4, cudaMemcpyDeviceToHost, st));
    if (E) DA_CU(cudaMemcpyAsync(eh.data(), ed, (size_t)R * 8, cudaMemcpyDeviceToHost, st));
    DA_CU(cudaStreamSynchronize(st));
    if (da_status e = check_kernel_flag(c)) return e;
    if (E)
        for (int r = 0; r < R; ++r)
            E[r] = is_int(c) ? (double)eh[r] : reinterpret_cast<const double*>(eh.data())[r];
    return DA_OK;
}

da_status da_anneal_plain(da_ctx* c, const float* beta, int64_t steps, float inc, int32_t R, uint64_t seed,
                          da_result* out)
{
    g_err.clear();
    if (da_status s = check_ctx(c)) return s;
    if (c->N > 1024) return fail(DA_EINVAL, "the plain form supports N <= 1024");
    if (c->dtype == DA_INT16) return fail(DA_EINVAL, "the plain form takes DA_INT8 or DA_FP32 contexts");
    if (steps < 0 || (steps > 0 && !beta)) return fail(DA_EINVAL, "bad schedule");
    if (!da::schedule_ok(beta, steps)) return fail(DA_EINVAL, "beta must be finite and >= 0");
    if (R < 1) return fail(DA_EINVAL, "replicas < 1");
    if (steps >= (1ll << 32)) return fail(DA_EINVAL, "steps >= 2^32");
    if (!(inc >= 0.f) || !std::isfinite(inc)) return fail(DA_EINVAL, "offset_inc must be finite and >= 0");
    CtxLock lock(c);
    cudaStream_t st = c->stream;
    const int nw = (c->N + 31) / 32;
    const size_t o_ws = 0;
    const size_t o_words = align_up(da::plain_workspace_bytes(c->N, R), 256);
    const size_t o_eex = o_words + align_up((size_t)2 * R * nw * 4, 256);
    const size_t o_part = o_eex + align_up((size_t)2 * R * 8, 256);
    const size_t o_beta = o_part + align_up((size_t)16 * ((c->N + 63) / 64) * 2 * R, 256);
    const size_t o_trace = o_beta + align_up((size_t)steps * 4, 256);
    const bool want_trace = out && out->trace;
    const size_t total = o_trace + (want_trace ? (size_t)R * steps * 4 : 0);
    if (da_status e = ensure_ws(c, total)) return e;
    char* base = static_cast<char*>(c->ws);
    std::vector<double> tracked((size_t)R);
    std::vector<int64_t> flips((size_t)R);
    DA_CU(cudaEventRecord(c->ev0, st));
    if (steps > 0) DA_CU(cudaMemcpyAsync(base + o_beta, beta, (size_t)steps * 4, cudaMemcpyHostToDevice, st));
    uint32_t* words = reinterpret_cast<uint32_t*>(base + o_words);
    long long* eex = reinterpret_cast<long long*>(base + o_eex);
    DA_CU(da::plain_anneal(c->W, c->diag, is_int(c), c->N, c->ldw, c->S, reinterpret_cast<const float*>(base + o_beta),
                           steps, inc, R, seed, base + o_ws, want_trace ? reinterpret_cast<int*>(base + o_trace) : nullptr,
                           words, eex, reinterpret_cast<long long*>(base + o_part), tracked.data(), flips.data(), st));
    DA_CU(cudaEventRecord(c->ev1, st));
    std::vector<long long> e((size_t)2 * R);
    DA_CU(cudaMemcpyAsync(e.data(), eex, e.size() * 8, cudaMemcpyDeviceToHost, st));
    if (out && out->final_x)
        DA_CU(cudaMemcpyAsync(out->final_x, words, (size_t)R * nw * 4, cudaMemcpyDeviceToHost, st));
    if (out && out->best_x)
        DA_CU(cudaMemcpyAsync(out->best_x, words + (size_t)R * nw, (size_t)R * nw * 4, cudaMemcpyDeviceToHost, st));
    if (want_trace && steps > 0)
        DA_CU(cudaMemcpyAsync(out->trace, base + o_trace, (size_t)R * steps * 4, cudaMemcpyDeviceToHost, st));
    DA_CU(cudaStreamSynchronize(st));
    if (da_status e = check_kernel_flag(c)) return e;
    if (!out) return DA_OK;
    float ms = 0.f;
    DA_CU(cudaEventElapsedTime(&ms, c->ev0, c->ev1));
    out->elapsed_s = ms * 1e-3;
    for (int r = 0; r < R; ++r) {
        const double ef = is_int(c) ? (double)e[r] : reinterpret_cast<const double*>(e.data())[r];
        const double eb = is_int(c) ? (double)e[R + r] : reinterpret_cast<const double*>(e.data())[R + r];
        if (out->final_E) out->final_E[r] = ef;
        if (out->best_E) out->best_E[r] = eb;
        if (out->max_drift) out->max_drift[r] = std::fabs(tracked[r] - ef);
        if (out->flips) out->flips[r] = flips[r];
    }
    return DA_OK;
}

da_status da_move_energy_percentiles(da_ctx* c, const uint32_t* x, int32_t R, const double* q, int32_t nq,
                                     double* out)
{
    g_err.clear();
    if (!q || !out || nq < 0) return fail(DA_EINVAL, "need q and out");
    if (da_status s = check_ctx(c)) return s;
    std::vector<char> h((size_t)std::max(R, 0) * c->N * 4);
    if (da_status s = states_common(c, x, R, h.data(), nullptr)) return s;
    const size_t words = (size_t)da_words(c->N);
    std::vector<double> up;
    up.reserve((size_t)R * c->N / 2);
    for (int r = 0; r < R; ++r)
        for (int i = 0; i < c->N; ++i) {
            const size_t at = (size_t)r * c->N + i;
            const double g = is_int(c) ? (double)reinterpret_cast<const int32_t*>(h.data())[at]
                                        : (double)reinterpret_cast<const float*>(h.data())[at];
            const bool xi = (x[(size_t)r * words + (i >> 5)] >> (i & 31)) & 1u;
            const double dE = xi ? -g : g;
            if (dE > 0.0) up.push_back(dE);
        }
    if (up.empty()) return fail(DA_EINVAL, "no proposed move raises the energy in these states");
    return da_percentiles(up.data(), (int64_t)up.size(), q, nq, out);
}

da_status da_profile_enable(da_ctx* c, int32_t on)
{
    g_err.clear();
    if (da_status s = check_ctx(c)) return s;
    CtxLock lock(c);
    c->prof = on != 0;
    c->prof_used = 0;
    return DA_OK;
}

da_status da_profile_read(da_ctx* c, int64_t* launches, double* total_ms)
{
    g_err.clear();
    if (da_status s = check_ctx(c)) return s;
    CtxLock lock(c);
    double ms = 0.0;
    for (size_t i = 0; i + 1 < c->prof_used; i += 2) {
        DA_CU(cudaEventSynchronize(c->prof_ev[i + 1]));
        float t = 0.f;
        DA_CU(cudaEventElapsedTime(&t, c->prof_ev[i], c->prof_ev[i + 1]));
        ms += t;
    }
    if (launches) *launches = (int64_t)(c->prof_used / 2);
    if (total_ms) *total_ms = ms;
    c->prof_used = 0;
    return DA_OK;
}

da_status da_energy(da_ctx* c, const uint32_t* x, int32_t R, double* E)
{
    g_err.clear();
    if (!E) return fail(DA_EINVAL, "E is null");
    return states_common(c, x, R, nullptr, E);
}

da_status da_field_recompute(da_ctx* c, const uint32_t* x, int32_t R, void* h)
{
    g_err.clear();
    if (!h) return fail(DA_EINVAL, "h is null");
    return states_common(c, x, R, h, nullptr);
}

}  // extern "C"

extern "C" da_status da_tune_shape(da_ctx* c, int32_t R, int64_t probe_steps, int32_t* V, int32_t* G, int32_t* rpb,
                                   int32_t* draw_warp)
{
    g_err.clear();
    if (da_status e = check_ctx(c)) return e;
    if (R < 1 || probe_steps < 1 || probe_steps > (1 << 20)) return fail(DA_EINVAL, "need R >= 1 and 1 <= probe_steps <= 2^20");
    CtxLock lock(c);
    // candidates: for each group size G the narrowest supported lane width that covers N, every
    // replicas-per-block the shape allows, and for G = 1 the producer-warp form
    std::vector<StepShape> cands;
    for (int g = 1; g <= 8; g *= 2) {
        StepShape s;
        s.G = g;
        for (int v = 4; v <= 32; v *= 2) {
            s.V = v;
            s.rpb = 1;
            if (da::step_shape_supported(s) && s.npad() >= c->N) break;
            s.V = 0;
        }
        if (s.V == 0) continue;
        if (s.npad() >= 4 * c->N && s.npad() > 128) continue;   // mostly idle lanes
        for (int r = 1; r <= 4; r *= 2) {
            s.rpb = r;
            if (!da::step_shape_supported(s)) continue;
            cands.push_back(s);
        }
        if (g == 1) {
            s.rpb = 1;
            s.ws = true;
            cands.push_back(s);
        }
    }
    if (cands.empty()) return fail(DA_EINVAL, "no launch shape covers N");
    const cudaStream_t st = c->stream;
    // probe schedule beta = 0: every trial is accepted, so every step flips (the common case of an
    // anneal over most of its schedule)
    const std::vector<float> beta((size_t)probe_steps, 0.0f);
    StepShape best = cands.front();
    float best_ms = 1e30f;
    for (const StepShape& s : cands) {
        const Layout L = plan(c, s, R, probe_steps, true, false, 0);
        if (da_status e = ensure_ws(c, L.total)) return e;
        RunBuffers b{static_cast<char*>(c->ws), L, s, R};
        DA_CU(cudaMemcpyAsync(b.base + L.beta, beta.data(), (size_t)probe_steps * 4, cudaMemcpyHostToDevice, st));
        const float* beta_dev = reinterpret_cast<const float*>(b.base + L.beta);
        float ms = 1e30f;
        for (int rep = 0; rep < 2; ++rep) {   // the first run also loads and configures the kernel
            if (da_status e = reset_state(c, b, st)) return e;
            if (da_status e = ensure_coal(c, b.s)) return e;
            StepParams p = base_params(c, b);
            p.beta = beta_dev;
            da::set_seed(p, 0x5eed);
            p.t0 = 0;
            p.t1 = probe_steps;
            DA_CU(cudaEventRecord(c->ev0, st));
            DA_CU(da::launch_step(step_wtype(c), s, p, false, st));
            DA_CU(cudaEventRecord(c->ev1, st));
            DA_CU(cudaEventSynchronize(c->ev1));
            float t = 0.f;
            DA_CU(cudaEventElapsedTime(&t, c->ev0, c->ev1));
            ms = std::min(ms, t);
        }
        if (da_status e = check_kernel_flag(c)) return e;
        if (ms < best_ms) {
            best_ms = ms;
            best = s;
        }
    }
    {
        std::lock_guard<std::mutex> lk(g_shape_mu);
        g_shape_cache[std::make_tuple(c->device, step_wtype(c), c->N, (int)R)] = best;
    }
    if (V) *V = best.V;
    if (G) *G = best.G;
    if (rpb) *rpb = best.rpb;
    if (draw_warp) *draw_warp = best.ws ? 1 : 0;
    return DA_OK;
}

namespace {

// A checkpoint into the workspace layout of an anneal: fields [R][npad] (zero
// padding), state words [2R][nw] (current, then best), scalars.  Host vectors
// that stage converted data are kept in `keep` until the stream is synchronised.
da_status restore_state(const da_ctx* c, const RunBuffers& b, const da_checkpoint* in, cudaStream_t st,
                        std::vector<std::vector<char>>& keep)
{
    const int R = b.R, N = c->N, npad = b.s.npad(), nw = b.s.nwords();
    const size_t words = (size_t)da_words(N);
    DA_CU(cudaMemsetAsync(b.h(), 0, (size_t)R * npad * 4, st));
    DA_CU(cudaMemsetAsync(b.x(), 0, (size_t)2 * R * nw * 4, st));
    const void* fsrc = in->fields;
    if (c->dtype == DA_INT8) {   // int32 fields, held as exact fp32 by the step kernel
        keep.emplace_back((size_t)R * N * 4);
        float* f = reinterpret_cast<float*>(keep.back().data());
        const int32_t* g = static_cast<const int32_t*>(in->fields);
        for (size_t k = 0; k < (size_t)R * N; ++k) f[k] = (float)g[k];
        fsrc = f;
    }
    DA_CU(cudaMemcpy2DAsync(b.h(), (size_t)npad * 4, fsrc, (size_t)N * 4, (size_t)N * 4, R, cudaMemcpyHostToDevice, st));
    DA_CU(cudaMemcpy2DAsync(b.x(), (size_t)nw * 4, in->x, words * 4, words * 4, R, cudaMemcpyHostToDevice, st));
    DA_CU(cudaMemcpy2DAsync(b.bestx(), (size_t)nw * 4, in->best_x, words * 4, words * 4, R, cudaMemcpyHostToDevice,
                            st));
    keep.emplace_back((size_t)R * sizeof(ReplicaScalars));
    ReplicaScalars* sc = reinterpret_cast<ReplicaScalars*>(keep.back().data());
    for (int r = 0; r < R; ++r) {
        sc[r] = ReplicaScalars{};
        sc[r].E = in->scalars[4 * r];
        sc[r].best = in->scalars[4 * r + 1];
        sc[r].flips = in->scalars[4 * r + 2];
        sc[r].m = (uint32_t)in->scalars[4 * r + 3];
        sc[r].check = 0;
    }
    DA_CU(cudaMemcpyAsync(b.sc(), sc, (size_t)R * sizeof(ReplicaScalars), cudaMemcpyHostToDevice, st));
    return DA_OK;
}

// The workspace after a segment (its best-state test resolved) into a
// checkpoint; the copies complete at the next synchronisation of st, then
// finish_saved converts what the step kernel holds in another form.
da_status save_state(const da_ctx* c, const RunBuffers& b, da_checkpoint* out, cudaStream_t st,
                     std::vector<std::vector<char>>& keep)
{
    const int R = b.R, N = c->N, npad = b.s.npad(), nw = b.s.nwords();
    const size_t words = (size_t)da_words(N);
    if (out->fields)
        DA_CU(cudaMemcpy2DAsync(out->fields, (size_t)N * 4, b.h(), (size_t)npad * 4, (size_t)N * 4, R,
                                cudaMemcpyDeviceToHost, st));
    if (out->x)
        DA_CU(cudaMemcpy2DAsync(out->x, words * 4, b.x(), (size_t)nw * 4, words * 4, R, cudaMemcpyDeviceToHost, st));
    if (out->best_x)
        DA_CU(cudaMemcpy2DAsync(out->best_x, words * 4, b.bestx(), (size_t)nw * 4, words * 4, R,
                                cudaMemcpyDeviceToHost, st));
    if (out->scalars) {
        keep.emplace_back((size_t)R * sizeof(ReplicaScalars));
        DA_CU(cudaMemcpyAsync(keep.back().data(), b.sc(), (size_t)R * sizeof(ReplicaScalars), cudaMemcpyDeviceToHost,
                              st));
    }
    return DA_OK;
}

void finish_saved(const da_ctx* c, int R, da_checkpoint* out, const std::vector<char>* sc_bytes)
{
    if (out->fields && c->dtype == DA_INT8) {   // exact fp32 integers back to int32, in place
        char* p = static_cast<char*>(out->fields);
        for (size_t k = 0; k < (size_t)R * c->N; ++k) {
            float f;
            std::memcpy(&f, p + 4 * k, 4);
            const int32_t g = (int32_t)f;
            std::memcpy(p + 4 * k, &g, 4);
        }
    }
    if (out->scalars && sc_bytes) {
        const ReplicaScalars* sc = reinterpret_cast<const ReplicaScalars*>(sc_bytes->data());
        for (int r = 0; r < R; ++r) {
            out->scalars[4 * r] = sc[r].E;
            out->scalars[4 * r + 1] = sc[r].best;
            out->scalars[4 * r + 2] = sc[r].flips;
            out->scalars[4 * r + 3] = (int64_t)sc[r].m;
        }
    }
}

}  // namespace

extern "C" da_status da_anneal_segment(da_ctx* c, const float* beta, int64_t total_steps, int64_t t0, int64_t t1,
                                       float inc, int32_t R, uint64_t seed, int64_t recompute_every,
                                       const da_checkpoint* in, da_checkpoint* out, da_result* res)
{
    g_err.clear();
    if (da_status e = check_ctx(c)) return e;
    if (!(0 <= t0 && t0 <= t1 && t1 <= total_steps && total_steps < (1ll << 32)))
        return fail(DA_EINVAL, "need 0 <= t0 <= t1 <= total_steps < 2^32");
    if (!in && t0 != 0) return fail(DA_EINVAL, "a segment that does not start at step 0 needs a checkpoint");
    if (in && (!in->x || !in->best_x || !in->fields || !in->scalars)) return fail(DA_EINVAL, "incomplete checkpoint");
    if (res && res->trace) return fail(DA_EINVAL, "segments write no trace");
    if (R < 1) return fail(DA_EINVAL, "replicas < 1");
    if (t1 > 0 && !beta) return fail(DA_EINVAL, "beta schedule is null");
    if (!(inc >= 0.f) || !std::isfinite(inc)) return fail(DA_EINVAL, "offset_inc must be finite and >= 0");
    if (recompute_every < 0) return fail(DA_EINVAL, "recompute_every < 0");
    if (t1 > 0 && !da::schedule_ok(beta, t1)) return fail(DA_EINVAL, "beta must be finite and >= 0");
    CtxLock lock(c);
    const cudaStream_t st = c->stream;
    const StepShape s = shape_for(c, R);
    if (s.npad() < c->N) return fail(DA_EINVAL, "launch shape too small for N");
    const Layout L = plan(c, s, R, t1, true, false, 0);
    if (da_status e = ensure_ws(c, L.total)) return e;
    RunBuffers b{static_cast<char*>(c->ws), L, s, R};
    std::vector<std::vector<char>> keep;
    DA_CU(cudaEventRecord(c->ev0, st));
    const float* beta_dev = reinterpret_cast<const float*>(b.base + L.beta);
    if (t1 > 0) DA_CU(cudaMemcpyAsync(b.base + L.beta, beta, (size_t)t1 * 4, cudaMemcpyHostToDevice, st));
    if (in) {
        if (da_status e = restore_state(c, b, in, st, keep)) return e;
    } else if (da_status e = reset_state(c, b, st)) {
        return e;
    }
    if (da_status e = run_anneal(c, b, beta_dev, t0, t1, inc, seed, recompute_every, nullptr, st)) return e;
    if (da_status e = evaluate(c, b, st)) return e;
    double* resd = reinterpret_cast<double*>(b.base + L.res);
    finalize_kernel<<<(R + 127) / 128, 128, 0, st>>>(is_int(c), R, b.sc(), b.eex(), resd, resd + R, resd + 2 * R,
                                                     reinterpret_cast<int64_t*>(resd + 3 * R));
    DA_CU(cudaGetLastError());
    DA_CU(cudaEventRecord(c->ev1, st));
    std::vector<double> hres((size_t)4 * R);
    DA_CU(cudaMemcpyAsync(hres.data(), resd, hres.size() * 8, cudaMemcpyDeviceToHost, st));
    const size_t words = (size_t)da_words(c->N);
    if (res && res->final_x)
        DA_CU(cudaMemcpy2DAsync(res->final_x, words * 4, b.x(), (size_t)s.nwords() * 4, words * 4, R,
                                cudaMemcpyDeviceToHost, st));
    if (res && res->best_x)
        DA_CU(cudaMemcpy2DAsync(res->best_x, words * 4, b.bestx(), (size_t)s.nwords() * 4, words * 4, R,
                                cudaMemcpyDeviceToHost, st));
    const size_t sc_idx = keep.size();
    if (out)
        if (da_status e = save_state(c, b, out, st, keep)) return e;
    DA_CU(cudaStreamSynchronize(st));
    if (da_status e = check_kernel_flag(c)) return e;
    if (out) finish_saved(c, R, out, out->scalars ? &keep[sc_idx] : nullptr);
    if (res) {
        float ms = 0.f;
        DA_CU(cudaEventElapsedTime(&ms, c->ev0, c->ev1));
        res->elapsed_s = ms * 1e-3;
        for (int r = 0; r < R; ++r) {
            if (res->final_E) res->final_E[r] = hres[r];
            if (res->best_E) res->best_E[r] = hres[R + r];
            if (res->max_drift) res->max_drift[r] = hres[2 * R + r];
            if (res->flips) res->flips[r] = reinterpret_cast<const int64_t*>(hres.data() + 3 * R)[r];
        }
    }
    return DA_OK;
}
