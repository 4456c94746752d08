// da_serve.cu -- the request loop: da_server_create / da_submit / da_poll.
//
// Admission: a request (one QUBO, its schedule and replica count) waits in a
// FIFO until its device memory fits the server's HBM budget and a request slot
// is free.  Then all of its work is queued on a stream of its own, without any
// host synchronisation: allocation from the server's memory pool, the upload
// of Q and the schedule, the instance build, the anneal as chunked step
// launches (the same kernels and launch shapes as a context; fp32 fields
// recomputed every recompute_every steps on the tensor cores, from an operand
// built in the request's own memory), the exact evaluation of the final and
// best states, and an event.  Requests run concurrently, each on its own
// stream, so one that arrives while others are on the GPU starts at once on
// the SMs they leave free (continuous batching at the granularity of kernels).
//
// Every kernel of this path takes the split of on-chip memory with the most
// shared memory (prefer_shared in da_internal.h): an SM runs blocks of several
// kernels at once only under one split, and a kernel left to the default
// would hold its SMs in a split where the next request's kernels cannot start
// until it ends.
//
// A worker thread admits, polls completion events, copies results and frees
// memory; da_poll waits on a request with a timeout.  da_cancel takes a queued
// request out of the queue, and makes a running one's remaining step launches
// return at once (a host-mapped stop flag per request slot that every step
// launch reads when it starts).
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "da.h"
#include "da_internal.h"

namespace da {

// Finalises a request: exact energies into E[3R], flips.
__global__ void serve_finalize_kernel(bool int8, int R, const ReplicaScalars* sc, const long long* eex, double* E,
                                      long long* flips)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    const double ef = int8 ? (double)eex[r] : __longlong_as_double(eex[r]);
    const double eb = int8 ? (double)eex[R + r] : __longlong_as_double(eex[R + r]);
    const double tr = int8 ? (double)sc[r].E : __longlong_as_double(sc[r].E);
    E[r] = ef;
    E[R + r] = eb;
    E[2 * R + r] = fabs(tr - ef);
    flips[r] = sc[r].flips;
}

}  // namespace da

// ---------------------------------------------------------------------------
// Host side.
namespace {

using Clock = std::chrono::steady_clock;

size_t al256(size_t v) { return (v + 255) / 256 * 256; }

// Admission stops while the running requests' step launches hold this many
// warps per SM: beyond it further requests would only share the SMs (and L2)
// with those already running, which stretches every request's latency.
constexpr int kWarpsPerSm = 8;

enum class ReqState { Queued, Running, Done, Failed };

struct Req {
    da_job job;
    int N = 0;
    bool integer = false;             // DA_INT8 or DA_INT16: exact fields and energies
    int dtype = DA_FP32;
    da::StepShape shape;              // launch shape of the step kernel
    da::HostInstance inst;            // checked at submit (ldw, S); W and diag built on the device at admission
    size_t bytes = 0;                 // device bytes charged to the budget
    size_t qcopy = 0;                 // the transient device copy of Q (N*N*4 bytes), charged
    bool qcopy_held = false;          //   to the budget from admission until the instance is built
    bool cancelled = false;           // da_cancel on a running request
    int slot = -1;
    ReqState state = ReqState::Queued;
    da_status err = DA_OK;
    std::string msg;
    char* dmem = nullptr;
    // offsets into dmem
    size_t o_Wc = 0;                  // the step couplings in the warp row order (0: not used)
    size_t o_W = 0, o_Wf = 0, o_diag = 0, o_beta = 0, o_h = 0, o_xs = 0, o_sc = 0, o_part = 0, o_eex = 0, o_E = 0,
           o_flips = 0, o_tc = 0, o_item = 0;
    bool resident = false;            // the whole anneal in one launch, replica state in registers
    da::BatchItemDev item{};          // its descriptor (copied to dmem + o_item)
    da::TcOperand tc;                 // fp32 requests: the tensor-core operand of W (in dmem)
    int tc_err = 0;                   // its bounded-wait flag, read back with the results
    int xs_stride = 0;                // words per replica in xs
    // results on the host
    std::vector<double> E;            // [3R]
    std::vector<uint32_t> xs;         // [2R][xs_stride]
    std::vector<long long> flips;     // [R]
    Clock::time_point t_submit, t_done;
    cudaStream_t stream = nullptr;    // from the server's stream pool while running
    cudaEvent_t done_ev = nullptr;
    cudaEvent_t built_ev = nullptr;   // recorded after the copy of Q is freed
};

}  // namespace

struct da_req {
    std::shared_ptr<Req> r;
    da_server* srv;
};

struct da_server {
    int dev = 0;
    int64_t budget = 0, used = 0;
    // warps of the running requests' step launches, and the most admitted at
    // once (a request is admitted alone whatever its size)
    long long warps = 0, warp_cap = 0;
    int max_slots = 0;
    std::atomic<int> resident_max_n{0};   // requests of at most this many variables run resident
    std::vector<int> free_slots;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<std::shared_ptr<Req>> pending;
    std::vector<std::shared_ptr<Req>> active;
    std::thread worker;
    bool quit = false;
    // streams and events of finished requests, kept for the next ones
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> events;
    // requests' device memory: a pool of the server's own that keeps what it
    // has reserved (a pool that trims at every synchronisation unmaps memory,
    // which waits for the running kernels)
    cudaMemPool_t pool = nullptr;
    // a stop flag per request slot in host-mapped memory, read by every step
    // launch of the request in that slot (set by da_cancel)
    int* stop = nullptr;
    // statistics
    long long kernel_launches = 0, completed = 0;
};

namespace {

da_status sfail(da_status s, const std::string& m)
{
    da::set_last_error(m);
    return s;
}

bool cu_ok_static(cudaError_t e, Req& q, const char* what)
{
    if (e == cudaSuccess) return true;
    cudaGetLastError();
    q.err = DA_ECUDA;
    q.msg = std::string(what) + ": " + cudaGetErrorString(e);
    return false;
}

// Device bytes of a request and its buffer offsets.
void plan_request(Req& q)
{
    const int R = q.job.replicas;
    const da::StepShape& sh = q.shape;
    size_t o = 0;
    auto take = [&](size_t b) { size_t at = o; o += al256(b); return at; };
    // W in the request's coupling type (what the exact final evaluation reads);
    // int8 requests anneal on the same couplings held as exact fp32 (Wf)
    q.o_W = take(da::instance_W_bytes(q.N, q.dtype));
    if (q.dtype == DA_INT8) q.o_Wf = take(da::instance_W_bytes(q.N, DA_FP32));
    q.o_diag = take((size_t)q.N * 4);
    q.o_Wc = 0;
    if (da::step_uses_coal(q.dtype == DA_INT8 ? da::kWInt8AsF32 : q.dtype, sh) && !q.resident)
        q.o_Wc = take(da::coal_W_bytes(q.N, sh));
    q.o_beta = take((size_t)q.job.steps * 4);
    q.xs_stride = sh.nwords();
    q.o_h = take((size_t)R * sh.npad() * 4);
    q.o_xs = take((size_t)2 * R * q.xs_stride * 4);
    q.o_sc = take((size_t)R * sizeof(da::ReplicaScalars));
    // partial energies of the exact evaluation: 64-column tiles on the tensor cores and on the
    // CUDA cores (integer requests)
    q.o_part = take(da::tc_partial_bytes(std::max(sh.npad(), q.N), 2 * R));
    q.o_eex = take((size_t)2 * R * 8);
    q.o_E = take((size_t)3 * R * 8);
    q.o_flips = take((size_t)R * 8);
    if (q.resident) q.o_item = take(sizeof(da::BatchItemDev) + 16);   // descriptor, then the work counter
    if (!q.integer)     // the tensor-core recompute's operand of W
        q.o_tc = take(da::tc_operand_bytes(da::kWFp32, q.N));
    q.bytes = o;
    q.qcopy = al256((size_t)q.N * q.N * 4);
}

// Device bytes a request holds at its peak (its buffers and the copy of Q).
size_t peak_bytes(const Req& q) { return q.bytes + q.qcopy; }

// Takes an event from the server's pool or creates one.
bool take_event(da_server* s, Req& q, cudaEvent_t* ev)
{
    if (!s->events.empty()) {
        *ev = s->events.back();
        s->events.pop_back();
        return true;
    }
    return cu_ok_static(cudaEventCreateWithFlags(ev, cudaEventDisableTiming), q, "event");
}

bool cu_ok(cudaError_t e, Req& q, const char* what) { return cu_ok_static(e, q, what); }

// Queue all of an admitted request's work on its stream.  Runs on the worker
// thread and returns without waiting for the GPU.
bool admit(da_server* s, Req& q, long long& launches)
{
    if (!s->streams.empty()) {
        q.stream = s->streams.back();
        s->streams.pop_back();
    } else if (!cu_ok(cudaStreamCreateWithFlags(&q.stream, cudaStreamNonBlocking), q, "stream")) {
        return false;
    }
    if (!take_event(s, q, &q.done_ev) || !take_event(s, q, &q.built_ev)) return false;
    cudaStream_t st = q.stream;
    if (da::pool_malloc_async(reinterpret_cast<void**>(&q.dmem), q.bytes, s->pool, st) != cudaSuccess) {
        cudaGetLastError();
        q.dmem = nullptr;
        q.err = DA_ENOMEM;
        q.msg = "device allocation of " + std::to_string(q.bytes) + " bytes";
        return false;
    }
    const int R = q.job.replicas;
    void* W = q.dmem + q.o_W;
    void* Wf = q.dtype == DA_INT8 ? q.dmem + q.o_Wf : nullptr;
    void* diag = q.dmem + q.o_diag;
    // W and diag from a transient device copy of Q (the caller keeps Q valid)
    {
        void* qd = nullptr;
        const size_t qbytes = (size_t)q.N * q.N * 4;
        if (da::pool_malloc_async(&qd, qbytes, s->pool, st) != cudaSuccess) {
            cudaGetLastError();
            q.err = DA_ENOMEM;
            q.msg = "device allocation of " + std::to_string(qbytes) + " bytes (copy of Q)";
            return false;
        }
        bool ok = cu_ok(cudaMemcpyAsync(qd, q.job.Q, qbytes, cudaMemcpyHostToDevice, st), q, "upload Q");
        ok = ok && cu_ok(da::launch_expand_instance(qd, q.N, q.inst.ldw, q.dtype, W,
                                                    static_cast<float*>(Wf), diag, st),
                         q, "build instance");
        launches += 3;
        da::pool_free_async(qd, st);
        if (!ok || !cu_ok(cudaEventRecord(q.built_ev, st), q, "event")) return false;
    }
    if (!q.integer) {
        if (!cu_ok(da::tc_operand_build_in(da::kWFp32, W, diag, q.N, q.inst.ldw, q.inst.S, q.dmem + q.o_tc, &q.tc, st),
                   q, "tensor-core operand"))
            return false;
        launches += 2;
    }
    void* Wc = q.o_Wc ? q.dmem + q.o_Wc : nullptr;
    if (Wc) {
        if (!cu_ok(da::launch_coalesce_W(static_cast<const float*>(q.dtype == DA_INT8 ? Wf : W), q.N, q.inst.ldw,
                                         q.shape.V, q.shape.G, static_cast<float*>(Wc), st),
                   q, "row-ordered couplings"))
            return false;
        launches += 1;
    }
    if (q.job.steps > 0 &&
        !cu_ok(cudaMemcpyAsync(q.dmem + q.o_beta, q.job.beta, (size_t)q.job.steps * 4, cudaMemcpyHostToDevice, st), q,
               "upload beta"))
        return false;
    const da::StepShape sh = q.shape;
    void* h = q.dmem + q.o_h;
    uint32_t* xs = reinterpret_cast<uint32_t*>(q.dmem + q.o_xs);
    da::ReplicaScalars* sc = reinterpret_cast<da::ReplicaScalars*>(q.dmem + q.o_sc);
    long long* part = reinterpret_cast<long long*>(q.dmem + q.o_part);
    long long* eex = reinterpret_cast<long long*>(q.dmem + q.o_eex);
    double* E = reinterpret_cast<double*>(q.dmem + q.o_E);
    long long* flips = reinterpret_cast<long long*>(q.dmem + q.o_flips);
    // int8 fields are held as exact fp32, as the steps on Wf expect; int16 fields are int32
    if (!cu_ok(da::launch_init_state(q.integer, diag, q.N, R, h, sh.npad(), st, q.dtype == DA_INT8), q, "init"))
        return false;
    if (!cu_ok(da::launch_zero(xs, (size_t)2 * R * q.xs_stride * 4, st), q, "init")) return false;
    if (!cu_ok(da::launch_zero(sc, (size_t)R * sizeof(da::ReplicaScalars), st), q, "init")) return false;
    launches += 3;
    da::StepParams p;
    p.W = q.dtype == DA_INT8 ? Wf : W;
    p.Wc = Wc;
    p.diag = diag;
    p.N = q.N;
    p.ldw = q.inst.ldw;
    p.R = R;
    p.npad = sh.npad();
    p.nw = sh.nwords();
    p.h = h;
    p.x = xs;
    p.bestx = xs + (size_t)R * q.xs_stride;
    p.sc = sc;
    p.beta = reinterpret_cast<const float*>(q.dmem + q.o_beta);
    p.inc = q.job.offset_inc;
    p.stop = s->stop + q.slot;
    da::set_seed(p, q.job.seed);
    const long long T = q.job.steps, P = q.integer ? 0 : q.job.recompute_every;
    const int wstep = q.dtype == DA_INT8 ? da::kWInt8AsF32 : q.dtype;
    if (q.resident && T > 0) {
        da::BatchItemDev& d = q.item;
        d.W = p.W;
        d.Wc = nullptr;   // the resident kernel reads W in the plain order
        d.diag = diag;
        d.beta = p.beta;
        d.xs = xs;
        d.sc = sc;
        d.trace = nullptr;
        d.T = T;
        d.recompute_every = P;
        d.unit0 = 0;
        d.seed = q.job.seed;
        d.N = q.N;
        d.ldw = q.inst.ldw;
        d.S = q.inst.S;
        d.R = R;
        d.inc = q.job.offset_inc;
        d.exact_shift = q.inst.exact_shift ? 1 : 0;
        d.stop = s->stop + q.slot;
        auto* item_dev = reinterpret_cast<da::BatchItemDev*>(q.dmem + q.o_item);
        auto* head_dev = reinterpret_cast<unsigned long long*>(q.dmem + q.o_item + sizeof(da::BatchItemDev));
        if (!cu_ok(cudaMemcpyAsync(item_dev, &d, sizeof(d), cudaMemcpyHostToDevice, st), q, "descriptor")) return false;
        if (!cu_ok(da::launch_resident_anneal(wstep, sh.V, item_dev, head_dev, R, st), q, "resident anneal"))
            return false;
        launches += 2;
    }
    for (long long t0 = 0; t0 < T && !q.resident; t0 = p.t1) {
        p.t0 = t0;
        p.t1 = std::min(T, t0 + (1ll << 14));
        if (P > 0) p.t1 = std::min(p.t1, (t0 / P + 1) * P);
        if (!cu_ok(da::launch_step(wstep, sh, p, false, st), q, "step")) return false;
        ++launches;
        if (P > 0 && p.t1 % P == 0) {
            if (!cu_ok(da::launch_recompute_tc(false, q.tc, diag, q.N, q.inst.S, xs, sh.nwords(), R, h, sh.npad(),
                                               reinterpret_cast<long long*>(sc), (int)(sizeof(da::ReplicaScalars) / 8),
                                               st, part),
                       q, "recompute"))
                return false;
            launches += 2;
        }
    }
    if (!cu_ok(da::launch_best_fixup(R, sc, q.integer, xs, xs + (size_t)R * q.xs_stride, q.xs_stride, st), q,
               "fixup"))
        return false;
    const bool ev_ok =
        q.integer ? cu_ok(da::launch_recompute_w(q.dtype, W, diag, q.N, q.inst.ldw, q.inst.S, xs, sh.nwords(), 2 * R,
                                                 nullptr, sh.npad(), eex, 1, st, part),
                          q, "evaluate")
                  : cu_ok(da::launch_recompute_tc(false, q.tc, diag, q.N, q.inst.S, xs, sh.nwords(), 2 * R, nullptr,
                                                  sh.npad(), eex, 1, st, part),
                          q, "evaluate");
    if (!ev_ok) return false;
    da::prefer_shared<da::serve_finalize_kernel>();
    da::serve_finalize_kernel<<<(R + 127) / 128, 128, 0, st>>>(q.integer, R, sc, eex, E, flips);
    if (!cu_ok(cudaGetLastError(), q, "finalize")) return false;
    launches += 4;
    return cu_ok(cudaEventRecord(q.done_ev, st), q, "event");
}

// Return a request's stream and event to the server and free its memory
// (stream-ordered: the next request on the stream comes after the free).
void release(da_server* s, Req& q)
{
    if (q.stream) {
        if (q.dmem) da::pool_free_async(q.dmem, q.stream);
        s->streams.push_back(q.stream);
    }
    if (q.done_ev) s->events.push_back(q.done_ev);
    if (q.built_ev) s->events.push_back(q.built_ev);
    q.dmem = nullptr;
    q.stream = nullptr;
    q.done_ev = nullptr;
    q.built_ev = nullptr;
}

// The budget a request returns when it leaves the GPU (its buffers, and the
// copy of Q if its release was not seen yet), and its slot and warps.
void uncharge(da_server* s, Req& q)
{
    s->used -= (int64_t)q.bytes + (q.qcopy_held ? (int64_t)q.qcopy : 0);
    q.qcopy_held = false;
    s->warps -= (long long)q.job.replicas * q.shape.G;
    s->free_slots.push_back(q.slot);
}

// Copy a finished request's results to the host; false on a CUDA error
// (recorded in q.err and q.msg).
bool finish(Req& q)
{
    const int R = q.job.replicas;
    q.E.resize((size_t)3 * R);
    q.xs.resize((size_t)2 * R * q.xs_stride);
    q.flips.resize((size_t)R);
    cudaStream_t st = q.stream;
    bool ok = cu_ok(cudaMemcpyAsync(q.E.data(), q.dmem + q.o_E, q.E.size() * 8, cudaMemcpyDeviceToHost, st), q,
                    "results");
    ok = ok && cu_ok(cudaMemcpyAsync(q.xs.data(), q.dmem + q.o_xs, q.xs.size() * 4, cudaMemcpyDeviceToHost, st), q,
                     "results");
    ok = ok && cu_ok(cudaMemcpyAsync(q.flips.data(), q.dmem + q.o_flips, q.flips.size() * 8, cudaMemcpyDeviceToHost,
                                     st),
                     q, "results");
    q.tc_err = 0;
    if (!q.integer)
        ok = ok && cu_ok(cudaMemcpyAsync(&q.tc_err, q.tc.err, sizeof(int), cudaMemcpyDeviceToHost, st), q, "results");
    ok = ok && cu_ok(cudaStreamSynchronize(st), q, "results");
    if (ok && q.tc_err) {
        q.err = DA_ETIMEOUT;
        q.msg = "a bounded wait inside the tensor-core recompute gave up; the results are invalid";
        return false;
    }
    return ok;
}

void worker_loop(da_server* s)
{
    cudaSetDevice(s->dev);
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        // admission, in arrival order, while memory and slots allow
        while (!s->pending.empty()) {
            std::shared_ptr<Req> q = s->pending.front();
            if (s->free_slots.empty() || s->used + (int64_t)peak_bytes(*q) > s->budget) break;
            const long long qw = (long long)q->job.replicas * q->shape.G;
            if (!s->active.empty() && s->warps + qw > s->warp_cap) break;
            s->warps += qw;
            s->pending.pop_front();
            q->slot = s->free_slots.back();
            s->free_slots.pop_back();
            s->used += (int64_t)peak_bytes(*q);
            q->qcopy_held = true;
            q->state = ReqState::Running;
            s->stop[q->slot] = 0;   // no step launch of this request is queued yet
            s->active.push_back(q);
            lk.unlock();
            long long launches = 0;
            const bool ok = admit(s, *q, launches);
            lk.lock();
            s->kernel_launches += launches;
            if (!ok) {
                if (q->stream) {            // what was queued, before the memory goes (without the lock)
                    lk.unlock();
                    cudaStreamSynchronize(q->stream);
                    lk.lock();
                }
                release(s, *q);
                q->state = ReqState::Failed;
                q->t_done = Clock::now();
                s->active.erase(std::find(s->active.begin(), s->active.end(), q));
                uncharge(s, *q);
                s->cv_done.notify_all();
            }
        }
        // the copy of Q of a request whose instance is built goes back to the budget
        for (auto& q : s->active) {
            if (q->qcopy_held && q->built_ev && cudaEventQuery(q->built_ev) == cudaSuccess) {
                s->used -= (int64_t)q->qcopy;
                q->qcopy_held = false;
            }
        }
        std::vector<std::shared_ptr<Req>> act = s->active;
        const bool idle = s->pending.empty() && s->active.empty();
        if (idle && s->quit) break;
        lk.unlock();
        // completions: results are copied without the lock; the state that
        // da_poll reads changes under it, after everything else it reads
        std::vector<std::pair<std::shared_ptr<Req>, bool>> fin;
        for (auto& q : act) {
            const cudaError_t e = cudaEventQuery(q->done_ev);
            if (e == cudaErrorNotReady) continue;
            bool ok = false;
            if (e != cudaSuccess) {
                cudaGetLastError();
                q->err = DA_ECUDA;
                q->msg = std::string("request: ") + cudaGetErrorString(e);
            } else if (q->cancelled) {
                q->err = DA_ECANCELED;
                q->msg = "cancelled";
            } else {
                ok = finish(*q);
            }
            q->t_done = Clock::now();
            fin.emplace_back(q, ok);
        }
        lk.lock();
        for (auto& [q, ok] : fin) {
            q->state = ok ? ReqState::Done : ReqState::Failed;
            release(s, *q);
            s->active.erase(std::find(s->active.begin(), s->active.end(), q));
            uncharge(s, *q);
            s->completed++;
        }
        if (!fin.empty()) s->cv_done.notify_all();
        if (fin.empty()) s->cv_work.wait_for(lk, std::chrono::microseconds(100));
    }
}

void destroy_resources(da_server* s)
{
    for (cudaStream_t st : s->streams) {
        cudaStreamSynchronize(st);
        cudaStreamDestroy(st);
    }
    for (cudaEvent_t ev : s->events) cudaEventDestroy(ev);
    s->streams.clear();
    s->events.clear();
    if (s->pool) cudaMemPoolDestroy(s->pool);
    s->pool = nullptr;
    if (s->stop) cudaFreeHost(s->stop);
    s->stop = nullptr;
}

}  // namespace

extern "C" {

da_status da_server_create(int64_t hbm_budget_bytes, int32_t max_requests, da_server** out)
{
    da::set_last_error("");
    if (!out) return sfail(DA_EINVAL, "out is null");
    *out = nullptr;
    if (hbm_budget_bytes <= 0 || max_requests < 1 || max_requests > 65536)
        return sfail(DA_EINVAL, "need a positive budget and 1 <= max_requests <= 65536");
    auto s = std::make_unique<da_server>();
    if (cudaGetDevice(&s->dev) != cudaSuccess) {
        cudaGetLastError();
        return sfail(DA_ECUDA, "no CUDA device");
    }
    s->budget = hbm_budget_bytes;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s->dev) != cudaSuccess) {
        cudaGetLastError();
        return sfail(DA_ECUDA, "no CUDA device");
    }
    s->warp_cap = (long long)kWarpsPerSm * sms;
    s->max_slots = max_requests;
    for (int i = max_requests - 1; i >= 0; --i) s->free_slots.push_back(i);
    cudaError_t e = da::prepare_step(da::kWFp32);
    if (e == cudaSuccess) e = da::prepare_step(da::kWInt8AsF32);
    if (e == cudaSuccess) e = da::prepare_step(da::kWInt16);
    if (e == cudaSuccess) e = da::prepare_field_kernels();
    if (e == cudaSuccess) e = da::prepare_tc_kernels();
    if (e == cudaSuccess) e = da::prepare_resident_kernels();
    if (e == cudaSuccess) {
        da::prefer_shared<da::serve_finalize_kernel>();
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return sfail(DA_ECUDA, std::string("kernels: ") + cudaGetErrorString(e));
    if ((e = cudaHostAlloc(reinterpret_cast<void**>(&s->stop), (size_t)max_requests * sizeof(int),
                           cudaHostAllocMapped)) != cudaSuccess) {
        cudaGetLastError();
        s->stop = nullptr;
        destroy_resources(s.get());
        return sfail(DA_ENOMEM, std::string("stop flags: ") + cudaGetErrorString(e));
    }
    std::memset(s->stop, 0, (size_t)max_requests * sizeof(int));
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = s->dev;
    e = cudaMemPoolCreate(&s->pool, &props);
    uint64_t keep = ~0ull;
    if (e == cudaSuccess) e = cudaMemPoolSetAttribute(s->pool, cudaMemPoolAttrReleaseThreshold, &keep);
    if (e != cudaSuccess) {
        cudaGetLastError();
        destroy_resources(s.get());
        return sfail(e == cudaErrorMemoryAllocation ? DA_ENOMEM : DA_ECUDA,
                     std::string("memory pool: ") + cudaGetErrorString(e));
    }
    da_server* raw = s.release();
    raw->worker = std::thread(worker_loop, raw);
    *out = raw;
    return DA_OK;
}

da_status da_submit(da_server* s, const da_job* job, da_req** out)
{
    da::set_last_error("");
    if (!s || !job || !out) return sfail(DA_EINVAL, "null argument");
    *out = nullptr;
    if (!job->Q || job->N < 1 || job->N > 8192) return sfail(DA_EINVAL, "need Q and 1 <= N <= 8192");
    if (job->dtype != DA_INT8 && job->dtype != DA_FP32 && job->dtype != DA_INT16)
        return sfail(DA_EINVAL, "unknown dtype");
    if (job->steps < 0 || job->steps >= (1ll << 32) || (job->steps > 0 && !job->beta))
        return sfail(DA_EINVAL, "bad schedule");
    if (job->steps > 0 && !da::schedule_ok(job->beta, job->steps))
        return sfail(DA_EINVAL, "beta must be finite and >= 0");
    if (job->replicas < 1 || job->replicas > 65536) return sfail(DA_EINVAL, "need 1 <= replicas <= 65536");
    if (!(job->offset_inc >= 0.f) || !std::isfinite(job->offset_inc) || job->recompute_every < 0)
        return sfail(DA_EINVAL, "bad offset or recompute period");
    auto q = std::make_shared<Req>();
    q->job = *job;
    q->N = (int)job->N;
    q->dtype = (int)job->dtype;
    q->integer = job->dtype != DA_FP32;
    std::string why;
    if (!da::build_instance(job->Q, q->N, job->dtype, q->inst, why)) return sfail(DA_EINVAL, why);
    // a context's launch shape: measured on a mix of concurrent requests it
    // gives more trials per second than the fewest warps per replica
    q->shape = da::default_shape(q->N, job->replicas);
    q->resident = q->N <= s->resident_max_n && q->shape.G == 1;
    plan_request(*q);
    if ((int64_t)peak_bytes(*q) > s->budget)
        return sfail(DA_EBUDGET, "request needs " + std::to_string(peak_bytes(*q)) +
                                     " bytes (with the transient copy of Q), over the budget of " +
                                     std::to_string(s->budget));
    q->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->quit) return sfail(DA_EBUSY, "the server is shutting down");
        s->pending.push_back(q);
    }
    s->cv_work.notify_all();
    *out = new da_req{q, s};
    return DA_OK;
}

da_status da_poll(da_req* req, int32_t timeout_us, da_result* out)
{
    da::set_last_error("");
    if (!req || !req->r) return sfail(DA_EINVAL, "null request");
    da_server* s = req->srv;
    Req& q = *req->r;
    {
        std::unique_lock<std::mutex> lk(s->mu);
        auto done = [&] { return q.state == ReqState::Done || q.state == ReqState::Failed; };
        if (timeout_us > 0) s->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), done);
        if (!done()) return timeout_us > 0 ? sfail(DA_ETIMEOUT, "not finished") : DA_ENOTREADY;
    }
    if (q.state == ReqState::Failed) return sfail(q.err == DA_OK ? DA_ECUDA : q.err, q.msg);
    if (!out) return DA_OK;
    const int R = q.job.replicas;
    const size_t words = (size_t)(q.N + 31) / 32;
    for (int r = 0; r < R; ++r) {
        if (out->final_E) out->final_E[r] = q.E[r];
        if (out->best_E) out->best_E[r] = q.E[R + r];
        if (out->max_drift) out->max_drift[r] = q.E[2 * R + r];
        if (out->flips) out->flips[r] = q.flips[r];
        for (size_t w = 0; w < words; ++w) {
            if (out->final_x) out->final_x[r * words + w] = q.xs[(size_t)r * q.xs_stride + w];
            if (out->best_x) out->best_x[r * words + w] = q.xs[((size_t)R + r) * q.xs_stride + w];
        }
    }
    out->elapsed_s = std::chrono::duration<double>(q.t_done - q.t_submit).count();
    return DA_OK;
}

void da_req_free(da_req* req) { delete req; }

da_status da_cancel(da_req* req)
{
    da::set_last_error("");
    if (!req || !req->r) return sfail(DA_EINVAL, "null request");
    da_server* s = req->srv;
    std::shared_ptr<Req> q = req->r;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (q->state == ReqState::Queued) {
            auto it = std::find(s->pending.begin(), s->pending.end(), q);
            if (it != s->pending.end()) s->pending.erase(it);
            q->state = ReqState::Failed;
            q->err = DA_ECANCELED;
            q->msg = "cancelled";
            q->t_done = Clock::now();
        } else if (q->state == ReqState::Running) {
            q->cancelled = true;
            // step launches that start from now on return at once; what is
            // already running finishes its chunk
            reinterpret_cast<volatile int*>(s->stop)[q->slot] = 1;
        }
    }
    s->cv_done.notify_all();
    s->cv_work.notify_all();
    return DA_OK;
}

da_status da_server_resident(da_server* s, int32_t max_n)
{
    if (!s || max_n < 0 || max_n > 1024) return sfail(DA_EINVAL, "need a server and 0 <= max_n <= 1024");
    s->resident_max_n = max_n;
    return DA_OK;
}

da_status da_server_stats(da_server* s, int64_t* completed, int64_t* kernel_launches, int64_t* bytes_in_use)
{
    if (!s) return sfail(DA_EINVAL, "null server");
    std::lock_guard<std::mutex> lk(s->mu);
    if (completed) *completed = s->completed;
    if (kernel_launches) *kernel_launches = s->kernel_launches;
    if (bytes_in_use) *bytes_in_use = s->used;
    return DA_OK;
}

void da_server_destroy(da_server* s)
{
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->quit = true;
    }
    s->cv_work.notify_all();
    if (s->worker.joinable()) s->worker.join();   // drains every submitted request
    destroy_resources(s);
    delete s;
}

}  // extern "C"
