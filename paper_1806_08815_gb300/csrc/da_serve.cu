// da_serve.cu -- the request loop: da_server_create / da_submit / da_poll.
//
// Admission: a request (one QUBO, its schedule and replica count) waits in a
// FIFO until its device memory fits the server's HBM budget and a request slot
// is free; then its instance is built and uploaded (stream-ordered
// allocations, so nothing synchronises against the running kernel).
//   N <= 1024: its replicas become units of the persistent kernel
//              (da_serve_kernel.cuh), appended to the ring while the kernel
//              runs; replica state never leaves the warp's registers.
//   N >  1024: its anneal runs as chunked multi-warp step launches on a stream
//              of its own, concurrently with the persistent kernel (which is
//              sized to leave room for them).
// A worker thread admits, launches, polls completion flags, copies results
// and frees memory; da_poll waits on a request with a timeout.
#include <algorithm>
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
#include "da_serve_kernel.cuh"

namespace da {

__global__ void __launch_bounds__(128) serve_kernel(const __grid_constant__ ServeParams sp)
{
    const int lane = threadIdx.x & 31;
    int idle = 0;
    for (;;) {
        unsigned long long u = ~0ull;
        int slot = 0, replica = 0;
        if (lane == 0) {
            cuda::atomic_ref<unsigned long long, cuda::thread_scope_system> tail(
                *const_cast<unsigned long long*>(sp.tail));
            for (;;) {
                if (*sp.stop) break;
                const unsigned long long t = tail.load(cuda::memory_order_acquire);
                const unsigned long long h = *reinterpret_cast<volatile unsigned long long*>(sp.head);
                if (h < t) {
                    if (atomicCAS(sp.head, h, h + 1) == h) {
                        u = h;
                        const volatile ServeUnit* e = sp.ring + (h % sp.cap);
                        slot = e->slot;
                        replica = e->replica;
                        break;
                    }
                    continue;
                }
                if (++idle > sp.idle_polls) break;
                __nanosleep(2000);
            }
        }
        u = __shfl_sync(0xffffffffu, u, 0);
        if (u == ~0ull) return;
        slot = __shfl_sync(0xffffffffu, slot, 0);
        replica = __shfl_sync(0xffffffffu, replica, 0);
        idle = 0;
        ServeDesc d;
        {
            // through L2: the slot's descriptor is rewritten between requests
            static_assert(sizeof(ServeDesc) % 16 == 0, "descriptor size");
            const int4* src = reinterpret_cast<const int4*>(sp.descs + slot);
            int4* dst = reinterpret_cast<int4*>(&d);
#pragma unroll
            for (int i = 0; i < (int)(sizeof(ServeDesc) / 16); ++i) dst[i] = __ldcg(src + i);
        }
        const int vcls = d.V == 4 ? 0 : d.V == 8 ? 1 : d.V == 16 ? 2 : 3;
        switch (d.int8 * 4 + vcls) {
        case 0: serve_detail::run_unit<float, 4>(d, replica); break;
        case 1: serve_detail::run_unit<float, 8>(d, replica); break;
        case 2: serve_detail::run_unit<float, 16>(d, replica); break;
        case 3: serve_detail::run_unit<float, 32>(d, replica); break;
        case 4: serve_detail::run_unit<int8_t, 4>(d, replica); break;
        case 5: serve_detail::run_unit<int8_t, 8>(d, replica); break;
        case 6: serve_detail::run_unit<int8_t, 16>(d, replica); break;
        default: serve_detail::run_unit<int8_t, 32>(d, replica); break;
        }
        if (lane == 0) {
            __threadfence();
            const unsigned int prev = atomicAdd(d.done, 1u);
            if (prev + 1 == (unsigned int)d.R) {
                __threadfence_system();
                *d.flag = 1u;
            }
        }
        __syncwarp();
    }
}

// Finalises a big (chunked) request: exact energies into E[3R], flips.
__global__ void serve_big_finalize(bool int8, int R, const ReplicaScalars* sc, const long long* eex, double* E,
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
constexpr unsigned long long kRingCap = 1ull << 20;
constexpr int kIdlePolls = 1 << 21;      // seconds of empty polling before a warp leaves on its own
// the host stops the kernel after this long without a request of its path in flight
constexpr auto kIdleStop = std::chrono::milliseconds(20);

size_t al256(size_t v) { return (v + 255) / 256 * 256; }

enum class ReqState { Queued, Running, Done, Failed };

struct Req {
    da_job job;
    int N = 0;
    bool int8 = false;
    bool big = false;                 // N > 1024: chunked path on its own stream
    da::StepShape shape;              // big path launch shape; small path: V in shape.V
    da::HostInstance inst;            // checked at submit (ldw, S); W and diag built on the device at admission
    size_t bytes = 0;                 // device bytes charged to the budget
    int slot = -1;
    ReqState state = ReqState::Queued;
    da_status err = DA_OK;
    std::string msg;
    char* dmem = nullptr;
    // offsets into dmem
    size_t o_W = 0, o_diag = 0, o_beta = 0, o_xs = 0, o_E = 0, o_flips = 0;
    size_t o_h = 0, o_sc = 0, o_part = 0, o_eex = 0;     // big path only
    int xs_stride = 0;                // words per replica in xs
    // results on the host
    std::vector<double> E;            // [3R]
    std::vector<uint32_t> xs;         // [2R][xs_stride]
    std::vector<long long> flips;     // [R]
    Clock::time_point t_submit, t_start, t_done;
    cudaStream_t stream = nullptr;    // big path
    cudaEvent_t done_ev = nullptr;    // big path
};

}  // namespace

struct da_req {
    std::shared_ptr<Req> r;
    da_server* srv;
};

struct da_server {
    int dev = 0, sms = 0;
    int64_t budget = 0, used = 0;
    int max_slots = 0;
    std::vector<int> free_slots;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<std::shared_ptr<Req>> pending;
    std::vector<std::shared_ptr<Req>> active;
    std::thread worker;
    bool quit = false;
    // device and host-mapped state of the persistent kernel
    da::ServeDesc* descs = nullptr;        // device [max_slots]
    unsigned int* done = nullptr;          // device [max_slots]
    unsigned long long* head = nullptr;    // device
    da::ServeUnit* ring_h = nullptr;       // mapped
    da::ServeUnit* ring_d = nullptr;
    unsigned long long* tail_h = nullptr;  // mapped
    unsigned long long* tail_d = nullptr;
    unsigned int* flags_h = nullptr;       // mapped [max_slots]
    unsigned int* flags_d = nullptr;
    int* stop_h = nullptr;                 // mapped
    int* stop_d = nullptr;
    unsigned long long tail = 0;           // units pushed
    unsigned long long units_done = 0;     // units of completed requests
    unsigned long long head_seen = 0;      // head read after the kernel last ended
    cudaStream_t s_kernel = nullptr, s_copy = nullptr;
    // requests' device memory: a pool of the server's own that keeps what it
    // has reserved (a pool that trims at every synchronisation unmaps memory,
    // which waits for the running kernels: admission would stall behind the
    // persistent kernel and behind every running anneal)
    cudaMemPool_t pool = nullptr;
    cudaEvent_t k_done = nullptr;
    bool k_running = false;
    bool k_stopping = false;               // stop raised because the kernel's path went idle
    std::chrono::steady_clock::time_point last_busy{};
    int kernel_blocks = 0;
    // statistics
    long long kernel_launches = 0, completed = 0;
};

namespace {

da_status sfail(da_status s, const std::string& m)
{
    da::set_last_error(m);
    return s;
}

// Device bytes of a request and its buffer offsets.
void plan_request(Req& q)
{
    const int R = q.job.replicas;
    const size_t esz = q.int8 ? 1 : 4;
    size_t o = 0;
    auto take = [&](size_t b) { size_t at = o; o += al256(b); return at; };
    q.o_W = take(da::instance_W_bytes(q.N, q.int8 ? DA_INT8 : DA_FP32));
    q.o_diag = take((size_t)q.N * 4);
    q.o_beta = take((size_t)q.job.steps * 4);
    if (!q.big) {
        q.xs_stride = q.shape.V;   // words per replica = 32V / 32
        q.o_xs = take((size_t)2 * R * q.xs_stride * 4);
    } else {
        q.xs_stride = q.shape.nwords();
        q.o_h = take((size_t)R * q.shape.npad() * 4);
        q.o_xs = take((size_t)2 * R * q.xs_stride * 4);
        q.o_sc = take((size_t)R * sizeof(da::ReplicaScalars));
        q.o_part = take((size_t)16 * ((std::max(q.shape.npad(), q.N) + 63) / 64) * 2 * R);
        q.o_eex = take((size_t)2 * R * 8);
    }
    q.o_E = take((size_t)3 * R * 8);
    q.o_flips = take((size_t)R * 8);
    (void)esz;
    q.bytes = o;
}

}  // namespace

namespace {

bool cu_ok(cudaError_t e, Req& q, const char* what)
{
    if (e == cudaSuccess) return true;
    cudaGetLastError();
    q.err = DA_ECUDA;
    q.msg = std::string(what) + ": " + cudaGetErrorString(e);
    return false;
}

// Upload an admitted request and start its work.  Runs on the worker thread.
bool admit(da_server* s, Req& q)
{
    if (cudaMallocFromPoolAsync(reinterpret_cast<void**>(&q.dmem), q.bytes, s->pool, s->s_copy) != cudaSuccess) {
        cudaGetLastError();
        q.dmem = nullptr;
        q.err = DA_ENOMEM;
        q.msg = "device allocation of " + std::to_string(q.bytes) + " bytes";
        return false;
    }
    const int R = q.job.replicas;
    // W and diag from a transient device copy of Q (the caller keeps Q valid)
    {
        void* qd = nullptr;
        const size_t qbytes = (size_t)q.N * q.N * 4;
        if (cudaMallocFromPoolAsync(&qd, qbytes, s->pool, s->s_copy) != cudaSuccess) {
            cudaGetLastError();
            q.err = DA_ENOMEM;
            q.msg = "device allocation of " + std::to_string(qbytes) + " bytes (copy of Q)";
            return false;
        }
        bool ok = cu_ok(cudaMemcpyAsync(qd, q.job.Q, qbytes, cudaMemcpyHostToDevice, s->s_copy), q, "upload Q");
        ok = ok && cu_ok(da::launch_expand_instance(qd, q.N, q.inst.ldw, q.int8 ? DA_INT8 : DA_FP32, q.dmem + q.o_W,
                                                    nullptr, q.dmem + q.o_diag, s->s_copy),
                         q, "build instance");
        cudaFreeAsync(qd, s->s_copy);
        if (!ok) return false;
    }
    if (q.job.steps > 0 &&
        !cu_ok(cudaMemcpyAsync(q.dmem + q.o_beta, q.job.beta, (size_t)q.job.steps * 4, cudaMemcpyHostToDevice, s->s_copy),
               q, "upload beta"))
        return false;
    const void* W = q.dmem + q.o_W;
    const void* diag = q.dmem + q.o_diag;
    const float* beta = reinterpret_cast<const float*>(q.dmem + q.o_beta);
    uint32_t* xs = reinterpret_cast<uint32_t*>(q.dmem + q.o_xs);
    double* E = reinterpret_cast<double*>(q.dmem + q.o_E);
    long long* flips = reinterpret_cast<long long*>(q.dmem + q.o_flips);
    if (!q.big) {
        da::ServeDesc d{};
        d.W = W;
        d.diag = diag;
        d.beta = beta;
        d.xs = xs;
        d.E = E;
        d.flips = flips;
        d.done = s->done + q.slot;
        d.flag = s->flags_d + q.slot;
        d.T = q.job.steps;
        d.P = q.int8 ? 0 : q.job.recompute_every;
        d.seed = q.job.seed;
        d.N = q.N;
        d.ldw = q.inst.ldw;
        d.S = q.inst.S;
        d.R = R;
        d.V = q.shape.V;
        d.int8 = q.int8 ? 1 : 0;
        d.inc = q.job.offset_inc;
        if (!cu_ok(cudaMemcpyAsync(s->descs + q.slot, &d, sizeof(d), cudaMemcpyHostToDevice, s->s_copy), q, "descriptor"))
            return false;
        if (!cu_ok(cudaMemsetAsync(s->done + q.slot, 0, sizeof(unsigned int), s->s_copy), q, "counter")) return false;
        reinterpret_cast<volatile unsigned int*>(s->flags_h)[q.slot] = 0u;
        if (!cu_ok(cudaStreamSynchronize(s->s_copy), q, "upload")) return false;
        for (int i = 0; i < R; ++i) s->ring_h[(s->tail + i) % kRingCap] = da::ServeUnit{q.slot, i};
        s->tail += (unsigned long long)R;
        __atomic_store_n(s->tail_h, s->tail, __ATOMIC_RELEASE);
    } else {
        if (!cu_ok(cudaStreamCreateWithFlags(&q.stream, cudaStreamNonBlocking), q, "stream")) return false;
        if (!cu_ok(cudaEventCreateWithFlags(&q.done_ev, cudaEventDisableTiming), q, "event")) return false;
        if (!cu_ok(cudaStreamSynchronize(s->s_copy), q, "upload")) return false;
        const da::StepShape sh = q.shape;
        void* h = q.dmem + q.o_h;
        da::ReplicaScalars* sc = reinterpret_cast<da::ReplicaScalars*>(q.dmem + q.o_sc);
        long long* part = reinterpret_cast<long long*>(q.dmem + q.o_part);
        long long* eex = reinterpret_cast<long long*>(q.dmem + q.o_eex);
        cudaStream_t st = q.stream;
        if (!cu_ok(da::launch_init_state(q.int8, diag, q.N, R, h, sh.npad(), st), q, "init")) return false;
        if (!cu_ok(cudaMemsetAsync(xs, 0, (size_t)2 * R * q.xs_stride * 4, st), q, "init")) return false;
        if (!cu_ok(cudaMemsetAsync(sc, 0, (size_t)R * sizeof(da::ReplicaScalars), st), q, "init")) return false;
        da::StepParams p;
        p.W = W;
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
        p.beta = beta;
        p.inc = q.job.offset_inc;
        da::set_seed(p, q.job.seed);
        const long long T = q.job.steps, P = q.int8 ? 0 : q.job.recompute_every;
        for (long long t0 = 0; t0 < T; t0 = p.t1) {
            p.t0 = t0;
            p.t1 = std::min(T, t0 + (1ll << 14));
            if (P > 0) p.t1 = std::min(p.t1, (t0 / P + 1) * P);
            if (!cu_ok(da::launch_step(q.int8 ? da::kWInt8 : da::kWFp32, sh, p, false, st), q, "step")) return false;
            if (P > 0 && p.t1 % P == 0 &&
                !cu_ok(da::launch_recompute(false, W, diag, q.N, q.inst.ldw, q.inst.S, xs, sh.nwords(), R, h, sh.npad(),
                                            reinterpret_cast<long long*>(sc), (int)(sizeof(da::ReplicaScalars) / 8),
                                            st, part),
                       q, "recompute"))
                return false;
        }
        if (!cu_ok(da::launch_best_fixup(R, sc, q.int8, xs, xs + (size_t)R * q.xs_stride, q.xs_stride, st), q, "fixup"))
            return false;
        if (!cu_ok(da::launch_recompute(q.int8, W, diag, q.N, q.inst.ldw, q.inst.S, xs, sh.nwords(), 2 * R, nullptr,
                                        sh.npad(), eex, 1, st, part),
                   q, "evaluate"))
            return false;
        da::serve_big_finalize<<<(R + 127) / 128, 128, 0, st>>>(q.int8, R, sc, eex, E, flips);
        if (!cu_ok(cudaGetLastError(), q, "finalize")) return false;
        if (!cu_ok(cudaEventRecord(q.done_ev, st), q, "event")) return false;
    }
    q.t_start = Clock::now();
    return true;
}

// Copy a finished request's results to the host and release its memory.
void finish(da_server* s, Req& q)
{
    const int R = q.job.replicas;
    q.E.resize((size_t)3 * R);
    q.xs.resize((size_t)2 * R * q.xs_stride);
    q.flips.resize((size_t)R);
    bool ok = cu_ok(cudaMemcpyAsync(q.E.data(), q.dmem + q.o_E, q.E.size() * 8, cudaMemcpyDeviceToHost, s->s_copy), q,
                    "results");
    ok = ok && cu_ok(cudaMemcpyAsync(q.xs.data(), q.dmem + q.o_xs, q.xs.size() * 4, cudaMemcpyDeviceToHost, s->s_copy),
                     q, "results");
    ok = ok && cu_ok(cudaMemcpyAsync(q.flips.data(), q.dmem + q.o_flips, q.flips.size() * 8, cudaMemcpyDeviceToHost,
                                     s->s_copy),
                     q, "results");
    ok = ok && cu_ok(cudaStreamSynchronize(s->s_copy), q, "results");
    if (q.dmem) cudaFreeAsync(q.dmem, s->s_copy);
    q.dmem = nullptr;
    if (q.done_ev) cudaEventDestroy(q.done_ev);
    if (q.stream) cudaStreamDestroy(q.stream);
    q.done_ev = nullptr;
    q.stream = nullptr;
    q.t_done = Clock::now();
    q.state = ok ? ReqState::Done : ReqState::Failed;
}

void launch_kernel(da_server* s)
{
    da::ServeParams sp;
    sp.descs = s->descs;
    sp.ring = s->ring_d;
    sp.tail = s->tail_d;
    sp.head = s->head;
    sp.stop = s->stop_d;
    sp.cap = kRingCap;
    sp.idle_polls = kIdlePolls;
    da::serve_kernel<<<s->kernel_blocks, 128, 0, s->s_kernel>>>(sp);
    if (cudaGetLastError() != cudaSuccess) return;
    cudaEventRecord(s->k_done, s->s_kernel);
    s->k_running = true;
    s->kernel_launches++;
}

void worker_loop(da_server* s)
{
    cudaSetDevice(s->dev);
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        // admission, in arrival order, while memory and slots allow
        while (!s->pending.empty()) {
            std::shared_ptr<Req> q = s->pending.front();
            if (s->free_slots.empty() || s->used + (int64_t)q->bytes > s->budget) break;
            if (!q->big && s->tail + (unsigned long long)q->job.replicas - s->units_done > kRingCap) break;
            s->pending.pop_front();
            q->slot = s->free_slots.back();
            s->free_slots.pop_back();
            s->used += (int64_t)q->bytes;
            q->state = ReqState::Running;
            s->active.push_back(q);
            lk.unlock();
            const bool ok = admit(s, *q);
            lk.lock();
            if (!ok) {
                if (q->dmem) cudaFreeAsync(q->dmem, s->s_copy);
                q->dmem = nullptr;
                q->state = ReqState::Failed;
                q->t_done = Clock::now();
                s->active.erase(std::find(s->active.begin(), s->active.end(), q));
                s->used -= (int64_t)q->bytes;
                s->free_slots.push_back(q->slot);
                s->cv_done.notify_all();
            }
        }
        std::vector<std::shared_ptr<Req>> act = s->active;
        const bool idle = s->pending.empty() && s->active.empty();
        if (idle && s->quit) break;
        lk.unlock();
        // the persistent kernel: relaunch while units are waiting
        if (s->k_running && cudaEventQuery(s->k_done) == cudaSuccess) {
            s->k_running = false;
            cudaMemcpyAsync(&s->head_seen, s->head, 8, cudaMemcpyDeviceToHost, s->s_copy);
            cudaStreamSynchronize(s->s_copy);
            if (s->k_stopping) {
                __atomic_store_n(s->stop_h, 0, __ATOMIC_RELEASE);
                s->k_stopping = false;
            }
        } else {
            cudaGetLastError();   // cudaErrorNotReady
        }
        // units pushed whose request has not completed: the kernel has work
        const auto now = Clock::now();
        if (s->tail > s->units_done) s->last_busy = now;
        if (s->k_running && !s->k_stopping && s->tail == s->units_done && now - s->last_busy > kIdleStop) {
            __atomic_store_n(s->stop_h, 1, __ATOMIC_RELEASE);
            s->k_stopping = true;
        }
        if (!s->k_running && s->tail > s->head_seen) launch_kernel(s);
        // completions
        std::vector<std::shared_ptr<Req>> fin;
        for (auto& q : act) {
            bool ready;
            if (q->big) {
                const cudaError_t e = cudaEventQuery(q->done_ev);
                if (e != cudaSuccess && e != cudaErrorNotReady) cudaGetLastError();
                ready = e != cudaErrorNotReady;
            } else {
                ready = reinterpret_cast<volatile unsigned int*>(s->flags_h)[q->slot] != 0u;
            }
            if (ready) {
                finish(s, *q);
                fin.push_back(q);
            }
        }
        lk.lock();
        for (auto& q : fin) {
            s->active.erase(std::find(s->active.begin(), s->active.end(), q));
            s->used -= (int64_t)q->bytes;
            s->free_slots.push_back(q->slot);
            if (!q->big) s->units_done += (unsigned long long)q->job.replicas;
            s->completed++;
        }
        if (!fin.empty()) s->cv_done.notify_all();
        if (fin.empty()) s->cv_work.wait_for(lk, std::chrono::microseconds(100));
    }
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
    if (cudaGetDevice(&s->dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&s->sms, cudaDevAttrMultiProcessorCount, s->dev) != cudaSuccess) {
        cudaGetLastError();
        return sfail(DA_ECUDA, "no CUDA device");
    }
    s->budget = hbm_budget_bytes;
    s->max_slots = max_requests;
    for (int i = max_requests - 1; i >= 0; --i) s->free_slots.push_back(i);
    auto bad = [&](cudaError_t e, const char* what) {
        cudaGetLastError();
        return sfail(e == cudaErrorMemoryAllocation ? DA_ENOMEM : DA_ECUDA,
                     std::string(what) + ": " + cudaGetErrorString(e));
    };
    cudaError_t e;
    {
        cudaMemPoolProps props{};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = s->dev;
        if ((e = cudaMemPoolCreate(&s->pool, &props)) != cudaSuccess) return bad(e, "memory pool");
        uint64_t keep = ~0ull;
        if ((e = cudaMemPoolSetAttribute(s->pool, cudaMemPoolAttrReleaseThreshold, &keep)) != cudaSuccess)
            return bad(e, "memory pool");
    }
    if ((e = cudaMalloc(&s->descs, sizeof(da::ServeDesc) * max_requests)) != cudaSuccess) return bad(e, "descriptors");
    if ((e = cudaMalloc(&s->done, sizeof(unsigned int) * max_requests)) != cudaSuccess) return bad(e, "counters");
    if ((e = cudaMalloc(&s->head, 8)) != cudaSuccess) return bad(e, "head");
    if ((e = cudaMemset(s->head, 0, 8)) != cudaSuccess) return bad(e, "head");
    if ((e = cudaHostAlloc(&s->ring_h, sizeof(da::ServeUnit) * kRingCap, cudaHostAllocMapped)) != cudaSuccess)
        return bad(e, "ring");
    if ((e = cudaHostAlloc(&s->tail_h, 8, cudaHostAllocMapped)) != cudaSuccess) return bad(e, "tail");
    if ((e = cudaHostAlloc(&s->flags_h, sizeof(unsigned int) * max_requests, cudaHostAllocMapped)) != cudaSuccess)
        return bad(e, "flags");
    if ((e = cudaHostAlloc(&s->stop_h, sizeof(int), cudaHostAllocMapped)) != cudaSuccess) return bad(e, "stop");
    *s->tail_h = 0;
    *s->stop_h = 0;
    std::memset(s->flags_h, 0, sizeof(unsigned int) * max_requests);
    if ((e = cudaHostGetDevicePointer(&s->ring_d, s->ring_h, 0)) != cudaSuccess) return bad(e, "ring");
    if ((e = cudaHostGetDevicePointer(&s->tail_d, s->tail_h, 0)) != cudaSuccess) return bad(e, "tail");
    if ((e = cudaHostGetDevicePointer(&s->flags_d, s->flags_h, 0)) != cudaSuccess) return bad(e, "flags");
    if ((e = cudaHostGetDevicePointer(&s->stop_d, s->stop_h, 0)) != cudaSuccess) return bad(e, "stop");
    if ((e = cudaStreamCreateWithFlags(&s->s_kernel, cudaStreamNonBlocking)) != cudaSuccess) return bad(e, "stream");
    if ((e = cudaStreamCreateWithFlags(&s->s_copy, cudaStreamNonBlocking)) != cudaSuccess) return bad(e, "stream");
    if ((e = cudaEventCreateWithFlags(&s->k_done, cudaEventDisableTiming)) != cudaSuccess) return bad(e, "event");
    // An SM runs blocks of several kernels at once only under one split of its
    // on-chip memory between L1 and shared memory.  The persistent kernel
    // needs no shared memory, and left to itself would put its SMs in a split
    // where every other kernel of the server (instance build, the anneals of
    // large requests) waits until it ends; it takes the split with the most
    // shared memory instead.
    if ((e = cudaFuncSetAttribute(reinterpret_cast<const void*>(da::serve_kernel),
                                  cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared)) !=
        cudaSuccess)
        return bad(e, "carveout");
    int per_sm = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, reinterpret_cast<const void*>(da::serve_kernel), 128, 0) !=
            cudaSuccess ||
        per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
    }
    // half of the resident capacity: the rest stays free for the chunked
    // launches of large requests
    s->kernel_blocks = std::max(1, per_sm / 2) * s->sms;
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
    if (job->dtype != DA_INT8 && job->dtype != DA_FP32)
        return sfail(DA_EINVAL, "the request loop takes DA_INT8 or DA_FP32 jobs");
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
    q->int8 = job->dtype == DA_INT8;
    q->big = q->N > 1024;
    std::string why;
    if (!da::build_instance(job->Q, q->N, q->int8 ? da::kWInt8 : da::kWFp32, q->inst, why)) return sfail(DA_EINVAL, why);
    if (q->big) {
        q->shape = da::default_shape(q->N, job->replicas);
    } else {
        int V = 4;
        while (32 * V < q->N) V *= 2;
        q->shape.V = V;
        q->shape.G = 1;
        q->shape.rpb = 4;
    }
    plan_request(*q);
    if ((int64_t)q->bytes > s->budget)
        return sfail(DA_EBUDGET, "request needs " + std::to_string(q->bytes) + " bytes, over the budget of " +
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
    __atomic_store_n(s->stop_h, 1, __ATOMIC_RELEASE);
    cudaStreamSynchronize(s->s_kernel);
    cudaStreamSynchronize(s->s_copy);
    if (s->k_done) cudaEventDestroy(s->k_done);
    if (s->s_kernel) cudaStreamDestroy(s->s_kernel);
    if (s->s_copy) cudaStreamDestroy(s->s_copy);
    cudaFree(s->descs);
    cudaFree(s->done);
    cudaFree(s->head);
    cudaFreeHost(s->ring_h);
    cudaFreeHost(s->tail_h);
    cudaFreeHost(s->flags_h);
    cudaFreeHost(s->stop_h);
    if (s->pool) cudaMemPoolDestroy(s->pool);
    delete s;
}

}  // extern "C"
