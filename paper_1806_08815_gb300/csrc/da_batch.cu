// da_batch.cu -- many instances of different sizes and coupling types annealed
// by one persistent launch per size class, captured in one CUDA graph.
//
// A work unit is one replica of one instance, run for all of its steps by one
// warp with its state in registers (WarpReplica): warps pull units from a
// device counter until none are left, so short and long instances share the
// GPU without a wave per instance.  fp32 units recompute their fields exactly
// inside the warp every `recompute_every` steps.  Units are grouped by
// (coupling type, V = variables per lane); each group is one persistent kernel
// whose configuration is chosen by a small autotuner that times short probes
// of the real work and caches the winner per device and class: warps per
// block, and where the rows of W come from (L2 in the plain order, L2 from the
// contexts' copies in the warp row order, or shared memory).  A class whose
// instances are small enough can stage W in shared memory: each block then
// takes a group of replicas of one instance (one per warp), copies that
// instance's W into shared memory once, and runs the group's anneals reading
// rows from there instead of from L2.
#include <algorithm>
#include <atomic>
#include <type_traits>
#include <chrono>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "da.h"
#include "da_internal.h"
#include "da_replica.cuh"

namespace da {

struct BatchClassParams {
    const BatchItemDev* items;
    int n_items;
    long long total_units;
    unsigned long long* head;   // work counter
    long long t_limit;          // > 0: run only this many steps per unit (autotuner probes)
    const int2* groups;         // shared-memory staging: (item, first replica) of each group
    long long n_groups;
    int pitch;                  // shared-memory staging: row pitch of the staged W (32 V entries)
};

namespace {

using step_detail::WarpReplica;

// One work unit: replica r of item it, all of its steps, by the calling warp;
// W points at the item's couplings (global memory, row pitch ldw) or at a
// copy staged in shared memory (SW, row pitch ldw = 32 V).
template <typename Tw, int V, bool SW, bool COAL = false>
__device__ __forceinline__ void run_unit(const BatchItemDev& it, int r, const Tw* W, int ldw, long long t_limit)
{
    // the precomputed draws (PRE) for V <= 16; the V = 32 kernel has no registers left for
    // them (measured slower)
    constexpr bool kPre = V <= 16;
    using R_ = WarpReplica<Tw, V, SW, kPre, (V >= 8), COAL>;
    using A = step_detail::Arith<Tw>;
    using H = typename R_::H;
    constexpr int nw = V;   // state words per replica (the padded width 32V / 32)
    const int lane = threadIdx.x & 31;
    R_ rp;
    rp.init(W, it.N, ldw, (uint32_t)r, it.xs + ((size_t)it.R + r) * nw);
#pragma unroll
    for (int v = 0; v < V; ++v) {
        if constexpr (std::is_same<Tw, step_detail::f32e>::value)   // int32 diagonal, exact in fp32
            rp.h[v] = ((rp.valid >> v) & 1u) ? __int2float_rn(static_cast<const int32_t*>(it.diag)[rp.base + v]) : 0.f;
        else
            rp.h[v] = ((rp.valid >> v) & 1u) ? static_cast<const H*>(it.diag)[rp.base + v] : H(0);
    }
    rp.xm = 0;
    rp.m = 0;
    rp.Ecur = 0;
    rp.Ebest = 0;
    rp.flips = 0;
    const PhiloxKeys keys(it.seed);
    const long long T = t_limit > 0 ? std::min(t_limit, it.T) : it.T;
    if constexpr (kPre) {
        rp.prep_draws(keys);
        if (T > 0) rp.draw_pre(0u, keys);
    } else {
        if (T > 0) rp.draw(0u, keys);
    }
    float beta_next = T > 0 ? it.beta[0] : 0.f;
    // the next step count (t + 1) at which the fp32 fields are recomputed: a running
    // target instead of a 64-bit remainder every step
    long long next_rec = std::is_same<Tw, float>::value && it.recompute_every > 0 ? it.recompute_every : -1;
    for (long long t = 0; t < T; ++t) {
        const float beta = beta_next;
        if (t + 1 < T) beta_next = it.beta[t + 1];
        const int k = rp.template step<false>(t, t + 1 < T, beta, it.inc, keys);
        if (it.trace && lane == 0) it.trace[(size_t)r * it.T + t] = k;
        if (it.stop && (t & 1023) == 1023 && *reinterpret_cast<const volatile int*>(it.stop)) break;
        if constexpr (std::is_same<Tw, float>::value) {
            if (t + 1 == next_rec) {
                next_rec += it.recompute_every;
                rp.recompute(static_cast<const float*>(it.diag), it.S, it.exact_shift != 0);
                // the draws of t + 1 again: lg is dead across the recompute, which frees its registers
                if (t + 1 < T) {
                    if constexpr (kPre) rp.draw_pre((uint32_t)(t + 1), keys);
                    else rp.draw((uint32_t)(t + 1), keys);
                }
            }
        }
    }
    rp.flush_best();
    const uint32_t word = rp.word();
    if (lane % R_::P == 0) it.xs[(size_t)r * nw + (rp.base >> 5)] = word;
    if (lane == 0) {
        ReplicaScalars s;
        s.E = A::store_e(rp.Ecur);
        s.best = A::store_e(rp.Ebest);
        s.flips = rp.flips;
        s.m = rp.m;
        s.check = 0;
        it.sc[r] = s;
    }
}

// COAL: rows of W from the items' copies in the one-warp row order (it.Wc).
template <typename Tw, int V, bool COAL = false>
__global__ void __launch_bounds__(128) batch_kernel(const __grid_constant__ BatchClassParams bp)
{
    const int lane = threadIdx.x & 31;
    for (;;) {
        unsigned long long unit = 0;
        if (lane == 0) unit = atomicAdd(bp.head, 1ull);
        unit = __shfl_sync(0xffffffffu, unit, 0);
        if (unit >= (unsigned long long)bp.total_units) break;
        // the item holding this unit (items sorted by unit0)
        int lo = 0, hi = bp.n_items - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if ((unsigned long long)bp.items[mid].unit0 <= unit) lo = mid;
            else hi = mid - 1;
        }
        const BatchItemDev it = bp.items[lo];
        const int r = (int)(unit - (unsigned long long)it.unit0);
        if constexpr (COAL) run_unit<Tw, V, false, true>(it, r, static_cast<const Tw*>(it.Wc), 32 * V, bp.t_limit);
        else run_unit<Tw, V, false>(it, r, static_cast<const Tw*>(it.W), it.ldw, bp.t_limit);
    }
}

// Shared-memory staging: the block takes group g = (item, r0) from the
// counter, copies rows 0..N-1 of the item's W into shared memory (row pitch
// 32 V, zeros beyond column N), and warp w runs replica r0 + w.
template <typename Tw, int V>
__global__ void __launch_bounds__(512) batch_kernel_smem(const __grid_constant__ BatchClassParams bp)
{
    extern __shared__ __align__(16) unsigned char wsm_raw[];
    Tw* Ws = reinterpret_cast<Tw*>(wsm_raw);
    __shared__ long long s_group;
    const int warp = threadIdx.x >> 5;
    for (;;) {
        __syncthreads();   // every warp is done with the previous group's copy
        if (threadIdx.x == 0) s_group = (long long)atomicAdd(bp.head, 1ull);
        __syncthreads();
        const long long g = s_group;
        if (g >= bp.n_groups) break;
        const int2 gi = bp.groups[g];
        const BatchItemDev it = bp.items[gi.x];
        const Tw* Wg = static_cast<const Tw*>(it.W);
        const int cols = bp.pitch;
        for (int e = threadIdx.x; e < it.N * cols; e += blockDim.x) {
            const int row = e / cols, col = e - row * cols;
            Tw v{};
            if (col < it.N) v = Wg[(size_t)row * it.ldw + col];
            Ws[e] = v;
        }
        __syncthreads();
        const int r = gi.y + warp;
        if (r < it.R) run_unit<Tw, V, true>(it, r, Ws, cols, bp.t_limit);
    }
}

typedef void (*BatchKernel)(BatchClassParams);

// Kernels per step coupling form wk: kWInt8AsF32 (int8 instances, exact fp32
// couplings), kWFp32, kWInt16 (16-bit couplings, int32 fields; rows from L2
// only: the staged copy holds 4-byte entries).
BatchKernel smem_kernel_for(int wk, int V)
{
    if (wk == kWInt16) return nullptr;
    if (wk == kWInt8AsF32) {
        switch (V) {
        case 4: return batch_kernel_smem<step_detail::f32e, 4>;
        case 8: return batch_kernel_smem<step_detail::f32e, 8>;
        }
    } else {
        switch (V) {
        case 4: return batch_kernel_smem<float, 4>;
        case 8: return batch_kernel_smem<float, 8>;
        }
    }
    return nullptr;
}

// The rows-from-L2 kernel of a class; coal: its items carry the row-ordered copies
// (the fp32 forms at V >= 8).
BatchKernel kernel_for(int wk, int V, bool coal)
{
    if (coal && wk == kWInt8AsF32) {
        switch (V) {
        case 8: return batch_kernel<step_detail::f32e, 8, true>;
        case 16: return batch_kernel<step_detail::f32e, 16, true>;
        case 32: return batch_kernel<step_detail::f32e, 32, true>;
        }
        return nullptr;
    }
    if (coal && wk == kWFp32) {
        switch (V) {
        case 8: return batch_kernel<float, 8, true>;
        case 16: return batch_kernel<float, 16, true>;
        case 32: return batch_kernel<float, 32, true>;
        }
        return nullptr;
    }
    if (wk == kWInt16) {
        switch (V) {
        case 4: return batch_kernel<int16_t, 4>;
        case 8: return batch_kernel<int16_t, 8>;
        case 16: return batch_kernel<int16_t, 16>;
        case 32: return batch_kernel<int16_t, 32>;
        }
    } else if (wk == kWInt8AsF32) {
        switch (V) {
        case 4: return batch_kernel<step_detail::f32e, 4>;
        case 8: return batch_kernel<step_detail::f32e, 8>;
        case 16: return batch_kernel<step_detail::f32e, 16>;
        case 32: return batch_kernel<step_detail::f32e, 32>;
        }
    } else {
        switch (V) {
        case 4: return batch_kernel<float, 4>;
        case 8: return batch_kernel<float, 8>;
        case 16: return batch_kernel<float, 16>;
        case 32: return batch_kernel<float, 32>;
        }
    }
    return nullptr;
}

// OR of the items' tensor-core error flags (a bounded wait inside an exact
// evaluation that gave up) into *out.
__global__ void collect_flags_kernel(int* const* flags, int n, int* out)
{
    int any = 0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) any |= *flags[i];
    any = __syncthreads_or(any);
    if (threadIdx.x == 0) *out = any;
}

__global__ void batch_finalize_kernel(bool int8, int R, const ReplicaScalars* sc, const long long* eex,
                                      double* out /* [4][R] */)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    const double ef = int8 ? (double)eex[r] : __longlong_as_double(eex[r]);
    const double eb = int8 ? (double)eex[R + r] : __longlong_as_double(eex[R + r]);
    const double tr = int8 ? (double)sc[r].E : __longlong_as_double(sc[r].E);
    out[r] = ef;
    out[R + r] = eb;
    out[2 * R + r] = fabs(tr - ef);
    reinterpret_cast<long long*>(out)[3 * R + r] = sc[r].flips;
}

size_t al(size_t v) { return (v + 255) / 256 * 256; }

// Autotuner: the configuration of the persistent kernel of one class (where
// rows of W come from, warps per block), chosen by timing probes of the class's
// own first units; cached per (device, class, whether staging fits, size of
// the probe: a class too small to fill the GPU is tuned again when it grows).
struct BatchConfig {
    bool smem = false;
    int warps_per_block = 4;
    bool coal = false;   // rows from L2 in the one-warp row order (BatchClass::coal)
};
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, bool, int>, BatchConfig> g_tune_cache;
std::map<std::tuple<int, int, int, bool, int>, std::string> g_tune_log;   // the probes behind each entry
thread_local std::string g_batch_desc;

// Steps per unit of a tuner probe.
constexpr long long kProbeSteps = 1024;

// Largest dynamic shared memory a block may ask for on sm_100-class GPUs.
constexpr size_t kMaxStagedBytes = 227u * 1024u;

int blocks_for(BatchKernel k, int warps_per_block, int sms, size_t smem)
{
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, reinterpret_cast<const void*>(k), warps_per_block * 32,
                                                      smem) != cudaSuccess ||
        per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
    }
    return per_sm * sms;
}

}  // namespace

// Host side of one class: items already laid out in device memory.
struct BatchClass {
    int wk;                      // step coupling form (kWInt8AsF32, kWFp32, kWInt16)
    int V;
    std::vector<int> item_idx;   // indices into the caller's item array
    BatchItemDev* items_dev;
    int n_items;
    long long units;
    unsigned long long* head;
    int2* groups_dev;            // room for the groups of 2 replicas (the smallest staged group)
    int max_N;
    BatchConfig cfg;
    std::string probes;          // the tuner's measurements, for da_batch_describe
    size_t staged_bytes() const { return (size_t)max_N * 32 * V * 4; }
    bool can_stage() const { return smem_kernel_for(wk, V) != nullptr && staged_bytes() <= kMaxStagedBytes; }
    // rows from L2 may come in the one-warp row order (every item carries its copy, Host::Wc)
    bool coal() const { return (wk == kWFp32 || wk == kWInt8AsF32) && V >= 8; }
};

// Groups of `wpb` replicas, each within one item, covering the first `units` units.
std::vector<int2> make_groups(const std::vector<int>& replicas_per_item, int wpb, long long units)
{
    std::vector<int2> g;
    long long covered = 0;
    for (int i = 0; i < (int)replicas_per_item.size() && covered < units; ++i)
        for (int r0 = 0; r0 < replicas_per_item[i] && covered < units; r0 += wpb) {
            g.push_back(make_int2(i, r0));
            covered += std::min(wpb, replicas_per_item[i] - r0);
        }
    return g;
}

// One launch of a class's kernel in configuration cfg over its first `units`
// units (all of them for the real run), t_limit steps per unit (0: all).
cudaError_t launch_class(const BatchClass& c, const std::vector<int>& reps, const BatchConfig& cfg, long long units,
                         long long t_limit, int sms, cudaStream_t st, bool upload_groups)
{
    BatchClassParams bp{c.items_dev, c.n_items, units, c.head, t_limit, nullptr, 0, 0};
    if (!cfg.smem) {
        BatchKernel k = kernel_for(c.wk, c.V, cfg.coal && c.coal());
        k<<<blocks_for(k, cfg.warps_per_block, sms, 0), cfg.warps_per_block * 32, 0, st>>>(bp);
        return cudaGetLastError();
    }
    BatchKernel k = smem_kernel_for(c.wk, c.V);
    const size_t bytes = c.staged_bytes();
    cudaError_t e = cudaFuncSetAttribute(reinterpret_cast<const void*>(k),
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    const std::vector<int2> groups = make_groups(reps, cfg.warps_per_block, units);
    if (upload_groups) {
        e = cudaMemcpyAsync(c.groups_dev, groups.data(), groups.size() * sizeof(int2), cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return e;
    }
    bp.groups = c.groups_dev;
    bp.n_groups = (long long)groups.size();
    bp.pitch = 32 * c.V;
    k<<<blocks_for(k, cfg.warps_per_block, sms, bytes), cfg.warps_per_block * 32, bytes, st>>>(bp);
    return cudaGetLastError();
}

// da_batch_force: staging -1 = the tuner's choice, 0 = rows from L2, 1 = staged where
// the class allows; warps per block 0 = the tuner's choice.
std::atomic<int> g_force_staging{-1}, g_force_wpb{0};

BatchConfig tune_class(BatchClass& c, const std::vector<int>& reps, int dev, int sms, cudaStream_t st)
{
    const int fs = g_force_staging.load(), fw = g_force_wpb.load();
    if (fs >= 0 || fw > 0) {
        BatchConfig cfg;
        cfg.smem = fs == 1 && c.can_stage();
        cfg.coal = fs == 2 && c.coal();
        cfg.warps_per_block = fw > 0 ? fw : (cfg.smem ? 8 : 4);
        if (!cfg.smem) cfg.warps_per_block = std::min(cfg.warps_per_block, 4);   // the L2 kernel's block limit
        if (cfg.smem) cfg.warps_per_block = std::max(cfg.warps_per_block, 2);
        c.probes = "forced";
        return cfg;
    }
    const long long units = std::min<long long>(c.units, (long long)sms * 16);
    int ubits = 0;
    while ((2ll << ubits) <= units) ++ubits;   // floor(log2(probe units))
    const auto key = std::make_tuple(dev, c.wk, c.V, c.can_stage(), ubits);
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        auto f = g_tune_cache.find(key);
        if (f != g_tune_cache.end()) {
            c.probes = "cached; " + g_tune_log[key];
            return f->second;
        }
    }
    std::vector<BatchConfig> cands;
    for (int wpb : {1, 2, 4}) cands.push_back(BatchConfig{false, wpb, false});
    if (c.coal())
        for (int wpb : {1, 2, 4}) cands.push_back(BatchConfig{false, wpb, true});
    if (c.can_stage())
        for (int wpb : {2, 4, 8, 16}) cands.push_back(BatchConfig{true, wpb, false});
    BatchConfig best = cands.front();
    float best_l2 = 1e30f, best_staged = 1e30f, best_coal = 1e30f;
    BatchConfig cfg_l2 = cands.front(), cfg_staged = cands.front(), cfg_coal = cands.front();
    auto label = [](const BatchConfig& cfg) {
        return std::string(cfg.smem ? "smem" : cfg.coal ? "l2r" : "l2") + "x" + std::to_string(cfg.warps_per_block);
    };
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        cudaGetLastError();
        return best;
    }
    std::string log;
    for (const BatchConfig& cfg : cands) {
        cudaMemsetAsync(c.head, 0, 8, st);
        cudaEventRecord(e0, st);
        cudaError_t le = launch_class(c, reps, cfg, units, kProbeSteps, sms, st, true);
        cudaEventRecord(e1, st);
        if (le == cudaSuccess) le = cudaStreamSynchronize(st);
        if (le != cudaSuccess) {
            cudaGetLastError();
            log += std::string(log.empty() ? "" : ", ") + label(cfg) + " failed: " + cudaGetErrorString(le);
            continue;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        log += std::string(log.empty() ? "" : ", ") + label(cfg) + " " + std::to_string(ms).substr(0, 6) + " ms";
        if (cfg.coal && ms < best_coal) {
            best_coal = ms;
            cfg_coal = cfg;
        }
        if (!cfg.smem && !cfg.coal && ms < best_l2) {
            best_l2 = ms;
            cfg_l2 = cfg;
        }
        if (cfg.smem && ms < best_staged) {
            best_staged = ms;
            cfg_staged = cfg;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    // the row-ordered rows are taken when their probe beats the plain order's by more than 1 %,
    // staging only when its probe beats the best L2 configuration by more than the run-to-run
    // spread of these probes (3 %)
    if (best_l2 < 1e30f) best = cfg_l2;
    if (best_coal < 0.99f * best_l2) {
        best = cfg_coal;
        best_l2 = best_coal;
    }
    if (best_staged < 0.97f * best_l2) best = cfg_staged;
    c.probes = "probes (" + std::to_string(units) + " replicas x " + std::to_string(kProbeSteps) + " steps): " + log;
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune_cache[key] = best;
    g_tune_log[key] = c.probes;
    return best;
}

}  // namespace da

using da::BatchClass;
using da::BatchItemDev;


namespace {
da_status bfail(da_status s, const std::string& m)
{
    da::set_last_error(m);
    return s;
}
}  // namespace

extern "C" da_status da_batch_anneal(const da_batch_item* items, int32_t n, double* elapsed_s)
{
    da::set_last_error("");
    if (!items || n < 1) return bfail(DA_EINVAL, "need items");
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return bfail(DA_ECUDA, "no device");
    struct Host {
        const void* W;       // couplings for the exact evaluation
        const void* Wstep;   // couplings in the step kernel's form (int8 instances: exact fp32)
        const void* Wc;      // the step couplings in the one-warp row order (fp32 forms, V >= 8), or null
        int dtype;           // da_dtype of the instance
        const void* diag;
        int N, ldw, S;
        bool int8;
        int V;
    };
    std::vector<Host> hi((size_t)n);
    for (int i = 0; i < n; ++i) {
        const da_batch_item& it = items[i];
        int64_t N = 0;
        da_dtype dt;
        if (!it.ctx || da_ctx_info(it.ctx, &N, &dt) != DA_OK) return bfail(DA_EINVAL, "item " + std::to_string(i) + ": bad context");
        if (N > 1024) return bfail(DA_EINVAL, "item " + std::to_string(i) + ": the batched launch takes N <= 1024");

        if (it.replicas < 1 || it.steps < 0 || it.steps >= (1ll << 32) || (it.steps > 0 && !it.beta))
            return bfail(DA_EINVAL, "item " + std::to_string(i) + ": bad replicas/steps/schedule");
        if (it.steps > 0 && !da::schedule_ok(it.beta, it.steps))
            return bfail(DA_EINVAL, "item " + std::to_string(i) + ": beta must be finite and >= 0");
        if (!(it.offset_inc >= 0.f) || !std::isfinite(it.offset_inc) || it.recompute_every < 0)
            return bfail(DA_EINVAL, "item " + std::to_string(i) + ": bad offset or recompute period");
        Host h{};
        int32_t ldw = 0, S = 0;
        da::ctx_device_view(it.ctx, &h.W, &h.diag, &ldw, &S, &h.Wstep);
        h.N = (int)N;
        h.ldw = ldw;
        h.S = S;
        h.int8 = dt != DA_FP32;   // integer couplings: exact fields and energies
        h.dtype = (int)dt;
        int V = 4;
        while (32 * V < h.N) V *= 2;
        h.V = V;
        h.Wc = nullptr;
        if ((dt == DA_FP32 || dt == DA_INT8) && V >= 8) {
            h.Wc = da::ctx_coal_W(it.ctx, V);
            if (!h.Wc) return bfail(DA_ENOMEM, "item " + std::to_string(i) + ": " + da_last_error());
        }
        hi[i] = h;
    }
    // device layout: per item betas, states, scalars, traces, results; per class descriptors
    std::vector<size_t> o_beta(n), o_xs(n), o_sc(n), o_tr(n), o_eex(n), o_part(n), o_res(n);
    size_t off = 0;
    for (int i = 0; i < n; ++i) {
        const int R = items[i].replicas, nw = hi[i].V;
        o_beta[i] = off; off += da::al((size_t)items[i].steps * 4);
        o_xs[i] = off; off += da::al((size_t)2 * R * nw * 4);
        o_sc[i] = off; off += da::al((size_t)R * sizeof(da::ReplicaScalars));
        o_tr[i] = off; off += items[i].out && items[i].out->trace ? da::al((size_t)R * items[i].steps * 4) : 0;
        o_eex[i] = off; off += da::al((size_t)2 * R * 8);
        o_part[i] = off; off += da::al(da::tc_partial_bytes(hi[i].N, 2 * R));
        o_res[i] = off; off += da::al((size_t)4 * R * 8);
    }
    std::map<std::pair<int, int>, BatchClass> classes;
    for (int i = 0; i < n; ++i) {
        const int wk = hi[i].dtype == DA_INT8 ? da::kWInt8AsF32 : hi[i].dtype;
        auto& c = classes[{wk, hi[i].V}];
        c.wk = wk;
        c.V = hi[i].V;
        c.max_N = std::max(c.max_N, hi[i].N);
        c.item_idx.push_back(i);
    }
    const size_t o_desc = off;
    off += da::al((size_t)n * sizeof(BatchItemDev));
    const size_t o_heads = off;
    off += da::al(classes.size() * 8);
    const size_t o_flags = off;   // the items' error-flag pointers, then their OR
    off += da::al((size_t)n * sizeof(int*) + sizeof(int));
    // per class: room for its groups of two replicas (the smallest group a staged launch uses)
    std::map<std::pair<int, int>, size_t> o_groups;
    for (auto& kv : classes) {
        size_t g = 0;
        for (int i : kv.second.item_idx) g += (size_t)(items[i].replicas + 1) / 2;
        o_groups[kv.first] = off;
        off += da::al(g * sizeof(int2));
    }
    char* base = nullptr;
    if (da::dev_malloc(reinterpret_cast<void**>(&base), off) != cudaSuccess) {
        cudaGetLastError();
        return bfail(DA_ENOMEM, "batch workspace of " + std::to_string(off) + " bytes");
    }
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    da_status status = DA_OK;
    auto cleanup = [&]() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        if (st) cudaStreamDestroy(st);
        da::dev_free(base);
    };
#define DA_B(call)                                                                         \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess) {                                                           \
            status = bfail(DA_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));  \
            cudaGetLastError();                                                            \
            cleanup();                                                                     \
            return status;                                                                 \
        }                                                                                  \
    } while (0)
    DA_B(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    DA_B(cudaEventCreate(&e0));
    DA_B(cudaEventCreate(&e1));
    std::vector<BatchItemDev> desc((size_t)n);
    {
        size_t di = 0;
        int ci = 0;
        for (auto& kv : classes) {
            BatchClass& c = kv.second;
            long long units = 0;
            c.items_dev = reinterpret_cast<BatchItemDev*>(base + o_desc) + di;
            c.n_items = (int)c.item_idx.size();
            c.head = reinterpret_cast<unsigned long long*>(base + o_heads) + ci;
            c.groups_dev = reinterpret_cast<int2*>(base + o_groups[kv.first]);
            for (int i : c.item_idx) {
                const da_batch_item& it = items[i];
                BatchItemDev d{};
                d.W = hi[i].Wstep;
                d.Wc = hi[i].Wc;
                d.diag = hi[i].diag;
                d.beta = reinterpret_cast<const float*>(base + o_beta[i]);
                d.xs = reinterpret_cast<uint32_t*>(base + o_xs[i]);
                d.sc = reinterpret_cast<da::ReplicaScalars*>(base + o_sc[i]);
                d.trace = it.out && it.out->trace ? reinterpret_cast<int*>(base + o_tr[i]) : nullptr;
                d.T = it.steps;
                d.recompute_every = hi[i].int8 ? 0 : it.recompute_every;
                d.unit0 = units;
                d.seed = it.seed;
                d.N = hi[i].N;
                d.ldw = hi[i].ldw;
                d.S = hi[i].S;
                d.R = it.replicas;
                d.inc = it.offset_inc;
                d.exact_shift = da::ctx_exact_shift(it.ctx) ? 1 : 0;
                desc[di++] = d;
                units += it.replicas;
            }
            c.units = units;
            ++ci;
        }
    }
    // uploads (outside the graph: the schedules, descriptors and error-flag pointers)
    {
        std::vector<int*> fl((size_t)n);
        for (int i = 0; i < n; ++i) fl[i] = da::ctx_tc_operand(items[i].ctx).err;
        DA_B(cudaMemcpyAsync(base + o_flags, fl.data(), fl.size() * sizeof(int*), cudaMemcpyHostToDevice, st));
        DA_B(cudaStreamSynchronize(st));
    }
    for (int i = 0; i < n; ++i)
        if (items[i].steps > 0)
            DA_B(cudaMemcpyAsync(base + o_beta[i], items[i].beta, (size_t)items[i].steps * 4, cudaMemcpyHostToDevice, st));
    {
        // descriptors in class order
        size_t di = 0;
        std::vector<BatchItemDev> ordered((size_t)n);
        for (auto& kv : classes)
            for (size_t q = 0; q < kv.second.item_idx.size(); ++q) ordered[di] = desc[di], ++di;
        DA_B(cudaMemcpyAsync(base + o_desc, ordered.data(), (size_t)n * sizeof(BatchItemDev), cudaMemcpyHostToDevice, st));
    }
    for (int i = 0; i < n; ++i)
        DA_B(cudaMemsetAsync(base + o_xs[i], 0, (size_t)2 * items[i].replicas * hi[i].V * 4, st));
    DA_B(cudaStreamSynchronize(st));
    // replicas of each class's items, in the class's item order (for the staged groups)
    std::map<std::pair<int, int>, std::vector<int>> reps;
    for (auto& kv : classes)
        for (int i : kv.second.item_idx) reps[kv.first].push_back(items[i].replicas);
    std::string desc_text;
    for (auto& kv : classes) {
        BatchClass& c = kv.second;
        c.cfg = da::tune_class(c, reps[kv.first], dev, sms, st);
        desc_text += std::string(desc_text.empty() ? "" : "; ") + (c.wk == da::kWFp32 ? "fp32" : c.wk == da::kWInt16 ? "int16" : "int8") + " V=" +
                     std::to_string(c.V) + " (N <= " + std::to_string(c.max_N) + ", " + std::to_string(c.n_items) +
                     " instances, " + std::to_string(c.units) + " replicas): " +
                     (c.cfg.smem ? "W staged in shared memory"
                                 : c.cfg.coal ? "rows of W from L2 in the one-warp row order" : "rows of W from L2") +
                     ", " +
                     std::to_string(c.cfg.warps_per_block) + " warps per block [" + c.probes + "]";
    }
    da::g_batch_desc = desc_text;
    for (int i = 0; i < n; ++i)
        DA_B(cudaMemsetAsync(base + o_xs[i], 0, (size_t)2 * items[i].replicas * hi[i].V * 4, st));
    // the staged classes' group tables for the whole run (uploaded before the capture)
    for (auto& kv : classes) {
        const BatchClass& c = kv.second;
        if (!c.cfg.smem) continue;
        const std::vector<int2> groups = da::make_groups(reps[kv.first], c.cfg.warps_per_block, c.units);
        DA_B(cudaMemcpyAsync(c.groups_dev, groups.data(), groups.size() * sizeof(int2), cudaMemcpyHostToDevice, st));
        DA_B(cudaStreamSynchronize(st));
    }
    DA_B(cudaStreamSynchronize(st));

    // the graph: persistent kernel per class, then the exact evaluation of every item
    DA_B(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    bool capture_ok = true;
    DA_B(cudaMemsetAsync(base + o_heads, 0, classes.size() * 8, st));
    std::string launch_err;
    for (auto& kv : classes) {
        const BatchClass& c = kv.second;
        const cudaError_t le = da::launch_class(c, reps[kv.first], c.cfg, c.units, 0, sms, st, false);
        if (le != cudaSuccess) {
            if (capture_ok) launch_err = std::string(" (class launch: ") + cudaGetErrorString(le) + ")";
            capture_ok = false;
        }
    }
    for (auto& kv : classes) {
        for (int i : kv.second.item_idx) {
            const int R = items[i].replicas, nw = hi[i].V;
            long long* eex = reinterpret_cast<long long*>(base + o_eex[i]);
            // the exact evaluation of final and best states on the tensor cores (the item's
            // context holds the operand of its couplings)
            if (da::launch_recompute_tc(hi[i].int8, da::ctx_tc_operand(items[i].ctx), hi[i].diag, hi[i].N, hi[i].S,
                                        reinterpret_cast<uint32_t*>(base + o_xs[i]), nw, 2 * R, nullptr, hi[i].N, eex,
                                        1, st, reinterpret_cast<long long*>(base + o_part[i])) != cudaSuccess)
                capture_ok = false;
            da::batch_finalize_kernel<<<(R + 127) / 128, 128, 0, st>>>(
                hi[i].int8, R, reinterpret_cast<da::ReplicaScalars*>(base + o_sc[i]), eex,
                reinterpret_cast<double*>(base + o_res[i]));
        }
    }
    int* flag_out = reinterpret_cast<int*>(base + o_flags + (size_t)n * sizeof(int*));
    da::collect_flags_kernel<<<1, 256, 0, st>>>(reinterpret_cast<int* const*>(base + o_flags), n, flag_out);
    cudaError_t ce = cudaStreamEndCapture(st, &graph);
    if (ce != cudaSuccess || !capture_ok) {
        status = bfail(DA_ECUDA, std::string("graph capture: ") + cudaGetErrorString(ce) + launch_err);
        cudaGetLastError();
        cleanup();
        return status;
    }
    DA_B(cudaGraphInstantiate(&exec, graph, 0));
    DA_B(cudaEventRecord(e0, st));
    DA_B(cudaGraphLaunch(exec, st));
    DA_B(cudaEventRecord(e1, st));
    // results
    for (int i = 0; i < n; ++i) {
        da_result* out = items[i].out;
        if (!out) continue;
        const int R = items[i].replicas, nw = hi[i].V;
        const size_t words = (size_t)(hi[i].N + 31) / 32;
        if (out->final_x)
            DA_B(cudaMemcpy2DAsync(out->final_x, words * 4, base + o_xs[i], (size_t)nw * 4, words * 4, R,
                                   cudaMemcpyDeviceToHost, st));
        if (out->best_x)
            DA_B(cudaMemcpy2DAsync(out->best_x, words * 4, base + o_xs[i] + (size_t)R * nw * 4, (size_t)nw * 4, words * 4,
                                   R, cudaMemcpyDeviceToHost, st));
        if (out->trace && items[i].steps > 0)
            DA_B(cudaMemcpyAsync(out->trace, base + o_tr[i], (size_t)R * items[i].steps * 4, cudaMemcpyDeviceToHost, st));
    }
    std::vector<std::vector<double>> res((size_t)n);
    for (int i = 0; i < n; ++i) {
        res[i].resize((size_t)4 * items[i].replicas);
        DA_B(cudaMemcpyAsync(res[i].data(), base + o_res[i], res[i].size() * 8, cudaMemcpyDeviceToHost, st));
    }
    int flag = 0;
    DA_B(cudaMemcpyAsync(&flag, flag_out, sizeof(int), cudaMemcpyDeviceToHost, st));
    DA_B(cudaStreamSynchronize(st));
    if (flag) {
        for (int i = 0; i < n; ++i) cudaMemsetAsync(da::ctx_tc_operand(items[i].ctx).err, 0, sizeof(int), st);
        cudaStreamSynchronize(st);
        status = bfail(DA_ETIMEOUT, "a bounded wait inside an exact evaluation gave up; the results are invalid");
        cleanup();
        return status;
    }
    float ms = 0.f;
    DA_B(cudaEventElapsedTime(&ms, e0, e1));
    if (elapsed_s) *elapsed_s = ms * 1e-3;
    for (int i = 0; i < n; ++i) {
        da_result* out = items[i].out;
        if (!out) continue;
        const int R = items[i].replicas;
        for (int r = 0; r < R; ++r) {
            if (out->final_E) out->final_E[r] = res[i][r];
            if (out->best_E) out->best_E[r] = res[i][R + r];
            if (out->max_drift) out->max_drift[r] = res[i][2 * R + r];
            if (out->flips) out->flips[r] = reinterpret_cast<const int64_t*>(res[i].data())[3 * R + r];
        }
        out->elapsed_s = ms * 1e-3;
    }
    cleanup();
    return DA_OK;
#undef DA_B
}

extern "C" da_status da_batch_describe(char* buf, int64_t len)
{
    if (!buf || len < 1) return DA_EINVAL;
    const std::string& d = da::g_batch_desc;
    const size_t n = std::min<size_t>(d.size(), (size_t)len - 1);
    std::memcpy(buf, d.data(), n);
    buf[n] = 0;
    return DA_OK;
}

extern "C" da_status da_batch_force(int32_t staging, int32_t warps_per_block)
{
    const bool wpb_ok = warps_per_block == 0 || warps_per_block == 1 || warps_per_block == 2 ||
                        warps_per_block == 4 || warps_per_block == 8 || warps_per_block == 16;
    if (staging < -1 || staging > 2 || !wpb_ok || (staging != 1 && warps_per_block > 4)) {
        da::set_last_error("staging in {-1, 0, 1, 2}; warps per block in {0, 1, 2, 4} (up to 16 when staged)");
        return DA_EINVAL;
    }
    if (staging == 1 && warps_per_block == 1) {
        da::set_last_error("a staged block runs at least 2 warps");
        return DA_EINVAL;
    }
    da::g_force_staging = staging;
    da::g_force_wpb = warps_per_block;
    return DA_OK;
}

namespace da {

cudaError_t launch_resident_anneal(int wk, int V, const BatchItemDev* item_dev, unsigned long long* head_dev, int R,
                                   cudaStream_t st)
{
    BatchKernel k = kernel_for(wk, V, false);   // a request's item carries no row-ordered copy
    if (!k) return cudaErrorInvalidValue;
    prefer_shared_fn(reinterpret_cast<const void*>(k));
    cudaError_t e = cudaMemsetAsync(head_dev, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    BatchClassParams bp{item_dev, 1, R, head_dev, 0, nullptr, 0, 0};
    k<<<R, 32, 0, st>>>(bp);   // one warp per replica, each SM it lands on shared with other requests
    return cudaGetLastError();
}

cudaError_t prepare_resident_kernels()
{
    for (int wk : {kWInt8AsF32, kWFp32, kWInt16})
        for (int V : {4, 8, 16, 32}) prefer_shared_fn(reinterpret_cast<const void*>(kernel_for(wk, V, false)));
    return cudaGetLastError();
}

}  // namespace da
