"""Benchmark of the Digital Annealer hot path on one GB300 (or N, one process each).

Workload (one "step" = one complete anneal): fully connected SK spin glass,
N = 1024, Gaussian couplings J_ij ~ N(0, 1)/sqrt(N) in an fp32 QUBO (4 MB),
1024 replicas, 2e5 DA steps, beta linear 0.1 -> 10, fp32 fields with the exact
field recompute every 1024 steps.  Metric: single-flip trials per second,
R * T * N / time, plus TTS99 from the hit rate of the best energy over all
runs.  The instance is synthetic (seeded), standing in for the paper's SK
instances.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line (rank 0).  --impl reference times the CPU oracle on the
host cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "single-flip trials/s (DA step, SK-Gaussian N=1024, 1024 replicas, 2e5 steps)"
UNIT = "trials/s"

C3 = dict(N=1024, replicas=1024, steps=200_000, recompute_every=1024, beta0=0.1, beta1=10.0, inc=0.0,
          instance_seed=0, seed=0)

# DRAM bytes per step-kernel launch (dram__bytes_read.sum + dram__bytes_write.sum) from one ncu
# capture of the headline workload, valid while the kernel source has the recorded hash.
# Warp instructions per replica-step of the step kernel (smsp__inst_executed.sum / (R x steps))
# from the same capture: the issue-slot roofline of a kernel bound by instruction issue.
STEP_INST_PER_REPLICA_STEP = 716.0
STEP_TRAFFIC = {"source_sha256_16": "80c60f7704049e9c", "bytes_per_launch": 8.5962e6}


def step_source_sha():
    import hashlib
    h = hashlib.sha256()
    for f in ("da_step.cuh", "da_replica.cuh", "da_step_common.cuh", "da_device.cuh"):
        h.update(open(os.path.join(ROOT, "paper_1806_08815_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def issue_roofline(replica_steps_per_launch, launch_s, sms, sm_ghz):
    """Issue-slot roofline of the step kernel (the resource that binds it: a chain of dependent
    instructions per step, no contraction, a few KB of row reads per replica-step from L2): warp
    instructions per launch (the ncu count per replica-step of this kernel source) over the launch
    time, against 4 warp-instructions per cycle per SM (one per scheduler) x SMs x the SM clock."""
    achieved = STEP_INST_PER_REPLICA_STEP * replica_steps_per_launch / launch_s / 1e9
    peak = sms * 4 * sm_ghz
    fresh = step_source_sha() == STEP_TRAFFIC["source_sha256_16"]
    if not fresh:
        print("bench.py: the step kernel changed since its instruction count was taken; the issue "
              "roofline uses the old count", file=sys.stderr)
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "G warp-inst/s", "frac": achieved / peak,
            "traffic": STEP_TRAFFIC["bytes_per_launch"] if fresh else None,
            "inst_per_replica_step": STEP_INST_PER_REPLICA_STEP, "count_matches_source": fresh,
            "peak_source": f"4 warp-instructions / cycle / SM x {sms} SMs x {sm_ghz:.3f} GHz (median SM clock "
                           "sampled during the timed region)",
            "basis": "ncu smsp__inst_executed.sum per replica-step x replica-steps per launch / launch time"}


def read_bandwidths(da, dev):
    """L2 read bandwidth measured on this GPU with the library's read kernel: a buffer of the size of
    the headline W (4 MB, the rows the step kernel reads) and one spread over every L2 slice (64 MB)."""
    import torch
    out = {}
    for key, mb in (("w_sized_4mb", 4), ("l2_64mb", 64)):
        buf = torch.zeros(mb << 20, dtype=torch.uint8, device=dev)
        out[key] = max(da.da_diag_read_bandwidth(buf, max(1, 4096 // mb)) for _ in range(3)) / 1e9
        del buf
    return out


def recompute_roofline(peaks, peak_src, N, R, n_recompute, rest_s):
    """Tensor roofline of the exact field recompute (tensor-core kernel + energy sum):
    time per recompute = (anneal time - step-kernel time) / (periodic recomputes + the final
    evaluation of 2R states, counted as 2); algorithmic work 2 N^2 R flop per recompute of R
    states, executed as 5 f16 digit planes (N = 1024)."""
    if n_recompute < 1 or rest_s <= 0:
        return None
    per = rest_s / (n_recompute + 2)
    algo = 2.0 * N * N * R
    peak = float(peaks.get("bf16_tflops", 1900.0))       # f16 and bf16 run at the same dense rate
    ach = algo / per / 1e12
    return {"bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
            "executed_tflops": 5 * ach, "per_recompute_us": per * 1e6, "peak_source": peak_src,
            "basis": "algorithmic 2 N^2 R flop per recompute; executed = 5 digit planes; time per recompute "
                     "from the anneal time minus the step-kernel time (includes the energy sums)"}


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            d = json.load(open(p))
            return d, "measured"
        except Exception:
            pass
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def hbm_peak(peaks):
    for k in ("hbm_gbs", "hbm_GBs", "hbm_copy_gbs", "hbm"):
        v = peaks.get(k)
        if isinstance(v, (int, float)):
            return float(v)
        if isinstance(v, dict):
            for kk in ("gbs", "value", "GB/s"):
                if isinstance(v.get(kk), (int, float)):
                    return float(v[kk])
    return 6800.0


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


def tts99(best_E, tau_run):
    """TTS99 = tau * R99 with theta from the Jeffreys posterior mean (Scaling Analysis section)."""
    Eref = float(np.min(best_E))
    tol = 1e-6 * max(1.0, abs(Eref))
    y = int(np.sum(best_E <= Eref + tol))
    r = len(best_E)
    theta = (y + 0.5) / (r + 1.0)
    # at least one run: above theta = 0.99 the formula gives fewer (as the bootstrap clamps)
    R99 = max(1.0, math.log(1 - 0.99) / math.log(1 - theta)) if theta < 1 else 1.0
    return dict(E_ref=Eref, hits=y, runs=r, theta=theta, R99=R99, tts99_s=tau_run * R99)


def _tts_from_best(best_E, tau_run):
    """TTS99 of one instance from its runs' best energies (reference = best over the runs)."""
    return tts99(np.asarray(best_E), tau_run)


def _hits_tts(best, E_ref, tau_run):
    """TTS99 of one form on one instance against a given reference energy (Jeffreys posterior)."""
    tol = 1e-6 * max(1.0, abs(E_ref))
    y = int(np.sum(np.asarray(best) <= E_ref + tol))
    r = len(best)
    theta = (y + 0.5) / (r + 1.0)
    R99 = max(1.0, math.log(1 - 0.99) / math.log(1 - theta)) if theta < 1 else 1.0
    return dict(hits=y, runs=r, theta=theta, tts99_s=tau_run * R99)


def batched_jobs(da, instances, n_inst=512, R=64, T=10_000, keep_Q=False):
    """The batched workload's items: n_inst SK instances, N uniform in {64, ..., 1024}, even items
    bimodal (int8, beta linear 0.05 -> 3, offset 1), odd items Gaussian (fp32, beta linear 0.1 -> 10,
    recompute every 1024), item i annealed with seed i.  Returns (jobs, [(bimodal, N)])."""
    rng = np.random.default_rng(1234)
    sizes = rng.choice([64, 128, 256, 512, 1024], n_inst)
    jobs, meta = [], []
    for i, N in enumerate(sizes):
        bim = i % 2 == 0
        q = instances.sk_bimodal(int(N), 1000 + i) if bim else instances.sk_gaussian(int(N), 1000 + i)
        beta = instances.beta_linear(0.05, 3.0, T) if bim else instances.beta_linear(0.1, 10.0, T)
        jobs.append(dict(ctx=da.da_create(q.Q), beta=beta, offset_inc=1.0 if bim else 0.0, replicas=R, seed=i,
                         recompute_every=0 if bim else 1024))
        if keep_Q:
            jobs[-1]["Q"] = q.Q
        meta.append((bim, int(N)))
    return jobs, meta


def run_batched(da, instances, n_inst=512, R=64, T=10_000, plain_per_class=2):
    """Batched launch: n_inst fully connected instances, N uniform in {64..1024}, half bimodal (int8),
    half Gaussian (fp32, exact recompute every 1024 steps), R replicas each, one persistent CUDA-graph
    launch.  Compared with the plain one-launch-per-step form run by itself, instance after instance,
    on a sample of the same instances (plain_per_class per coupling type and size) for the full T
    steps with the same schedules and seeds: trials/s of both, and TTS99 of both at the hit rate each
    measures against the instance's best energy over the runs of both forms."""
    jobs, meta = batched_jobs(da, instances, n_inst, R, T)
    da.da_batch_anneal(jobs[:8])                      # warm-up
    outs, el = da.da_batch_anneal(jobs)               # (the tuner probes each class before the graph runs)
    config = da.da_batch_describe()
    trials = sum(R * T * N for _, N in meta)
    tau_b = el / (n_inst * R)
    # the plain form itself on a sample of the instances, full length
    sample = []
    for cls in sorted(set(meta)):
        sample += [i for i, m in enumerate(meta) if m == cls][:plain_per_class]
    j0 = jobs[sample[0]]
    da.da_anneal_plain(j0["ctx"], j0["beta"][:64], j0["offset_inc"], R, 0)   # warm-up
    p_time, p_trials, b_trials, rows = 0.0, 0, 0, []
    for i in sample:
        j = jobs[i]
        rp = da.da_anneal_plain(j["ctx"], j["beta"], j["offset_inc"], R, j["seed"])
        p_time += rp["elapsed_s"]
        p_trials += R * T * meta[i][1]
        b_trials += R * T * meta[i][1]
        E_ref = float(min(outs[i]["best_E"].min(), rp["best_E"].min()))
        tb = _hits_tts(outs[i]["best_E"], E_ref, tau_b)
        tp = _hits_tts(rp["best_E"], E_ref, rp["elapsed_s"] / R)
        rows.append((meta[i], tb, tp))
    plain_value = p_trials / p_time
    tts_b = [r[1]["tts99_s"] for r in rows]
    tts_p = [r[2]["tts99_s"] for r in rows]
    return {"workload": f"{n_inst} SK instances, N in {{64,128,256,512,1024}}, half bimodal int8 / half "
                        f"Gaussian fp32, {R} replicas, {T} steps, one persistent CUDA-graph launch",
            "value": trials / el, "unit": UNIT, "seconds": el, "configuration": config,
            "plain_gpu": {"value": plain_value, "unit": UNIT, "instances": len(sample),
                          "basis": f"the plain form run by itself on {len(sample)} of the instances "
                                   f"({plain_per_class} per coupling type and size), full {T} steps, same seeds"},
            "speedup_vs_plain": (trials / el) / plain_value,
            "tts99_median_s": float(np.median(tts_b)), "tts99_median_plain_s": float(np.median(tts_p)),
            "tts99_speedup_median": float(np.median(np.array(tts_p) / np.array(tts_b))),
            "hit_fraction_mean": {"batched": float(np.mean([r[1]["hits"] / r[1]["runs"] for r in rows])),
                                  "plain": float(np.mean([r[2]["hits"] / r[2]["runs"] for r in rows]))},
            "tts99_basis": "sampled instances; reference = best energy over the runs of both forms; "
                           "theta per form from its own hits (Jeffreys); tau = batched graph time / all runs, "
                           "plain time / R"}


def run_ptda(da, instances, L=32, K=32, sweeps=100):
    """PTDA: SK bimodal N = 512, K = 32 geometric betas in 0.2-5.0, exchange after every sweep."""
    q = instances.sk_bimodal(512, 77)
    betas = instances.beta_geometric(0.2, 5.0, K)
    ctx = da.da_create(q.Q)
    da.da_pt(ctx, betas, 2, 2, 0)
    r = da.da_pt(ctx, betas, sweeps, L, 1)
    trials = L * K * sweeps * q.N * q.N
    acc = r["swaps"].sum(axis=0) / (L * sweeps)
    # the adaptive ladder (ends fixed, gaps moved towards equal exchange rates) over the first
    # half of the sweeps; acceptance measured over the second half
    ra = da.da_pt(ctx, betas, sweeps, L, 1, swap_trace=True, adapt_every=5, adapt_sweeps=sweeps // 2)
    acc_a = ra["swap_trace"][:, sweeps // 2:, :].mean(axis=(0, 1))
    return {"workload": f"SK bimodal N=512, {K} geometric betas 0.2-5.0, {L} ladders, {sweeps} sweeps, "
                        "device-side exchange after every sweep",
            "value": trials / r["elapsed_s"], "unit": UNIT, "seconds": r["elapsed_s"],
            "exchange_acceptance_min": float(acc.min()), "exchange_acceptance_mean": float(acc.mean()),
            "best_E": float(r["best_E"].min()),
            "adaptive": {"value": trials / ra["elapsed_s"], "unit": UNIT,
                         "basis": "ladder adapted every 5 sweeps over the first half, rates over the second",
                         "exchange_acceptance_min": float(acc_a.min()),
                         "exchange_acceptance_max": float(acc_a.max()),
                         "best_E": float(ra["best_E"].min())}}


# DA temperatures (T_h, T_l) per density of the Erdos-Renyi study (appendix table of the
# density experiment), in the units of the Ising Hamiltonian.
DENSITY_TEMPS = {0.1: (20, 2.0), 0.2: (50, 2.0), 0.3: (60, 2.0), 0.4: (65, 2.5), 0.5: (75, 3.0),
                 0.6: (75, 3.0), 0.7: (60, 3.5), 0.8: (65, 3.5), 0.9: (70, 4.0)}


def run_density(da, instances, per_density=8, R=100, T=100_000):
    """Density sweep: Erdos-Renyi graphs with bimodal couplings, N = 1024, zero biases, nine
    densities 10..90 %, 100 runs per instance from x = 0, beta linear 1/T_h -> 1/T_l (the
    study's temperatures), offset off; one batched launch per density.  The step's cost does
    not depend on the density (every row of W is dense in HBM), which the per-density
    throughputs show; TTS99 per instance against the best energy over its runs."""
    out = {}
    N = 1024
    for d, (Th, Tl) in DENSITY_TEMPS.items():
        beta = instances.beta_linear(1.0 / Th, 1.0 / Tl, T)
        jobs = []
        for k in range(per_density):
            q = instances.erdos_renyi_bimodal(N, d, k)
            jobs.append(dict(ctx=da.da_create(q.Q), beta=beta, offset_inc=0.0, replicas=R, seed=k,
                             recompute_every=0))
        da.da_batch_anneal(jobs[:1])
        outs, el = da.da_batch_anneal(jobs)
        tau = el / (per_density * R)
        tts = [_tts_from_best(o["best_E"], tau) for o in outs]
        # Algorithm 3: bootstrap distribution of the median TTS over the instances
        boot = da.da_tts_bootstrap([t["hits"] for t in tts], [t["runs"] for t in tts], tau, 50, 2000, 0)
        p5, p95 = da.da_percentiles(boot, [5, 95])
        out[f"{int(round(d * 100))}%"] = {
            "value": per_density * R * T * N / el, "unit": UNIT, "seconds": el,
            "tts99_median_s": float(np.median([t["tts99_s"] for t in tts])),
            "tts50_bootstrap_s": {"mean": float(boot.mean()), "p5": float(p5), "p95": float(p95)},
            "hit_fraction_mean": float(np.mean([t["hits"] / t["runs"] for t in tts]))}
    return {"workload": f"Erdos-Renyi bimodal N={N}, densities 10..90 %, {per_density} instances x {R} runs "
                        f"per density, {T} steps, beta linear 1/T_h -> 1/T_l per density, offset off",
            "per_density": out}


def run_fixed_point(da, instances, R=1024, T=200_000):
    """The DA's fixed-point precision against fp32 on the headline workload: the SK-Gaussian
    instance scaled to 16-bit couplers / 26-bit biases and rounded (da_quantize), annealed as a
    DA_INT16 context with beta / scale; best states of both evaluated exactly in the original
    fp32 problem."""
    q = instances.sk_gaussian(C3["N"], C3["instance_seed"])
    beta = instances.beta_linear(C3["beta0"], C3["beta1"], T)
    ctx_f = da.da_create(q.Q)
    rf = da.da_anneal(ctx_f, beta, C3["inc"], R, 11, recompute_every=C3["recompute_every"])
    Qi, scale = da.da_quantize(q.Q)
    ctx_i = da.da_create(Qi, da.DA_INT16)
    ri = da.da_anneal(ctx_i, (beta / scale).astype(np.float32), C3["inc"], R, 11)
    Ei = da.da_energy(ctx_f, ri["best_x"])
    Ef = rf["best_E"]
    Eref = float(min(Ef.min(), Ei.min()))
    tol = 1e-6 * abs(Eref)
    return {"workload": f"SK-Gaussian N={C3['N']}, {R} replicas, {T} steps, beta linear "
                        f"{C3['beta0']} -> {C3['beta1']}; fp32 vs 16-bit couplers (scale {scale:.6g})",
            "value": R * T * C3["N"] / ri["elapsed_s"], "unit": UNIT, "fp32_value": R * T * C3["N"] / rf["elapsed_s"],
            "best_E_mean": {"fp32": float(Ef.mean()), "int16": float(Ei.mean())},
            "best_E_min": {"fp32": float(Ef.min()), "int16": float(Ei.min())},
            "hits_of_common_best": {"fp32": int((Ef <= Eref + tol).sum()), "int16": int((Ei <= Eref + tol).sum())},
            "relative_gap_of_means": float((Ei.mean() - Ef.mean()) / abs(Ef.mean()))}


def _serve_stream(da, pool, betas, picks, gaps, R, T, budget, resident_max_n=0):
    """Submit requests pool[picks[k]] at the inter-arrival gaps, wait for all; per-request results."""
    srv = da.Server(budget, 1024)
    srv.resident(resident_max_n)
    warm = da.da_submit(srv, pool[0].Q, betas[pool[0].bimodal][:100], 0.0, 4, 0)
    da.da_poll(warm, 60_000_000)
    n_req = len(picks)
    reqs = [None] * n_req
    t0 = time.perf_counter()

    def feed():
        t = t0
        for k in range(n_req):
            t += gaps[k]
            d = t - time.perf_counter()
            if d > 0:
                time.sleep(d)
            q = pool[picks[k]]
            reqs[k] = da.da_submit(srv, q.Q, betas[q.bimodal], 1.0 if q.bimodal else 0.0, R, k,
                                   0 if q.bimodal else 1024)

    th = threading.Thread(target=feed)
    th.start()
    th.join()
    res = [da.da_poll(reqs[k], 600_000_000) for k in range(n_req)]
    t1 = time.perf_counter()
    stats = srv.stats()
    srv.close()
    return res, t1 - t0, stats


def served_pool(instances, T=50_000, rng=None):
    """The served workload's instances: 24 SK QUBOs with N log-uniform in [256, 8192], even ones
    bimodal (int8; beta linear 0.05 -> 3, offset 1), odd ones Gaussian (fp32; beta linear 0.1 -> 10,
    recompute every 1024).  Returns (pool, {bimodal: beta schedule})."""
    rng = np.random.default_rng(99) if rng is None else rng
    pool = []
    for i in range(24):
        N = int(round(np.exp(rng.uniform(np.log(256), np.log(8192)))))
        bim = i % 2 == 0
        pool.append(instances.sk_bimodal(N, 3000 + i) if bim else instances.sk_gaussian(N, 3000 + i))
    betas = {True: instances.beta_linear(0.05, 3.0, T), False: instances.beta_linear(0.1, 10.0, T)}
    return pool, betas


def run_served(da, instances, n_req=64, rate=200.0, R=32, T=50_000, budget=120 << 30, sustained_req=512,
               sustained_rate=40.0, plain_max=6, resident_max_n=0):
    """Serving: Poisson arrivals (mean `rate` req/s) of fully connected QUBOs, N log-uniform in
    [256, 8192], half bimodal / half Gaussian, R replicas, T steps, HBM budget 120 GB.  Beside the
    burst at `rate`, a longer stream at a rate the GPU sustains, and the plain one-launch-per-step
    form on the requests it can take (N <= 1024), run one after another with the same seeds:
    trials/s and per-request TTS99 of both forms against the best energy of both."""
    rng = np.random.default_rng(99)
    pool, betas = served_pool(instances, T, rng)
    picks = rng.integers(0, len(pool), n_req)
    gaps = rng.exponential(1.0 / rate, n_req)
    res, makespan, stats = _serve_stream(da, pool, betas, picks, gaps, R, T, budget, resident_max_n)
    trials = sum(R * T * pool[i].N for i in picks)
    lat = np.array([o["latency_s"] for o in res])
    out = {"workload": f"{n_req} requests, Poisson {rate:.0f} req/s, N log-uniform 256-8192 (pool of 24 "
                       f"instances), half bimodal / half Gaussian, {R} replicas, {T} steps, HBM budget "
                       f"{budget >> 30} GB",
           "value": trials / makespan, "unit": UNIT, "makespan_s": makespan,
           "p50_latency_s": float(np.percentile(lat, 50)), "p99_latency_s": float(np.percentile(lat, 99)),
           "mean_latency_s": float(lat.mean()), "kernel_launches": stats["kernel_launches"],
           "resident_max_n": resident_max_n}
    if sustained_req < 1:
        return out
    # a longer stream at a rate the GPU sustains (the burst above is beyond one GPU's throughput, so
    # its latencies are mostly queueing)
    picks2 = rng.integers(0, len(pool), sustained_req)
    gaps2 = rng.exponential(1.0 / sustained_rate, sustained_req)
    res2, makespan2, _ = _serve_stream(da, pool, betas, picks2, gaps2, R, T, budget, resident_max_n)
    lat2 = np.array([o["latency_s"] for o in res2])
    out["sustained"] = {"requests": sustained_req, "rate_req_s": sustained_rate,
                        "value": sum(R * T * pool[i].N for i in picks2) / makespan2, "unit": UNIT,
                        "makespan_s": makespan2, "p50_latency_s": float(np.percentile(lat2, 50)),
                        "p99_latency_s": float(np.percentile(lat2, 99))}
    # the plain form on requests of the sustained stream with at most 1024 variables (its limit), one
    # after another, same instance, schedule and seed as the request
    small, seen = [], set()
    for k, i in enumerate(picks2):
        if pool[i].N <= 1024 and i not in seen:
            small.append((k, i))
            seen.add(i)
    small = small[:plain_max]
    if small:
        q0 = pool[small[0][1]]
        c0 = da.da_create(q0.Q)
        da.da_anneal_plain(c0, betas[q0.bimodal][:64], 0.0, R, 0)      # warm-up
        da.da_destroy(c0)
        p_time, p_trials, tts_s, tts_p = 0.0, 0, [], []
        for k, i in small:
            q = pool[i]
            ctx = da.da_create(q.Q)
            rp = da.da_anneal_plain(ctx, betas[q.bimodal], 1.0 if q.bimodal else 0.0, R, k)
            da.da_destroy(ctx)
            p_time += rp["elapsed_s"]
            p_trials += R * T * q.N
            E_ref = float(min(res2[k]["best_E"].min(), rp["best_E"].min()))
            tts_s.append(_hits_tts(res2[k]["best_E"], E_ref, lat2[k] / R)["tts99_s"])
            tts_p.append(_hits_tts(rp["best_E"], E_ref, rp["elapsed_s"] / R)["tts99_s"])
        out["plain_gpu"] = {"value": p_trials / p_time, "unit": UNIT, "requests": len(small),
                            "basis": f"the plain form on {len(small)} requests of the sustained stream with "
                                     "N <= 1024, one after another, same instances, schedules and seeds"}
        out["tts99_median_s"] = float(np.median(tts_s))
        out["tts99_median_plain_s"] = float(np.median(tts_p))
        out["tts99_basis"] = ("requests of the sustained stream; reference = best energy over the runs of both "
                              "forms; tau = request latency / R (served, submit to result, including queueing) "
                              "and device time / R (plain, run alone)")
    return out


def run_configs(da, instances):
    """The two smaller workloads of the target, each annealed once by the library and once by the
    plain one-launch-per-step form (same schedule and seeds): trials/s and TTS99 of both at the hit
    rate each measures against the best energy over the runs of both.
      sk_bimodal_n64:   SK bimodal N = 64, 64 replicas, 1e4 steps, beta linear 0.05 -> 3, offset 1;
      lattice2d_l32:    2D Gaussian spin glass on a 32 x 32 torus (N = 1024, kept dense), 128
                        replicas, 1e5 steps, beta geometric 0.1 -> 5, offset 0.5."""
    out = {}
    cases = [("sk_bimodal_n64", instances.sk_bimodal(64, 0), instances.beta_linear(0.05, 3.0, 10_000), 1.0, 64, 0),
             ("lattice2d_l32", instances.lattice2d(32, 0, True), instances.beta_geometric(0.1, 5.0, 100_000), 0.5,
              128, 1024)]
    for name, q, beta, inc, R, P in cases:
        ctx = da.da_create(q.Q)
        da.da_anneal(ctx, beta[:256], inc, R, 0, recompute_every=P)           # warm-up
        r = da.da_anneal(ctx, beta, inc, R, 0, recompute_every=P)
        da.da_anneal_plain(ctx, beta[:64], inc, R, 0)                          # warm-up
        rp = da.da_anneal_plain(ctx, beta, inc, R, 0)
        trials = R * beta.size * q.N
        E_ref = float(min(r["best_E"].min(), rp["best_E"].min()))
        t_lib = _hits_tts(r["best_E"], E_ref, r["elapsed_s"] / R)
        t_plain = _hits_tts(rp["best_E"], E_ref, rp["elapsed_s"] / R)
        out[name] = {"value": trials / r["elapsed_s"], "unit": UNIT, "seconds": r["elapsed_s"],
                     "tts99_s": t_lib["tts99_s"], "hits": t_lib["hits"], "runs": t_lib["runs"],
                     "mean_best_E": float(np.mean(r["best_E"])),
                     "plain_gpu": {"value": trials / rp["elapsed_s"], "unit": UNIT, "tts99_s": t_plain["tts99_s"],
                                   "hits": t_plain["hits"], "mean_best_E": float(np.mean(rp["best_E"]))},
                     "E_ref": E_ref}
        da.da_destroy(ctx)
    return out


def profile_case(da, instances, case):
    """Small runs of the library's other kernels for ncu captures: `batched` (a two-class batched
    launch: fp32 N = 1024 from L2, int8 N = 64 staged), `ptda` (SK bimodal N = 512, 32 betas,
    20 sweeps), `plain` (the plain form, 200 steps of the headline workload), `g8` (fp32
    N = 8192, 32 replicas: the 8-warp step kernel)."""
    if case == "batched":
        T = 2048
        jobs = []
        for i in range(64):
            q = instances.sk_gaussian(1024, 500 + i)
            jobs.append(dict(ctx=da.da_create(q.Q), beta=instances.beta_linear(0.1, 10.0, T), offset_inc=0.0,
                             replicas=64, seed=i, recompute_every=1024))
        for i in range(128):
            q = instances.sk_bimodal(64, 700 + i)
            jobs.append(dict(ctx=da.da_create(q.Q), beta=instances.beta_linear(0.05, 3.0, T), offset_inc=1.0,
                             replicas=64, seed=i))
        da.da_batch_force(1, 16)
        _, el = da.da_batch_anneal(jobs)
        da.da_batch_force(-1, 0)
        return {"seconds": el, "config": da.da_batch_describe()}
    if case == "ptda":
        ctx = da.da_create(instances.sk_bimodal(512, 77).Q)
        return {"seconds": da.da_pt(ctx, instances.beta_geometric(0.2, 5.0, 32), 20, 32, 1)["elapsed_s"]}
    if case == "plain":
        ctx = da.da_create(instances.sk_gaussian(1024, 0).Q)
        beta = instances.beta_linear(0.1, 10.0, 200_000)[100_000:100_200]
        return {"seconds": da.da_anneal_plain(ctx, beta, 0.0, 1024, 0)["elapsed_s"]}
    if case == "g8":
        ctx = da.da_create(instances.sk_gaussian(8192, 3).Q)
        r = da.da_anneal(ctx, instances.beta_linear(0.1, 10.0, 4096), 0.0, 32, 0, recompute_every=1024)
        return {"seconds": r["elapsed_s"]}
    raise ValueError(case)


def cpu_baseline(sample_R=None, sample_T=32768):
    """The oracle, as it stands, on the host cores over a bounded sample of the workload."""
    import oracle
    from paper_1806_08815_gb300 import instances
    cores = os.cpu_count() or 1
    R = sample_R or 2 * cores
    q = instances.sk_gaussian(C3["N"], C3["instance_seed"])
    beta = instances.beta_linear(C3["beta0"], C3["beta1"], C3["steps"])[:sample_T]
    t0 = time.perf_counter()
    oracle.da_anneal(q.Q, beta, R=R, seed=C3["seed"], inc=C3["inc"], recompute_every=C3["recompute_every"],
                     nthreads=cores)
    dt = time.perf_counter() - t0
    trials = R * sample_T * C3["N"]
    return {"value": trials / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{R} replicas x first {sample_T} of the 2e5 steps (N=1024 fp32, recompute every 1024), "
                      f"{dt:.1f} s wall"}


def rank_seed(rank: int) -> int:
    """Replicas only: rank r anneals its own replica set with seed C3 seed + r (no exchange)."""
    return C3["seed"] + rank


def max_over_ranks(t: float, dist, device) -> float:
    """The slowest rank's time (the job's time); identity without a process group."""
    if dist is None:
        return t
    import torch
    tt = torch.tensor([t], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def _free_port() -> int:
    import socket
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def spawn_ranks(n: int) -> int:
    """--gpus N without a launcher: start N ranks of this script (one process per GPU) with
    torch.distributed.run on this node, and return their exit status."""
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", f"--nproc-per-node={n}",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()),
           os.path.abspath(__file__), *sys.argv[1:]]
    return subprocess.call(cmd)


def run_reference(args, rank, world):
    if rank != 0:
        return
    res = []
    for i in range(args.warmup + args.steps):
        cb = cpu_baseline(sample_T=1024 if i < args.warmup else 4096)
        if i >= args.warmup:
            res.append(cb)
    v = statistics.median(r["value"] for r in res)
    cb = res[-1]
    cb["value"] = v
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "sk_gaussian_N1024_R1024_T2e5 (bounded sample on host cores)"},
            "cpu_baseline": cb, "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--steps-per-anneal", type=int, default=C3["steps"])
    ap.add_argument("--plain-steps", type=int, default=10_000,
                    help="steps of the plain one-launch-per-step GPU form timed beside (0 = skip)")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the batched, PTDA and served workloads reported beside the headline")
    ap.add_argument("--kernel-case", action="store_true",
                    help="run two 2048-step anneals from the middle of the schedule and exit (for ncu captures)")
    ap.add_argument("--profile-case", choices=["batched", "ptda", "plain", "g8"],
                    help="run one small case of another kernel and exit (for ncu captures)")
    ap.add_argument("--served-case", action="store_true",
                    help="run the served workload once, print its figures and exit (for ncu launch lists)")
    args = ap.parse_args()

    if args.gpus > 1 and "WORLD_SIZE" not in os.environ:
        sys.exit(spawn_ranks(args.gpus))
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world != args.gpus and rank == 0:
        print(f"bench.py: --gpus {args.gpus} but the launcher started {world} ranks; timing {world}",
              file=sys.stderr)
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_1806_08815_gb300 import binding as da
    from paper_1806_08815_gb300 import instances
    da.lib()

    dev = torch.device("cuda", local)
    if args.profile_case:
        print(json.dumps({"profile_case": args.profile_case, **profile_case(da, instances, args.profile_case)}))
        return
    if args.served_case:
        r = run_served(da, instances, sustained_req=0)
        print(json.dumps({"served_case": r["workload"], **{k: v for k, v in r.items() if k != "workload"}}))
        return
    N, R, T, P = C3["N"], C3["replicas"], args.steps_per_anneal, C3["recompute_every"]
    q = instances.sk_gaussian(N, C3["instance_seed"])
    beta = instances.beta_linear(C3["beta0"], C3["beta1"], T)
    seed = rank_seed(rank)              # weak scaling: each rank anneals its own 1024 replicas
    ctx = da.da_create(q.Q)
    # the autotuner's launch shape for this instance class (not for the profiling case, whose
    # launch list must hold only the anneal's own launches)
    shape = None if args.kernel_case else da.da_tune_shape(ctx, R)
    beta_dev = torch.from_numpy(beta).to(dev)
    Wd = da.da_words(N)
    out = dict(final_E=torch.zeros(R, dtype=torch.float64, device=dev),
               best_E=torch.zeros(R, dtype=torch.float64, device=dev),
               best_x=torch.zeros((R, Wd), dtype=torch.int32, device=dev),
               max_drift=torch.zeros(R, dtype=torch.float64, device=dev),
               flips=torch.zeros(R, dtype=torch.int64, device=dev))
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # 256 MB > 129 MB L2

    def one_step():
        da.da_anneal_async(ctx, beta_dev, T, C3["inc"], R, seed, P, out, stream)

    if args.kernel_case:
        mid = torch.from_numpy(instances.beta_linear(C3["beta0"], C3["beta1"], C3["steps"])[100_000:102_048]).to(dev)
        for _ in range(2):
            da.da_anneal_async(ctx, mid, mid.numel(), C3["inc"], R, seed, P, out, stream)
            stream.synchronize()
        print(json.dumps({"kernel_case": "sk_gaussian_N1024_R1024 steps 100000..102047", "ok": True}))
        return

    for _ in range(args.warmup):
        one_step()
    stream.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    times = []
    da.da_profile_enable(ctx, True)
    for _ in range(args.steps):
        with torch.cuda.stream(stream):
            flush.fill_(1.0)
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        one_step()
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1) / 1e3)
    launches, step_ms = da.da_profile_read(ctx)
    da.da_profile_enable(ctx, False)
    clk = clocks.stop()
    t_step = max_over_ranks(float(np.mean(times)), dist, dev)
    trials = R * T * N
    value = world * trials / t_step

    best_E = out["best_E"].cpu().numpy()
    drift = out["max_drift"].cpu().numpy()
    tts = tts99(best_E, t_step / R)

    # end to end through the blocking host API: Q and beta uploaded, results read back
    e2e_times = []
    res_bytes = 0
    for _ in range(max(1, min(args.steps, 2))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        c2 = da.da_create(q.Q)
        r2 = da.da_anneal(c2, beta, C3["inc"], R, seed, recompute_every=P)
        da.da_destroy(c2)
        e2e_times.append(time.perf_counter() - t0)
        res_bytes = sum(r2[k].nbytes for k in ("final_E", "best_E", "final_x", "best_x", "max_drift", "flips"))
    e2e_v = world * trials / float(np.mean(e2e_times))

    # the plain one-launch-per-step GPU form on a sample of the same workload
    plain = None
    if rank == 0 and args.plain_steps > 0:
        Tp = min(args.plain_steps, T)
        da.da_anneal_plain(ctx, beta[:64], C3["inc"], R, seed)            # warm-up
        torch.cuda.synchronize()
        rp = da.da_anneal_plain(ctx, beta[:Tp], C3["inc"], R, seed)
        plain = {"value": R * Tp * N / rp["elapsed_s"], "unit": UNIT,
                 "sample": f"first {Tp} steps of the schedule, {R} replicas, one launch per step",
                 "speedup_of_value": value / (world * R * Tp * N / rp["elapsed_s"])}

    # rooflines of the step kernel: the issue slots it is bound by, and its bytes.  Algorithmic
    # bytes per replica-step: one fp32 row of W (4N) for every applied flip; the nominal figure
    # adds the replica state (fields 4N + state bits N/8) that stays in registers
    peaks, peak_src = load_peaks()
    hbm = hbm_peak(peaks)
    bw = read_bandwidths(da, dev)
    per_launch_steps = min(P, T)
    replica_steps = R * per_launch_steps
    avg_launch_s = (step_ms / 1e3) / max(launches, 1)
    flip_frac = float(out["flips"].sum().item()) / (R * T)
    algo_bytes = replica_steps * flip_frac * 4 * N
    nominal_bytes = replica_steps * (4 * N + 4 * N + N // 8)
    algo_gbs = algo_bytes / avg_launch_s / 1e9
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    sm_ghz = (clk["sm_mhz"] if clk and clk.get("sm_mhz") else 2070.0) / 1e3
    roofline = issue_roofline(replica_steps, avg_launch_s, sms, sm_ghz)
    roofline["kernel"] = "step_kernel_g1<float,V=32>"
    roofline["memory"] = {
        "algorithmic_bytes_per_launch": algo_bytes, "flips_per_replica_step": flip_frac,
        "achieved_gbs": algo_gbs,
        "l2_w_sized_gbs": bw["w_sized_4mb"], "frac_l2_w_sized": algo_gbs / bw["w_sized_4mb"],
        "l2_peak_gbs": bw["l2_64mb"], "frac_l2_peak": algo_gbs / bw["l2_64mb"],
        "hbm_gbs": hbm, "frac_hbm": algo_gbs / hbm, "hbm_source": peak_src,
        "nominal_bytes_per_launch": nominal_bytes, "nominal_gbs": nominal_bytes / avg_launch_s / 1e9,
        "nominal_frac_hbm": nominal_bytes / avg_launch_s / 1e9 / hbm,
        "basis": "algorithmic: one 4N-byte row of W per applied flip (replica state stays in registers); "
                 "nominal: row + fields + state bits every replica-step; L2 bandwidths measured here with "
                 "16-byte L1-bypassing reads (da_diag_read_bandwidth), HBM from the measured copy peak"}
    n_step_launches = math.ceil(T / P)
    n_recompute = T // P
    # init, step launches, 2 per recompute (tensor-core recompute with the states expanded in the kernel,
    # energy sum), the same 2 for the final evaluation, best-state fixup, finalize
    gpu_launches = 1 + n_step_launches + 2 * n_recompute + 2 + 1 + 1

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_step * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "sk_gaussian_N1024_R1024_T2e5", "N": N, "replicas": R, "steps_per_anneal": T,
                   "recompute_every": P, "beta": f"linear {C3['beta0']} -> {C3['beta1']}",
                   "offset_inc": C3["inc"], "parallelism": f"replicas x{world}", "launch_shape": shape,
                   "l2": "flushed (256 MB write) before every timed step"},
        "e2e": {"value": e2e_v, "unit": UNIT, "h2d_bytes_per_step": int(q.Q.nbytes + beta.nbytes),
                "d2h_bytes_per_step": int(res_bytes)},
        "gpu_launches": gpu_launches * args.steps,
        "roofline": roofline,
        "step_kernel": {"launches": launches, "avg_launch_ms": avg_launch_s * 1e3,
                        "share_of_step": (step_ms / 1e3) / (t_step * args.steps)},
        "roofline_recompute": recompute_roofline(peaks, peak_src, N, R, n_recompute,
                                                 t_step - (step_ms / 1e3) / args.steps),
        "tts99": tts,
        "plain_gpu": plain,
        "max_fp32_drift": float(drift.max()),
    }
    if clk:
        line["clocks"] = clk
    if rank == 0 and not args.no_extras:
        line["batched"] = run_batched(da, instances)
        line["ptda"] = run_ptda(da, instances)
        line["served"] = run_served(da, instances)
        line["density"] = run_density(da, instances)
        line["fixed_point"] = run_fixed_point(da, instances)
        line["configs"] = run_configs(da, instances)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
