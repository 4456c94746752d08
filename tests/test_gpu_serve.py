"""The request loop (da_server_create / da_submit / da_poll): every request's
result is the same alone and in the mix, whatever else is on the GPU.

Requests of mixed sizes and coupling types are submitted together (each runs
as chunked launches on a stream of its own, concurrently with the others, in
the launch shape the server picks for the load); each must equal da_anneal on
the same instance, schedule and seed, bit for bit.  A budget that admits one request at a time must give the same
results, and a request that can never fit is refused."""
import concurrent.futures

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def da():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1806_08815_gb300 import binding
    return binding


def _jobs(inst):
    rng = np.random.default_rng(7)
    jobs = []
    for n, N in enumerate([64, 300, 1024, 96, 1500, 512, 2048]):
        q = inst.sk_bimodal(N, n) if n % 2 == 0 else inst.sk_gaussian(N, n)
        T = int(rng.integers(300, 1200))
        jobs.append(dict(Q=q.Q, beta=inst.beta_linear(0.1, 4.0, T), inc=0.5 if n % 3 == 0 else 0.0,
                         R=int(rng.integers(2, 24)), seed=500 + n, P=0 if q.bimodal else 256))
    return jobs


def _alone(da, j):
    ctx = da.da_create(j["Q"])
    return da.da_anneal(ctx, j["beta"], j["inc"], j["R"], j["seed"], recompute_every=j["P"])


def _same(a, b):
    for k in ("final_x", "best_x", "flips", "final_E", "best_E", "max_drift"):
        assert np.array_equal(a[k], b[k]), k


def test_results_same_alone_and_in_the_mix(da):
    from paper_1806_08815_gb300 import instances as inst
    jobs = _jobs(inst)
    srv = da.Server(8 << 30, 64)
    reqs = [da.da_submit(srv, j["Q"], j["beta"], j["inc"], j["R"], j["seed"], j["P"]) for j in jobs]
    outs = [da.da_poll(r, 60_000_000) for r in reqs]
    stats = srv.stats()
    srv.close()
    assert stats["completed"] == len(jobs) and stats["kernel_launches"] >= 1
    for j, o in zip(jobs, outs):
        assert o is not None and o["latency_s"] > 0
        _same(o, _alone(da, j))


def test_tight_budget_queues_and_gives_the_same_results(da):
    from paper_1806_08815_gb300 import instances as inst
    jobs = _jobs(inst)[:4]
    srv = da.Server(64 << 20, 2)
    reqs = [da.da_submit(srv, j["Q"], j["beta"], j["inc"], j["R"], j["seed"], j["P"]) for j in jobs]
    outs = [da.da_poll(r, 60_000_000) for r in reqs]
    srv.close()
    for j, o in zip(jobs, outs):
        _same(o, _alone(da, j))


def test_request_over_budget_is_refused(da):
    from paper_1806_08815_gb300 import instances as inst
    q = inst.sk_gaussian(2048, 1)
    srv = da.Server(1 << 20, 4)
    with pytest.raises(da.DAError) as e:
        da.da_submit(srv, q.Q, inst.beta_linear(0.1, 1.0, 10), 0.0, 4, 0)
    assert e.value.status == 3
    srv.close()


def test_short_request_is_not_held_behind_a_long_one(da):
    """Requests run concurrently: a short request submitted while a long one
    runs finishes long before it (the long one leaves SMs free), and both
    results equal da_anneal."""
    from paper_1806_08815_gb300 import instances as inst
    long_q = inst.sk_gaussian(2048, 11)
    short_q = inst.sk_bimodal(64, 12)
    long_beta = inst.beta_linear(0.1, 4.0, 60_000)
    short_beta = inst.beta_linear(0.1, 4.0, 500)
    srv = da.Server(8 << 30, 8)
    warm = da.da_submit(srv, short_q.Q, short_beta, 0.5, 2, 1)
    da.da_poll(warm, 60_000_000)
    rl = da.da_submit(srv, long_q.Q, long_beta, 0.0, 16, 3, 1024)
    rs = da.da_submit(srv, short_q.Q, short_beta, 0.5, 4, 4)
    os_ = da.da_poll(rs, 60_000_000)
    ol = da.da_poll(rl, 120_000_000)
    srv.close()
    assert os_["latency_s"] < 0.5 * ol["latency_s"], (os_["latency_s"], ol["latency_s"])
    _same(os_, _alone(da, dict(Q=short_q.Q, beta=short_beta, inc=0.5, R=4, seed=4, P=0)))
    _same(ol, _alone(da, dict(Q=long_q.Q, beta=long_beta, inc=0.0, R=16, seed=3, P=1024)))


def test_degenerate_and_largest_requests(da):
    """N = 1, no steps, one replica, and the largest N of both coupling types
    through the request loop, each equal to da_anneal."""
    from paper_1806_08815_gb300 import instances as inst
    jobs = [dict(Q=np.array([[5]], np.int32), beta=inst.beta_linear(0.1, 2.0, 50), inc=1.0, R=1, seed=1, P=0),
            dict(Q=inst.sk_gaussian(33, 2).Q, beta=np.zeros(0, np.float32), inc=0.0, R=3, seed=2, P=16),
            dict(Q=inst.sk_bimodal(8192, 3).Q, beta=inst.beta_linear(0.1, 3.0, 300), inc=1.0, R=5, seed=3, P=0),
            dict(Q=inst.sk_gaussian(8192, 4).Q, beta=inst.beta_linear(0.1, 3.0, 300), inc=0.0, R=3, seed=4, P=128)]
    srv = da.Server(16 << 30, 8)
    reqs = [da.da_submit(srv, j["Q"], j["beta"], j["inc"], j["R"], j["seed"], j["P"]) for j in jobs]
    outs = [da.da_poll(r, 120_000_000) for r in reqs]
    srv.close()
    for j, o in zip(jobs, outs):
        _same(o, _alone(da, j))


def test_fixed_point_requests_in_the_mix(da):
    """DA_INT16 requests (the DA's 16-bit couplers: Gaussian instances scaled by da_quantize,
    beta divided by the scale) run in the request loop beside int8 and fp32 requests, and each
    equals da_anneal on a DA_INT16 context bit for bit."""
    from paper_1806_08815_gb300 import instances as inst
    jobs = []
    for n, N in enumerate([96, 700, 1300, 3000]):
        q = inst.sk_gaussian(N, 40 + n)
        Qi, scale = da.da_quantize(q.Q)
        beta = (inst.beta_linear(0.1, 6.0, 500 + 100 * n) / scale).astype(np.float32)
        jobs.append(dict(Q=Qi, beta=beta, inc=0.0 if n % 2 else 2000.0, R=5 + 3 * n, seed=70 + n))
    mix = _jobs(inst)[:3]
    srv = da.Server(8 << 30, 64)
    reqs = [da.da_submit(srv, j["Q"], j["beta"], j["inc"], j["R"], j["seed"], 0, dtype=da.DA_INT16) for j in jobs]
    reqs_mix = [da.da_submit(srv, j["Q"], j["beta"], j["inc"], j["R"], j["seed"], j["P"]) for j in mix]
    outs = [da.da_poll(r, 60_000_000) for r in reqs]
    outs_mix = [da.da_poll(r, 60_000_000) for r in reqs_mix]
    srv.close()
    for j, o in zip(jobs, outs):
        ctx = da.da_create(j["Q"], da.DA_INT16)
        ref = da.da_anneal(ctx, j["beta"], j["inc"], j["R"], j["seed"])
        _same(o, ref)
        assert np.all(o["max_drift"] == 0)
    for j, o in zip(mix, outs_mix):
        _same(o, _alone(da, j))


def test_resident_requests_equal_chunked_ones(da):
    """Requests of at most 1024 variables run resident (one launch for the whole anneal, replica
    state in registers, fp32 fields recomputed by each warp) beside larger chunked ones: every
    result equals da_anneal bit for bit; a cancelled resident request stops within 1024 steps."""
    import time
    from paper_1806_08815_gb300 import instances as inst
    jobs = _jobs(inst)
    srv = da.Server(8 << 30, 64)
    srv.resident(1024)
    reqs = [da.da_submit(srv, j["Q"], j["beta"], j["inc"], j["R"], j["seed"], j["P"]) for j in jobs]
    outs = [da.da_poll(r, 60_000_000) for r in reqs]
    for j, o in zip(jobs, outs):
        _same(o, _alone(da, j))
    q = inst.sk_bimodal(1024, 8)
    long_req = da.da_submit(srv, q.Q, np.full(3_000_000, 1.0, np.float32), 1.0, 32, 1)
    time.sleep(0.2)
    t0 = time.perf_counter()
    da.da_cancel(long_req)
    with pytest.raises(da.DAError) as e:
        da.da_poll(long_req, 60_000_000)
    assert e.value.status == 8 and time.perf_counter() - t0 < 1.5
    srv.close()


def test_full_size_served_requests_sampled_replicas(da):
    """The served workload at full size: its largest fp32 and int8 instances and two smaller
    ones (32 replicas, 5*10^4 steps, recompute every 1024 for fp32, HBM budget 120 GB) run
    together through the request loop; sampled replicas of the two largest are rerun alone by
    the oracle (final and best states, flips bit for bit; best energies exact for int8,
    within 1e-12 relative for fp32)."""
    import oracle
    from bench import served_pool
    from paper_1806_08815_gb300 import instances as inst
    pool, betas = served_pool(inst)
    big_f = max((i for i, q in enumerate(pool) if not q.bimodal), key=lambda i: pool[i].N)
    big_i = max((i for i, q in enumerate(pool) if q.bimodal), key=lambda i: pool[i].N)
    small = [i for i, q in enumerate(pool) if q.N <= 1024][:2]
    picks = [big_f, big_i] + small
    sampled = ((big_f, 5), (big_i, 20))

    def rerun(k):
        i, r = sampled[k]
        q = pool[i]
        return oracle.da_anneal(q.Q, betas[q.bimodal], R=1, seed=k, inc=1.0 if q.bimodal else 0.0,
                                replica_base=r, recompute_every=0 if q.bimodal else 1024)

    ex = concurrent.futures.ThreadPoolExecutor(2)      # the oracle's C calls run beside the GPU work
    refs = [ex.submit(rerun, k) for k in range(len(sampled))]
    srv = da.Server(120 << 30, 64)
    reqs = []
    for k, i in enumerate(picks):
        q = pool[i]
        reqs.append(da.da_submit(srv, q.Q, betas[q.bimodal], 1.0 if q.bimodal else 0.0, 32, k,
                                 0 if q.bimodal else 1024))
    outs = [da.da_poll(r, 600_000_000) for r in reqs]
    srv.close()
    for k, (i, r) in enumerate(sampled):
        q, o = pool[i], outs[k]
        ref = refs[k].result()
        assert np.array_equal(o["final_x"][r], ref["x_final"][0]), (q.N, r)
        assert np.array_equal(o["best_x"][r], ref["x_best"][0]), (q.N, r)
        assert o["flips"][r] == ref["flips"][0], (q.N, r)
        Eb = float(oracle.energy(q.Q, ref["x_best"])[0])
        if q.bimodal:
            assert o["best_E"][r] == Eb
        else:
            assert abs(o["best_E"][r] - Eb) <= 1e-12 * max(1.0, abs(Eb))
