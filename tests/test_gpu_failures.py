"""Error paths of the library under host-side failure injection, and request
cancellation (GPU).

Allocation failure is injected on the host (da_diag_fail_alloc: the library's
next device allocations fail as if the device were out of memory, without
being attempted), so no test here faults, hangs or exhausts the GPU.  Checked:
every failing call returns DA_ENOMEM, leaves no device allocation behind
(da_diag_live_allocations), and the context or server keeps working with
results identical to an undisturbed run.  Cancellation: a queued request leaves
the queue at once, a running one stops at its next step launch, and both give
their memory back to the server's budget.
"""
import time

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
    binding.lib()
    yield binding
    binding.da_diag_fail_alloc(0, 0)


def _live(da):
    return da.da_diag_live_allocations()


@pytest.mark.parametrize("kind", ["int8", "fp32"])
def test_create_fails_cleanly_at_every_allocation(da, kind):
    from paper_1806_08815_gb300 import instances
    q = instances.sk_bimodal(200, 1) if kind == "int8" else instances.sk_gaussian(200, 1)
    base = _live(da)
    k = 0
    while True:
        da.da_diag_fail_alloc(k, 1)
        try:
            ctx = da.da_create(q.Q)
        except da.DAError as e:
            assert e.status == 2, str(e)
            now = _live(da)
            assert now["count"] == base["count"] and now["bytes"] == base["bytes"], (k, now, base)
            k += 1
            assert k < 20
            continue
        da.da_diag_fail_alloc(0, 0)
        break
    assert k >= 3, "da_create makes at least W, diag and the copy of Q"
    # the context made after the failures works and equals a fresh one
    beta = instances.beta_linear(0.05, 3.0, 300)
    a = da.da_anneal(ctx, beta, 1.0 if kind == "int8" else 0.0, 8, 4, recompute_every=0 if kind == "int8" else 64)
    ctx2 = da.da_create(q.Q)
    b = da.da_anneal(ctx2, beta, 1.0 if kind == "int8" else 0.0, 8, 4, recompute_every=0 if kind == "int8" else 64)
    for key in ("final_E", "best_E", "final_x", "best_x", "flips"):
        assert np.array_equal(a[key], b[key]), key
    da.da_destroy(ctx)
    da.da_destroy(ctx2)
    now = _live(da)
    assert now["count"] == base["count"] and now["bytes"] == base["bytes"]


def test_anneal_workspace_failure_leaves_the_context_usable(da):
    from paper_1806_08815_gb300 import instances
    q = instances.sk_gaussian(96, 2)
    beta = instances.beta_linear(0.1, 6.0, 500)
    ctx = da.da_create(q.Q)
    before = _live(da)
    da.da_diag_fail_alloc(0, 1)
    with pytest.raises(da.DAError) as e:
        da.da_anneal(ctx, beta, 0.0, 16, 9, recompute_every=128)
    assert e.value.status == 2
    assert _live(da)["count"] == before["count"]
    da.da_diag_fail_alloc(0, 0)
    got = da.da_anneal(ctx, beta, 0.0, 16, 9, recompute_every=128)
    ctx2 = da.da_create(q.Q)
    ref = da.da_anneal(ctx2, beta, 0.0, 16, 9, recompute_every=128)
    for key in ("final_E", "best_E", "final_x", "best_x", "flips"):
        assert np.array_equal(got[key], ref[key]), key
    da.da_destroy(ctx)
    da.da_destroy(ctx2)


@pytest.mark.parametrize("after", [0, 1])
def test_server_keeps_serving_after_a_failed_admission(da, after):
    """after = 0: the request's buffers cannot be allocated; after = 1: its
    buffers are, the transient copy of Q is not (the buffers must be freed)."""
    from paper_1806_08815_gb300 import instances
    q1 = instances.sk_bimodal(300, 3)
    q2 = instances.sk_gaussian(200, 4)
    beta = instances.beta_linear(0.05, 3.0, 400)
    srv = da.Server(1 << 30, 8)
    base = _live(da)
    da.da_diag_fail_alloc(after, 1)
    bad = da.da_submit(srv, q1.Q, beta, 1.0, 8, 5)
    with pytest.raises(da.DAError) as e:
        da.da_poll(bad, 60_000_000)
    assert e.value.status == 2, str(e.value)
    da.da_diag_fail_alloc(0, 0)
    assert srv.stats()["bytes_in_use"] == 0
    good1 = da.da_submit(srv, q1.Q, beta, 1.0, 8, 5)
    good2 = da.da_submit(srv, q2.Q, beta, 0.0, 8, 6, 64)
    r1 = da.da_poll(good1, 60_000_000)
    r2 = da.da_poll(good2, 60_000_000)
    for qq, r, inc, seed, rec in ((q1, r1, 1.0, 5, 0), (q2, r2, 0.0, 6, 64)):
        ctx = da.da_create(qq.Q)
        ref = da.da_anneal(ctx, beta, inc, 8, seed, recompute_every=rec)
        for key in ("final_E", "best_E", "final_x", "best_x", "flips"):
            assert np.array_equal(r[key], ref[key]), key
        da.da_destroy(ctx)
    st = srv.stats()
    assert st["bytes_in_use"] == 0 and st["completed"] >= 2
    srv.close()
    now = _live(da)
    assert now["count"] == base["count"]


def test_budget_counts_the_transient_copy_of_q(da):
    """An fp32 request at N = 4096 holds W (64 MB) and, until its instance is
    built, the 64 MB copy of Q: a 100 MB budget can never admit it."""
    from paper_1806_08815_gb300 import instances
    q = instances.sk_gaussian(4096, 1)
    srv = da.Server(100 << 20, 4)
    with pytest.raises(da.DAError) as e:
        da.da_submit(srv, q.Q, instances.beta_linear(0.1, 1.0, 10), 0.0, 4, 0)
    assert e.value.status == 3
    srv.close()


def test_cancel_queued_and_running_requests(da):
    from paper_1806_08815_gb300 import instances
    q = instances.sk_bimodal(1024, 8)
    T_long = 3_000_000
    beta_long = np.full(T_long, 1.0, np.float32)
    srv = da.Server(8 << 30, 1)               # one slot: the second request waits in the queue
    long_req = da.da_submit(srv, q.Q, beta_long, 1.0, 32, 1)
    time.sleep(0.2)
    queued = da.da_submit(srv, q.Q, beta_long[:1000], 1.0, 8, 2)
    da.da_cancel(queued)
    with pytest.raises(da.DAError) as e:
        da.da_poll(queued, 0)
    assert e.value.status == 8
    t0 = time.perf_counter()
    da.da_cancel(long_req)
    with pytest.raises(da.DAError) as e:
        da.da_poll(long_req, 60_000_000)
    dt = time.perf_counter() - t0
    assert e.value.status == 8
    # 3e6 steps of 32 replicas take seconds; the cancelled request stops after the
    # launch that was running (16384 steps)
    assert dt < 1.5, dt
    deadline = time.time() + 10
    while srv.stats()["bytes_in_use"] != 0 and time.time() < deadline:
        time.sleep(0.01)
    assert srv.stats()["bytes_in_use"] == 0
    # the server goes on: a new request equals da_anneal
    beta = instances.beta_linear(0.05, 3.0, 500)
    r = da.da_poll(da.da_submit(srv, q.Q, beta, 1.0, 8, 3), 60_000_000)
    ctx = da.da_create(q.Q)
    ref = da.da_anneal(ctx, beta, 1.0, 8, 3)
    for key in ("final_E", "best_E", "final_x", "best_x", "flips"):
        assert np.array_equal(r[key], ref[key]), key
    da.da_destroy(ctx)
    # cancelling a finished request changes nothing
    done = da.da_submit(srv, q.Q, beta, 1.0, 8, 3)
    r2 = da.da_poll(done, 60_000_000)
    da.da_cancel(done)
    assert np.array_equal(r2["best_E"], ref["best_E"])
    srv.close()


def test_batched_launch_allocation_failure(da):
    """The batched launch's workspace cannot be allocated: DA_ENOMEM, nothing left behind, and
    the next launch gives each item its da_anneal results."""
    from paper_1806_08815_gb300 import instances
    q1, q2 = instances.sk_bimodal(100, 1), instances.sk_gaussian(300, 2)
    beta = instances.beta_linear(0.1, 3.0, 300)
    c1, c2 = da.da_create(q1.Q), da.da_create(q2.Q)
    jobs = [dict(ctx=c1, beta=beta, offset_inc=0.5, replicas=8, seed=3),
            dict(ctx=c2, beta=beta, offset_inc=0.0, replicas=5, seed=4, recompute_every=64)]
    base = _live(da)
    da.da_diag_fail_alloc(0, 1)
    with pytest.raises(da.DAError) as e:
        da.da_batch_anneal(jobs)
    assert e.value.status == 2
    now = _live(da)
    assert now["count"] == base["count"] and now["bytes"] == base["bytes"]
    da.da_diag_fail_alloc(0, 0)
    outs, _ = da.da_batch_anneal(jobs)
    for j, o in zip(jobs, outs):
        ref = da.da_anneal(j["ctx"], beta, j["offset_inc"], j["replicas"], j["seed"],
                           recompute_every=j.get("recompute_every", 0))
        for key in ("final_E", "best_E", "final_x", "best_x", "flips"):
            assert np.array_equal(o[key], ref[key]), key
    da.da_destroy(c1)
    da.da_destroy(c2)
