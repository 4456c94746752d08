"""Checkpoint and resume (da_anneal_segment, GPU).

An anneal run in segments, each resumed from the checkpoint the previous one
wrote, must give exactly the results of one anneal over the whole schedule: the
random numbers are keyed by the absolute step, the fp32 recompute falls on
absolute multiples of its period, and the offset count and best state travel in
the checkpoint.  Cuts are placed on and between recompute points and inside
the launch chunks.  A checkpoint's integer fields are the exact fields of its
states, and a first segment equals a shorter anneal that stops there.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

KEYS = ("final_E", "best_E", "final_x", "best_x", "flips", "max_drift")


@pytest.fixture(scope="module")
def da():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1806_08815_gb300 import binding
    binding.lib()
    return binding


def _instance(da, kind, N):
    from paper_1806_08815_gb300 import instances
    if kind == "i8":
        return da.da_create(instances.sk_bimodal(N, 31).Q)
    if kind == "f32":
        return da.da_create(instances.sk_gaussian(N, 31).Q)
    Qi, _ = da.da_quantize(instances.sk_gaussian(N, 31).Q)
    return da.da_create(Qi, da.DA_INT16)


@pytest.mark.parametrize("kind,N,R,T,cuts,P,inc", [
    ("i8", 200, 12, 3000, [700, 1900], 0, 1.0),
    ("f32", 300, 10, 3000, [1024, 1500, 2047], 256, 0.25),
    ("i16", 150, 8, 2000, [999], 0, 0.0),
    ("f32", 1500, 6, 1200, [300, 900], 128, 0.0),
])
def test_segments_equal_one_anneal(da, kind, N, R, T, cuts, P, inc):
    from paper_1806_08815_gb300 import instances
    ctx = _instance(da, kind, N)
    beta = instances.beta_linear(0.1, 4.0, T)
    if kind == "i16":
        beta = (beta / 300.0).astype(np.float32)
    seed = 17
    full = da.da_anneal(ctx, beta, inc, R, seed, recompute_every=P)
    ck, t = None, 0
    for i, t1 in enumerate(cuts + [T]):
        res, ck = da.da_anneal_segment(ctx, beta, t, t1, inc, R, seed, P, ck)
        if i == 0:   # the first segment equals an anneal that stops at its end
            short = da.da_anneal(ctx, beta[:t1], inc, R, seed, recompute_every=P)
            for k in KEYS:
                assert np.array_equal(res[k], short[k]), ("first segment", k)
        if kind != "f32":   # integer fields in the checkpoint are exact
            assert np.array_equal(ck["fields"], da.da_field_recompute(ctx, ck["x"]))
        t = t1
    for k in KEYS:
        assert np.array_equal(res[k], full[k]), k
    assert np.array_equal(ck["x"], full["final_x"])
    assert np.array_equal(ck["scalars"][:, 2], full["flips"])


def test_segment_arguments(da):
    from paper_1806_08815_gb300 import instances
    ctx = _instance(da, "i8", 64)
    beta = instances.beta_linear(0.1, 3.0, 100)
    with pytest.raises(da.DAError):          # no checkpoint for a segment that starts later
        da.da_anneal_segment(ctx, beta, 10, 20, 0.0, 4, 1)
    with pytest.raises(da.DAError):          # t1 beyond the schedule
        da.da_anneal_segment(ctx, beta, 0, 200, 0.0, 4, 1)
    # an empty first segment is the start state
    res, ck = da.da_anneal_segment(ctx, beta, 0, 0, 0.0, 4, 1)
    assert np.all(ck["x"] == 0) and np.all(res["flips"] == 0) and np.all(res["final_E"] == 0)
