"""The allocation-free anneal entry point (da_anneal_static) against the
context-based one (da_anneal_async) on the same instance.

Callers that cannot allocate device memory (a service that reserves all GPU
memory up front, code inside another framework's allocator-free region)
use da_anneal_static, which keeps its intermediate buffers in one fixed device
array.  Two calls in a row must each reproduce the context-based results
exactly (integer anneal: bit-exact), so the shared array carries nothing from
one call to the next.  This file is collected last on purpose.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _device_instance(torch, Q, ldw):
    N = Q.shape[0]
    W = np.triu(Q.astype(np.int64), 1)
    W = (W + W.T).astype(np.int8)
    Wp = np.zeros((N, ldw), np.int8)
    Wp[:, :N] = W
    return (torch.from_numpy(Wp).cuda(), torch.from_numpy(np.diag(Q).astype(np.int32).copy()).cuda())


def _outputs(torch, R, words, T):
    dev = torch.device("cuda", 0)
    return dict(final_E=torch.zeros(R, dtype=torch.float64, device=dev),
                best_E=torch.zeros(R, dtype=torch.float64, device=dev),
                final_x=torch.zeros((R, words), dtype=torch.int32, device=dev),
                best_x=torch.zeros((R, words), dtype=torch.int32, device=dev),
                flips=torch.zeros(R, dtype=torch.int64, device=dev),
                trace=torch.zeros((R, T), dtype=torch.int32, device=dev))


@pytest.mark.parametrize("N", [64, 100, 1024])
def test_static_anneal_matches_context_anneal_twice(N):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1806_08815_gb300 import binding as da
    from paper_1806_08815_gb300 import instances

    q = instances.sk_bimodal(N, 5)
    R, T = 48, 1500
    beta = torch.from_numpy(instances.beta_linear(0.05, 3.0, T)).cuda()
    ldw = da.da_static_pitch(N)
    assert ldw >= N
    W_dev, d_dev = _device_instance(torch, q.Q, ldw)
    ctx = da.da_create(q.Q)
    s = torch.cuda.Stream()
    words = da.da_words(N)
    for seed in (11, 12):                         # two calls in a row on the shared array
        ref = _outputs(torch, R, words, T)
        got = _outputs(torch, R, words, T)
        da.da_anneal_async(ctx, beta, T, 1.0, R, seed, 0, ref, s)
        da.da_anneal_static(W_dev, d_dev, N, ldw, beta, T, 1.0, R, seed, got, s)
        s.synchronize()
        for k in ref:
            assert torch.equal(ref[k], got[k]), (seed, k)
        assert int(got["flips"].sum()) > 0


def test_static_anneal_rejects_oversize():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1806_08815_gb300 import binding as da
    N = 1024
    ldw = da.da_static_pitch(N)
    W = torch.zeros((N, ldw), dtype=torch.int8, device="cuda")
    d = torch.zeros(N, dtype=torch.int32, device="cuda")
    beta = torch.zeros(10, dtype=torch.float32, device="cuda")
    with pytest.raises(da.DAError):
        da.da_anneal_static(W, d, N, ldw, beta, 10, 0.0, 1 << 16, 0, {}, 0)
    with pytest.raises(da.DAError):
        da.da_anneal_static(W, d, 2000, ldw, beta, 10, 0.0, 4, 0, {}, 0)


def test_static_anneal_rejects_misaligned_pointers():
    """A W that is not 16-byte aligned (e.g. a slice of a caller's buffer), a
    misaligned diagonal or result array, and a pitch beyond int range are
    refused on the host, before anything reaches the device."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1806_08815_gb300 import binding as da
    N = 64
    ldw = da.da_static_pitch(N)
    buf = torch.zeros(N * ldw + 64, dtype=torch.int8, device="cuda")
    d = torch.zeros(N + 4, dtype=torch.int32, device="cuda")
    beta = torch.zeros(10, dtype=torch.float32, device="cuda")
    for off in (1, 4, 8):
        W = buf[off:off + N * ldw]
        with pytest.raises(da.DAError, match="16-byte aligned"):
            da.da_anneal_static(W, d, N, ldw, beta, 10, 0.0, 4, 0, {}, 0)
    W = buf[:N * ldw]
    dbytes = d.view(torch.int8)
    with pytest.raises(da.DAError, match="4-byte aligned"):
        da.da_anneal_static(W, dbytes[2:2 + 4 * N], N, ldw, beta, 10, 0.0, 4, 0, {}, 0)
    E = torch.zeros(8 * 4 + 8, dtype=torch.int8, device="cuda")
    with pytest.raises(da.DAError, match="aligned to their element size"):
        da.da_anneal_static(W, d, N, ldw, beta, 10, 0.0, 4, 0, {"final_E": E[4:]}, 0)
    with pytest.raises(da.DAError, match="INT_MAX"):
        da.da_anneal_static(W, d, N, 1 << 31, beta, 10, 0.0, 4, 0, {}, 0)
    # the aligned call still runs
    torch.cuda.synchronize()
    out = {"flips": torch.zeros(4, dtype=torch.int64, device="cuda")}
    da.da_anneal_static(W, d, N, ldw, beta, 10, 0.0, 4, 0, out, 0)
    torch.cuda.synchronize()
