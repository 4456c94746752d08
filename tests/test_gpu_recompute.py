"""GPU parity of the exact field recompute (the tensor-core form behind
da_field_recompute, da_energy and every recompute inside an anneal) against
the oracle's fixed-point definition, bit for bit.

Sizes span several 64-variable and 128-state tiles with ragged tails on both
sides, up to the largest N the library accepts; the coefficient mixes include
a wide dynamic range (so the low digit planes matter to the rounding) and
int8 couplings at both ends of their range.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def da():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1806_08815_gb300 as m
    return m


def _states(rng, R, N):
    X = (rng.random((R, N)) < rng.uniform(0.05, 0.95, (R, 1))).astype(np.int64)
    X[0] = 0
    if R > 1:
        X[1] = 1
    return X


def _check_f32(da, Q, R, seed, sample=None):
    import oracle
    rng = np.random.default_rng(seed)
    N = Q.shape[0]
    ctx = da.da_create(Q)
    xp = oracle.pack(_states(rng, R, N))
    h = da.da_field_recompute(ctx, xp)
    E = da.da_energy(ctx, xp)
    rows = range(R) if sample is None else sorted(set([0, 1, R - 1]) | set(rng.choice(R, sample, replace=False)))
    for r in rows:
        hr, _, _ = oracle.recompute_f32(Q, xp[r])
        assert np.array_equal(h[r].view(np.uint32), hr.view(np.uint32)), r
        assert E[r] == oracle.recompute_energy_f32(Q, xp[r]), r


def _check_int8(da, Q, R, seed, sample=None):
    import oracle
    rng = np.random.default_rng(seed)
    N = Q.shape[0]
    ctx = da.da_create(Q)
    xp = oracle.pack(_states(rng, R, N))
    h = da.da_field_recompute(ctx, xp)
    E = da.da_energy(ctx, xp)
    ref = oracle.energy(Q, xp)
    assert np.array_equal(E, ref.astype(float))
    rows = range(R) if sample is None else sorted(set([0, 1, R - 1]) | set(rng.choice(R, sample, replace=False)))
    d = np.diag(Q).astype(np.int64)
    for r in rows:
        assert np.array_equal(h[r].astype(np.int64), oracle.fields_int(Q, xp[r]) + d), r


@pytest.mark.parametrize("N,R", [(1, 3), (2, 2), (63, 129), (64, 128), (65, 127), (130, 300), (1000, 257),
                                 (1024, 128), (2049, 5)])
def test_fp32_sk_gaussian(da, N, R):
    from paper_1806_08815_gb300 import instances
    _check_f32(da, instances.sk_gaussian(N, 10 + N).Q, R, N, sample=None if N * R <= 70000 else 24)


@pytest.mark.parametrize("N", [4096, 8192])
def test_fp32_largest_sizes(da, N):
    from paper_1806_08815_gb300 import instances
    _check_f32(da, instances.sk_gaussian(N, 3).Q, 130, N, sample=6)


@pytest.mark.parametrize("N", [97, 640])
def test_fp32_wide_dynamic_range(da, N):
    """Coefficients 2^k u with k uniform in [-40, 40]: many of them sit far
    below the largest, so the fp32 rounding of a sum depends on every digit."""
    rng = np.random.default_rng(N)
    Q = np.triu(np.ldexp(rng.uniform(-1, 1, (N, N)), rng.integers(-40, 41, (N, N)))).astype(np.float32)
    _check_f32(da, Q, 150, N + 1)


def test_fp32_sums_that_cancel(da):
    """A coefficient that cancels the rest exactly: the exact sum is tiny
    compared with its terms, which an fp32 or fp64 accumulation would lose."""
    rng = np.random.default_rng(5)
    N = 300
    Q = np.triu(rng.standard_normal((N, N)).astype(np.float32), 1)
    Q[0, 1:] = 1e4
    Q[1, 2:] = -1e4
    np.fill_diagonal(Q, rng.standard_normal(N).astype(np.float32))
    _check_f32(da, Q, 140, 6)


@pytest.mark.parametrize("N,R", [(64, 129), (77, 9), (1024, 200), (3000, 140)])
def test_int8(da, N, R):
    rng = np.random.default_rng(N)
    Q = np.triu(rng.integers(-128, 128, (N, N)), 1).astype(np.int32)
    Q[0, 1:] = -128
    Q[1, 2:] = 127
    np.fill_diagonal(Q, rng.integers(-5000, 5000, N))
    _check_int8(da, Q, R, N, sample=None if N <= 1024 else 8)
