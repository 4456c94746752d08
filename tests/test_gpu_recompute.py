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


def test_fixed_point_conversion_matches_intrinsics(da):
    """round(w 2^S), ties to even, in integer arithmetic (as the recompute
    kernels evaluate it) against the 64-bit conversion instruction and an
    exact host evaluation, over all exponents, subnormals, zeros and ties."""
    rng = np.random.default_rng(11)
    bits = rng.integers(0, 0x7F800000, 400_000, dtype=np.uint32)          # every finite magnitude
    bits |= (rng.integers(0, 2, bits.size, dtype=np.uint32) << 31)
    w = bits.view(np.float32)
    ew = np.floor(np.log2(np.maximum(np.abs(w.astype(np.float64)), 2.0 ** -149))).astype(np.int64)
    S = np.array([rng.integers(-170, 62 - e) for e in ew], np.int32)       # |w 2^S| < 2^62
    # exact ties k + 1/2 and values just around them
    k = rng.integers(0, 1 << 22, 20_000)
    St = rng.integers(1, 40, k.size).astype(np.int32)
    wt = np.ldexp((2 * k + 1).astype(np.float64), -St - 1).astype(np.float32)
    w = np.concatenate([w, wt, np.nextafter(wt, np.float32(np.inf)), np.nextafter(wt, np.float32(-np.inf)),
                        np.float32([0.0, -0.0, 1.5, 2.5, -2.5, 0.5, -0.5])])
    S = np.concatenate([S, St, St, St, np.int32([0, 0, 0, 0, 0, 0, 0])])
    got, ref = da.binding.da_diag_fixed(w, S)
    assert np.array_equal(got, ref)
    exact = np.rint(np.ldexp(w.astype(np.float64), S)).astype(np.int64)   # exact product, round half even
    assert np.array_equal(got, exact)


def test_scaled_float_conversion_matches_intrinsics(da):
    """fl32(v) 2^-S (round to nearest even, then scale) in integer arithmetic
    against __ll2float_rn + ldexpf, over every magnitude, ties, and results
    that are subnormal or overflow."""
    rng = np.random.default_rng(12)
    mag = rng.integers(0, 63, 300_000)
    v = (rng.integers(0, 1 << 62, mag.size, dtype=np.int64) >> (62 - mag)) * rng.choice([-1, 1], mag.size)
    ties = np.array([(1 << 25) + 2, (1 << 25) + 6, (1 << 24) + 1, (1 << 24) + 3, (1 << 40) + (1 << 16),
                     (1 << 40) + (3 << 16), (1 << 62), (1 << 62) - 1, 1, 0, -1], np.int64)
    v = np.concatenate([v, ties, -ties])
    S = rng.integers(-80, 200, v.size).astype(np.int32)
    S[-2 * ties.size:] = rng.integers(-5, 60, 2 * ties.size)
    got, ref = da.binding.da_diag_scaled(v, S)
    assert np.array_equal(got.view(np.uint32), ref.view(np.uint32))
    host = np.ldexp(v.astype(np.float32).astype(np.float64), -S.astype(np.int64))
    normal = (np.abs(host) >= 2.0 ** -126) & (np.abs(host) < 2.0 ** 128)
    assert np.array_equal(got[normal].astype(np.float64), host[normal])


@pytest.mark.parametrize("N,R", [(130, 129), (1000, 150), (5000, 140)])
def test_int16(da, N, R):
    """16-bit couplings (two digit planes) at both ends of their range, 26-bit diagonal."""
    rng = np.random.default_rng(N + 1)
    Q = np.triu(rng.integers(-32767, 32768, (N, N)), 1).astype(np.int32)
    Q[0, 1:] = -32767
    Q[1, 2:] = 32767
    np.fill_diagonal(Q, rng.integers(-(2 ** 25) + 1, 2 ** 25, N))
    import oracle
    ctx = da.da_create(Q, da.DA_INT16)
    xp = oracle.pack(_states(rng, R, N))
    assert np.array_equal(da.da_energy(ctx, xp), oracle.energy(Q, xp).astype(float))
    h = da.da_field_recompute(ctx, xp)
    d = np.diag(Q).astype(np.int64)
    for r in sorted({0, 1, R - 1} | set(rng.choice(R, 6, replace=False))):
        assert np.array_equal(h[r].astype(np.int64), oracle.fields_int(Q, xp[r]) + d), r


@pytest.mark.parametrize("dtype_name,N", [("DA_INT8", 33), ("DA_INT16", 1000), ("DA_FP32", 4097)])
def test_instance_reads_upper_triangle_only(da, dtype_name, N):
    """The device-side instance build mirrors the upper triangle: values below
    the diagonal change nothing, and the fields match the oracle's."""
    import oracle
    rng = np.random.default_rng(N + 7)
    dtype = getattr(da, dtype_name)
    if dtype_name == "DA_FP32":
        Q = np.triu(rng.standard_normal((N, N))).astype(np.float32)
        junk = rng.standard_normal((N, N)).astype(np.float32) * 1e30
    else:
        hi = 127 if dtype_name == "DA_INT8" else 32767
        Q = np.triu(rng.integers(-hi, hi + 1, (N, N)), 1).astype(np.int32)
        np.fill_diagonal(Q, rng.integers(-1000, 1000, N))
        junk = rng.integers(-2 ** 31, 2 ** 31, (N, N)).astype(np.int32)
    Qj = Q + np.tril(junk, -1)
    xp = oracle.pack(_states(rng, 9, N))
    a = da.da_field_recompute(da.da_create(Q, dtype), xp)
    b = da.da_field_recompute(da.da_create(Qj, dtype), xp)
    assert np.array_equal(a.view(np.uint32), b.view(np.uint32))
    for r in (0, 1, 5):
        if dtype_name == "DA_FP32":
            hr, _, _ = oracle.recompute_f32(Q, xp[r])
            assert np.array_equal(a[r].view(np.uint32), hr.view(np.uint32)), r
        else:
            ref = oracle.fields_int(Q, xp[r]) + np.diag(Q).astype(np.int64)
            assert np.array_equal(a[r].astype(np.int64), ref), r
