"""GPU parity: the CUDA path, called through the C ABI, against the CPU oracle.

Integer (bimodal) runs must reproduce the oracle's flip trajectory bit for bit;
so must fp32 runs, whose every decision and field update is one IEEE fp32
operation on both sides and whose periodic recompute is an exact fixed-point
sum.  Energies of identical states agree to fp64 rounding (1e-12 relative).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

NT = 8   # oracle threads


@pytest.fixture(scope="module")
def da():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1806_08815_gb300 as m
    return m


@pytest.fixture(scope="module")
def inst():
    from paper_1806_08815_gb300 import instances
    return instances


def _compare_anneal(got, ref, Q, exact_int):
    import oracle
    assert np.array_equal(got["trace"], ref["trace"])
    assert np.array_equal(got["final_x"], ref["x_final"])
    assert np.array_equal(got["best_x"], ref["x_best"])
    assert np.array_equal(got["flips"], ref["flips"])
    Ef = oracle.energy(Q, got["final_x"])
    Eb = oracle.energy(Q, got["best_x"])
    if exact_int:
        assert np.array_equal(got["final_E"], Ef.astype(float))
        assert np.array_equal(got["best_E"], Eb.astype(float))
        assert np.array_equal(got["final_E"], ref["E_final"])
        assert np.all(got["max_drift"] == 0)
    else:
        assert np.allclose(got["final_E"], Ef, rtol=1e-12, atol=1e-12)
        assert np.allclose(got["best_E"], Eb, rtol=1e-12, atol=1e-12)
        # the tracked fp32 energy stays within 1e-5 relative of the exact one
        assert np.all(got["max_drift"] <= 1e-5 * np.maximum(1.0, np.abs(Ef)))


def test_device_exp_matches_oracle_exhaustively(da):
    """Every fp32 x with 2^-30 <= -x <= 16.7 (all arguments the kernels evaluate
    beyond the round-to-1 region), and a sample of the rest, bit for bit."""
    import oracle
    lo = np.float32(-(2.0 ** -30)).view(np.uint32)
    hi = np.float32(-16.7).view(np.uint32)
    step = 1 << 25
    for start in range(int(lo), int(hi) + 1, step):
        bits = np.arange(start, min(start + step, int(hi) + 1), dtype=np.uint32)
        x = bits.view(np.float32)
        assert np.array_equal(da.binding.da_diag_expf(x).view(np.uint32), oracle.expf(x).view(np.uint32))
    rng = np.random.default_rng(0)
    x = np.concatenate([-rng.random(1 << 20).astype(np.float32) * 200, -rng.random(1 << 16).astype(np.float32) * 1e-9,
                        np.array([0.0, -0.0, -86.0, -86.00001, -np.inf], np.float32)])
    assert np.array_equal(da.binding.da_diag_expf(x).view(np.uint32), oracle.expf(x).view(np.uint32))


def test_log_uniform_error_bound(da):
    """log2 U as the step kernels keep it for every draw, for each of the 2^24
    values of U = (w >> 8) + 1: its error against log2 U in fp64 (about one fp32
    ulp near 24: 1.99e-6 measured, below 2^-18) is far inside the decision band
    2^-15."""
    U = np.arange(1, 2 ** 24 + 1, dtype=np.int64)
    w = ((U - 1) << 8).astype(np.uint32)
    L = da.binding.da_diag_log_uniform(w)
    err = np.abs(L.astype(np.float64) - np.log2(U.astype(np.float64)))
    assert err.max() < 2.0 ** -18
    assert L[0] == 0.0 and L[-1] == 24.0


def test_log_domain_decision_matches_exact_test(da):
    """The step kernels decide s = delta beta log2(e) + log2 U against 24 -+ 2^-15
    (their decide_log: sign bits of s - (24 - 2^-15), packed pairs, the band by an
    unsigned minimum; called here through a diagnostic kernel) and fall back to the
    exact test inside that band: for trials placed
    right at the acceptance boundary (relative offsets 2^-30 .. 2^-8 either side),
    random trials, delta <= 0, beta = 0 and u = 1 its decision equals
    delta <= 0 || u < exp_neg(-fl(beta delta))."""
    import oracle
    rng = np.random.default_rng(7)
    n = 1 << 22
    U = rng.integers(1, 2 ** 24 + 1, n)
    beta = np.exp(rng.uniform(np.log(0.01), np.log(50.0), n)).astype(np.float32)
    rho = rng.choice([-1.0, 1.0], n) * 2.0 ** -rng.uniform(8, 30, n)
    delta = (-np.log(U * 2.0 ** -24) / beta.astype(np.float64) * (1 + rho)).astype(np.float32)
    m = 1 << 20
    U2 = rng.integers(1, 2 ** 24 + 1, m)
    b2 = rng.uniform(0, 20, m).astype(np.float32)
    b2[:1000] = 0.0
    d2 = rng.normal(0, 3, m).astype(np.float32)
    d2[1000:2000] = 0.0
    d2[2000:3000] = -0.0
    U2[3000:4000] = 2 ** 24
    U = np.concatenate([U, U2])
    beta = np.concatenate([beta, b2])
    delta = np.concatenate([delta, d2])
    w = (((U - 1) << 8) | rng.integers(0, 256, U.size)).astype(np.uint32)
    got, band = da.binding.da_diag_accept_log(delta, beta, w)
    x = np.minimum(-(beta * delta), np.float32(0.0)).astype(np.float32)    # fp32 product
    exact = (delta <= 0) | (U * 2.0 ** -24 < oracle.expf(x).astype(np.float64))
    assert np.array_equal(got, exact)
    assert band[n:].mean() < 1e-3        # typical trials rarely need the exact test


def test_device_philox_matches_oracle(da):
    import oracle
    rng = np.random.default_rng(1)
    ck = rng.integers(0, 2 ** 32, size=(4096, 6), dtype=np.uint64).astype(np.uint32)
    ck[:3] = [[0] * 6, [0xFFFFFFFF] * 6, [0x243f6a88, 0x85a308d3, 0x13198a2e, 0x03707344, 0xa4093822, 0x299f31d0]]
    got = da.binding.da_diag_philox(ck)
    for row, g in zip(ck[:512], got[:512]):
        assert np.array_equal(g, oracle.philox(row[:4], row[4:]))
    assert [hex(v) for v in got[0]] == ["0x6627e8d5", "0xe169c58d", "0xbc57ac4c", "0x9b00dbd8"]


def test_sk_bimodal_n64_full_config(da, inst):
    """Fully connected +-1 spin glass, N = 64, 64 replicas, 10^4 steps, beta linear
    0.05 -> 3.0, offset increment 1, seed 0: bit-exact trajectories."""
    import oracle
    q = inst.sk_bimodal(64, 0)
    beta = inst.beta_linear(0.05, 3.0, 10_000)
    ctx = da.da_create(q.Q)
    got = da.da_anneal(ctx, beta, 1.0, 64, 0, trace=True)
    ref = oracle.da_anneal(q.Q, beta, R=64, seed=0, inc=1.0, trace=True, nthreads=NT)
    _compare_anneal(got, ref, q.Q, True)


SHAPES = [(0, 0, 0), (4, 1, 4), (8, 1, 3), (4, 2, 2), (4, 4, 1), (8, 8, 1), (8, 2, 1)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("N", [1, 33, 100])
def test_int8_ragged_sizes_all_shapes(da, inst, N, shape):
    import oracle
    q = inst.random_qubo(N, N + 1, True, -5, 5)
    if N > 1:
        q = inst.Instance(q.name, N, np.triu(q.Q).astype(np.int32), 0.0, q.J)
    beta = inst.beta_linear(0.1, 2.5, 700)
    ctx = da.da_create(q.Q)
    if shape[0]:
        if 32 * shape[0] * shape[1] < N:
            pytest.skip("shape smaller than N")
        da.da_set_launch_shape(ctx, *shape)
    got = da.da_anneal(ctx, beta, 0.5, 13, 7, trace=True)
    ref = oracle.da_anneal(q.Q, beta, R=13, seed=7, inc=0.5, trace=True, nthreads=NT)
    _compare_anneal(got, ref, q.Q, True)


@pytest.mark.parametrize("density", [0.1, 0.5, 0.9])
def test_erdos_renyi_density_instances(da, inst, density):
    """Bimodal couplings on G(N, p) graphs (the density study), beta linear 1/T_h -> 1/T_l
    from its temperature table, offset off: bit-exact trajectories at N = 256, and at the
    study's N = 1024 on sampled replicas of a 100-run launch."""
    import oracle
    from bench import DENSITY_TEMPS
    Th, Tl = DENSITY_TEMPS[density]
    q = inst.erdos_renyi_bimodal(256, density, 1)
    beta = inst.beta_linear(1.0 / Th, 1.0 / Tl, 2000)
    ctx = da.da_create(q.Q)
    got = da.da_anneal(ctx, beta, 0.0, 10, 3, trace=True)
    ref = oracle.da_anneal(q.Q, beta, R=10, seed=3, inc=0.0, trace=True, nthreads=NT)
    _compare_anneal(got, ref, q.Q, True)
    q = inst.erdos_renyi_bimodal(1024, density, 2)
    beta = inst.beta_linear(1.0 / Th, 1.0 / Tl, 3000)
    ctx = da.da_create(q.Q)
    got = da.da_anneal(ctx, beta, 0.0, 100, 5)
    for r in (0, 63, 99):
        ref = oracle.da_anneal(q.Q, beta, R=1, seed=5, inc=0.0, replica_base=r)
        assert np.array_equal(got["best_x"][r], ref["x_best"][0])
        assert got["best_E"][r] == ref["E_best"][0]


@pytest.mark.parametrize("N,dtype", [(33, "i8"), (100, "i8"), (700, "i8"), (1024, "f32"), (200, "f32")])
def test_draw_warp_on_and_off(da, inst, N, dtype):
    """The G = 1 step with and without its producer warp: both reproduce the oracle."""
    import oracle
    q = inst.sk_bimodal(N, N) if dtype == "i8" else inst.sk_gaussian(N, N)
    beta = inst.beta_linear(0.05, 4.0 if dtype == "i8" else 9.0, 1500)
    rec = 0 if dtype == "i8" else 512
    ref = oracle.da_anneal(q.Q, beta, R=9, seed=4, inc=0.5, recompute_every=rec, trace=True, nthreads=NT)
    for on in (True, False):
        ctx = da.da_create(q.Q)
        da.binding.da_set_draw_warp(ctx, on)
        got = da.da_anneal(ctx, beta, 0.5, 9, 4, recompute_every=rec, trace=True)
        _compare_anneal(got, ref, q.Q, dtype == "i8")


@pytest.mark.parametrize("N,shape", [(300, (0, 0, 0)), (300, (16, 1, 2)), (1000, (0, 0, 0)), (1000, (8, 4, 1)),
                                     (1500, (0, 0, 0)), (1500, (32, 2, 2)), (2100, (0, 0, 0)), (2100, (16, 8, 1)),
                                     (3000, (32, 4, 1))])
def test_int8_larger_sizes(da, inst, N, shape):
    import oracle
    q = inst.sk_bimodal(N, 3)
    beta = inst.beta_linear(0.02, 1.5, 300)
    ctx = da.da_create(q.Q)
    if shape[0]:
        da.da_set_launch_shape(ctx, *shape)
    got = da.da_anneal(ctx, beta, 1.0, 6, 11, trace=True)
    ref = oracle.da_anneal(q.Q, beta, R=6, seed=11, inc=1.0, trace=True, nthreads=NT)
    _compare_anneal(got, ref, q.Q, True)


@pytest.mark.parametrize("shape", [(0, 0, 0), (4, 2, 2), (8, 1, 4), (8, 4, 1), (16, 2, 2), (32, 4, 1)])
def test_fp32_sk_gaussian_with_recompute(da, inst, shape):
    import oracle
    q = inst.sk_gaussian(256, 5)
    beta = inst.beta_linear(0.2, 8.0, 3000)
    ctx = da.da_create(q.Q)
    if shape[0]:
        da.da_set_launch_shape(ctx, *shape)
    got = da.da_anneal(ctx, beta, 0.25, 16, 5, recompute_every=256, trace=True)
    ref = oracle.da_anneal(q.Q, beta, R=16, seed=5, inc=0.25, recompute_every=256, trace=True, nthreads=NT)
    _compare_anneal(got, ref, q.Q, False)


def test_fp32_lattice_l32_geometric(da, inst):
    """2D Gaussian torus L = 32 (N = 1024) kept dense, geometric beta 0.1 -> 5.0, offset 0.5."""
    import oracle
    q = inst.lattice2d(32, 0, True)
    beta = inst.beta_geometric(0.1, 5.0, 2000)
    ctx = da.da_create(q.Q)
    got = da.da_anneal(ctx, beta, 0.5, 8, 2, recompute_every=1024, trace=True)
    ref = oracle.da_anneal(q.Q, beta, R=8, seed=2, inc=0.5, recompute_every=1024, trace=True, nthreads=NT)
    _compare_anneal(got, ref, q.Q, False)


def test_fp32_sk_n1024_recompute_1024(da, inst):
    import oracle
    q = inst.sk_gaussian(1024, 0)
    beta = inst.beta_linear(0.5, 10.0, 2100)
    ctx = da.da_create(q.Q)
    got = da.da_anneal(ctx, beta, 0.0, 4, 0, recompute_every=1024, trace=True)
    ref = oracle.da_anneal(q.Q, beta, R=4, seed=0, inc=0.0, recompute_every=1024, trace=True, nthreads=NT)
    _compare_anneal(got, ref, q.Q, False)


def test_full_size_sk_n1024_sampled_replicas(da, inst):
    """The benchmark's launch (SK Gaussian N = 1024, 1024 replicas, 2e5 steps, recompute
    every 1024) checked on two sampled replicas that the oracle reruns alone."""
    import oracle
    from bench import C3
    q = inst.sk_gaussian(C3["N"], C3["instance_seed"])
    beta = inst.beta_linear(C3["beta0"], C3["beta1"], C3["steps"])
    ctx = da.da_create(q.Q)
    da.binding.da_tune_shape(ctx, C3["replicas"])      # the launch shape the benchmark times
    got = da.da_anneal(ctx, beta, C3["inc"], C3["replicas"], C3["seed"], recompute_every=C3["recompute_every"])
    for r in (0, 777):
        ref = oracle.da_anneal(q.Q, beta, R=1, seed=C3["seed"], inc=C3["inc"], replica_base=r,
                               recompute_every=C3["recompute_every"])
        assert np.array_equal(got["final_x"][r], ref["x_final"][0])
        assert np.array_equal(got["best_x"][r], ref["x_best"][0])
        assert got["flips"][r] == ref["flips"][0]
        assert abs(got["best_E"][r] - oracle.energy(q.Q, ref["x_best"])[0]) <= 1e-12 * abs(got["best_E"][r])


def test_full_size_batched_sampled_replicas(da, inst):
    """The benchmark's batched launch (512 instances, N in {64, ..., 1024}, half int8 / half fp32,
    64 replicas, 10^4 steps, the tuner's configuration per class) checked on sampled replicas of
    one item per coupling type at the smallest and largest size, each rerun alone by the oracle."""
    import oracle
    from bench import batched_jobs
    import concurrent.futures
    jobs, meta = batched_jobs(da, inst, keep_Q=True)
    picked = [meta.index(cls) for cls in ((True, 64), (False, 64), (True, 1024), (False, 1024))]
    sampled = [(i, r) for i in picked for r in (0, 37)]

    def rerun(ir):
        j = jobs[ir[0]]
        return oracle.da_anneal(j["Q"], j["beta"], R=1, seed=j["seed"], inc=j["offset_inc"], replica_base=ir[1],
                                recompute_every=j["recompute_every"])

    ex = concurrent.futures.ThreadPoolExecutor(NT)     # the oracle's C calls run beside the GPU work
    refs = {ir: ex.submit(rerun, ir) for ir in sampled}
    outs, el = da.binding.da_batch_anneal(jobs)
    assert el > 0
    for i in picked:
        j, o = jobs[i], outs[i]
        for r in (0, 37):
            ref = refs[(i, r)].result()
            assert np.array_equal(o["final_x"][r], ref["x_final"][0]), (meta[i], r)
            assert np.array_equal(o["best_x"][r], ref["x_best"][0]), (meta[i], r)
            assert o["flips"][r] == ref["flips"][0], (meta[i], r)
            Eb = oracle.energy(j["Q"], ref["x_best"])[0]
            if meta[i][0]:
                assert o["best_E"][r] == Eb
            else:
                assert abs(o["best_E"][r] - Eb) <= 1e-12 * max(1.0, abs(Eb))


def test_edge_cases(da, inst):
    import oracle
    q = inst.sk_bimodal(40, 9)
    ctx = da.da_create(q.Q)
    # zero steps: everything stays at x = 0
    got = da.da_anneal(ctx, np.zeros(0, np.float32), 1.0, 3, 1)
    assert np.all(got["final_x"] == 0) and np.all(got["final_E"] == 0) and np.all(got["flips"] == 0)
    # beta = 0: every trial accepted, a flip at every step
    got = da.da_anneal(ctx, np.zeros(50, np.float32), 0.0, 2, 1, trace=True)
    ref = oracle.da_anneal(q.Q, np.zeros(50, np.float32), R=2, seed=1, trace=True)
    assert np.array_equal(got["trace"], ref["trace"]) and np.all(got["trace"] >= 0)
    # zero temperature, offset off, from a local minimum: nothing is ever accepted
    Q = np.triu(np.random.default_rng(0).integers(-3, 4, (20, 20)), 1).astype(np.int32)
    Q[np.arange(20), np.arange(20)] = 50
    ctx2 = da.da_create(Q)
    got = da.da_anneal(ctx2, np.full(30, 1e6, np.float32), 0.0, 2, 1, trace=True)
    assert np.all(got["trace"] == -1)
    # and with the offset on, the first flip comes at the closed-form step
    got = da.da_anneal(ctx2, np.full(40, 1e6, np.float32), 2.0, 2, 1, trace=True)
    assert np.all(got["trace"][:, :25] == -1) and np.all(got["trace"][:, 25] >= 0)


def test_schedule_must_be_finite_and_nonnegative(da, inst):
    q = inst.sk_bimodal(40, 1)
    ctx = da.da_create(q.Q)
    for bad in (-1.0, np.inf, np.nan):
        beta = np.full(10, 0.5, np.float32)
        beta[3] = bad
        with pytest.raises(da.DAError) as e:
            da.da_anneal(ctx, beta, 0.0, 2, 0)
        assert e.value.status == 1


def test_results_do_not_depend_on_replica_count(da, inst):
    q = inst.sk_bimodal(64, 4)
    beta = inst.beta_linear(0.05, 3.0, 500)
    ctx = da.da_create(q.Q)
    a = da.da_anneal(ctx, beta, 1.0, 40, 9, trace=True)
    b = da.da_anneal(ctx, beta, 1.0, 7, 9, trace=True)
    assert np.array_equal(a["trace"][:7], b["trace"])


def test_energy_and_recompute_entry_points(da, inst):
    import oracle
    rng = np.random.default_rng(3)
    for q in (inst.sk_bimodal(77, 1), inst.sk_gaussian(130, 2)):
        ctx = da.da_create(q.Q)
        X = rng.integers(0, 2, (9, q.N))
        xp = oracle.pack(X)
        E = da.da_energy(ctx, xp)
        ref = oracle.energy(q.Q, xp)
        h = da.da_field_recompute(ctx, xp)
        if q.bimodal:
            assert np.array_equal(E, ref.astype(float))
            for r in range(9):
                assert np.array_equal(h[r], oracle.fields_int(q.Q, xp[r]) + np.diag(q.Q))
        else:
            assert np.allclose(E, ref, rtol=1e-12, atol=1e-12)
            for r in range(9):
                hr, _, _ = oracle.recompute_f32(q.Q, xp[r])
                assert np.array_equal(h[r].view(np.uint32), hr.view(np.uint32))
                assert E[r] == oracle.recompute_energy_f32(q.Q, xp[r])


def test_async_device_resident_matches_blocking(da, inst):
    import torch
    q = inst.sk_gaussian(200, 8)
    beta = inst.beta_linear(0.3, 6.0, 1500)
    ctx = da.da_create(q.Q)
    ref = da.da_anneal(ctx, beta, 0.5, 10, 4, recompute_every=500)
    dev = torch.device("cuda", 0)
    W = da.da_words(q.N)
    out = dict(final_E=torch.zeros(10, dtype=torch.float64, device=dev),
               best_E=torch.zeros(10, dtype=torch.float64, device=dev),
               final_x=torch.zeros((10, W), dtype=torch.int32, device=dev),
               flips=torch.zeros(10, dtype=torch.int64, device=dev))
    s = torch.cuda.Stream()
    bd = torch.from_numpy(beta).to(dev)
    torch.cuda.synchronize()
    da.da_anneal_async(ctx, bd, beta.size, 0.5, 10, 4, 500, out, s)
    s.synchronize()
    assert np.array_equal(out["final_E"].cpu().numpy(), ref["final_E"])
    assert np.array_equal(out["best_E"].cpu().numpy(), ref["best_E"])
    assert np.array_equal(out["final_x"].cpu().numpy().view(np.uint32), ref["final_x"])
    assert np.array_equal(out["flips"].cpu().numpy(), ref["flips"])


@pytest.mark.parametrize("dtype", ["int8", "fp32"])
def test_ptda_matches_oracle(da, inst, dtype):
    import oracle
    q = inst.sk_bimodal(128, 2) if dtype == "int8" else inst.sk_gaussian(96, 2)
    betas = inst.beta_geometric(0.2, 5.0, 8)
    ctx = da.da_create(q.Q)
    got = da.da_pt(ctx, betas, 12, 5, 6, swap_trace=True)
    ref = oracle.ptda(q.Q, betas, 12, L=5, seed=6, nthreads=NT)
    assert np.array_equal(got["swap_trace"], ref["swap_trace"])
    assert np.array_equal(got["temp_of"], ref["temp_of"])
    assert np.array_equal(got["swaps"], ref["swaps"])
    assert np.array_equal(got["best_x"], ref["x_best"])
    Eb = oracle.energy(q.Q, got["best_x"].reshape(-1, da.da_words(q.N))).reshape(5, 8)
    if dtype == "int8":
        assert np.array_equal(got["best_E"], ref["E_best"])
        assert np.array_equal(got["final_E"], ref["E_final"])
    else:
        assert np.allclose(got["best_E"], Eb, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("dtype", ["i8", "f32"])
def test_adaptive_ptda_matches_oracle(da, inst, dtype):
    """PTDA with the adaptive ladder: every exchange decision, the final ladder, the
    replicas' temperatures and best states agree with the oracle bit for bit."""
    import oracle
    q = inst.sk_bimodal(64, 9) if dtype == "i8" else inst.sk_gaussian(64, 9)
    b0 = inst.beta_geometric(0.05, 2.0 if dtype == "i8" else 4.0, 8)
    ref = oracle.ptda(q.Q, b0, 120, 6, 3, nthreads=NT, adapt_every=10, adapt_sweeps=80)
    ctx = da.da_create(q.Q)
    got = da.da_pt(ctx, b0, 120, 6, 3, swap_trace=True, adapt_every=10, adapt_sweeps=80)
    assert np.array_equal(got["betas"].view(np.uint32), ref["betas"].view(np.uint32))
    assert not np.array_equal(got["betas"], b0)
    assert np.array_equal(got["swap_trace"], ref["swap_trace"])
    assert np.array_equal(got["swaps"], ref["swaps"])
    assert np.array_equal(got["temp_of"], ref["temp_of"])
    assert np.array_equal(got["best_x"], ref["x_best"])
    with pytest.raises(da.DAError):
        da.da_pt(ctx, b0, 10, 2, 3, adapt_every=-1)


def test_ptda_c4b_shape(da, inst):
    """SK bimodal N = 512, 32 geometric betas in 0.2-5.0, exchange every sweep."""
    import oracle
    q = inst.sk_bimodal(512, 0)
    betas = inst.beta_geometric(0.2, 5.0, 32)
    ctx = da.da_create(q.Q)
    got = da.da_pt(ctx, betas, 3, 2, 1, swap_trace=True)
    ref = oracle.ptda(q.Q, betas, 3, L=2, seed=1, nthreads=NT)
    assert np.array_equal(got["swap_trace"], ref["swap_trace"])
    assert np.array_equal(got["best_E"], ref["E_best"])
    assert np.array_equal(got["temp_of"], ref["temp_of"])


@pytest.mark.parametrize("kind", ["int8", "fp32"])
def test_plain_form_matches_oracle(da, inst, kind):
    """The one-launch-per-step baseline draws the same numbers and uses the same fp32
    arithmetic (exact for integer couplings) and no recompute."""
    import oracle
    q = inst.sk_bimodal(100, 4) if kind == "int8" else inst.sk_gaussian(200, 4)
    beta = inst.beta_linear(0.1, 4.0, 600)
    ctx = da.da_create(q.Q)
    got = da.da_anneal_plain(ctx, beta, 0.5, 9, 21, trace=True)
    ref = oracle.da_anneal(q.Q, beta, R=9, seed=21, inc=0.5, recompute_every=0, trace=True, nthreads=NT)
    assert np.array_equal(got["trace"], ref["trace"])
    assert np.array_equal(got["final_x"], ref["x_final"])
    assert np.array_equal(got["best_x"], ref["x_best"])
    assert np.array_equal(got["flips"], ref["flips"])
    fast = da.da_anneal(ctx, beta, 0.5, 9, 21, recompute_every=0, trace=True)
    assert np.array_equal(fast["trace"], got["trace"])


def test_batched_launch_matches_single_instances(da, inst):
    """Mixed sizes and coupling types in one batched launch: every item equals its own
    da_anneal run (and, through it, the oracle) bit for bit."""
    import oracle
    rng = np.random.default_rng(0)
    jobs, refs = [], []
    sizes = [64, 128, 96, 256, 512, 1024, 300]
    for n, N in enumerate(sizes):
        q = inst.sk_bimodal(N, n) if n % 2 == 0 else inst.sk_gaussian(N, n)
        T = int(rng.integers(200, 900))
        beta = inst.beta_linear(0.1, 3.0, T)
        ctx = da.da_create(q.Q)
        R = int(rng.integers(3, 40))
        P = 0 if q.bimodal else 128
        jobs.append(dict(ctx=ctx, beta=beta, offset_inc=0.5, replicas=R, seed=100 + n, recompute_every=P, trace=True))
        refs.append(da.da_anneal(ctx, beta, 0.5, R, 100 + n, recompute_every=P, trace=True))
    outs, el = da.binding.da_batch_anneal(jobs)
    assert el > 0
    for o, r in zip(outs, refs):
        for k in ("trace", "final_x", "best_x", "flips", "final_E", "best_E", "max_drift"):
            assert np.array_equal(o[k], r[k]), k
    # one fp32 item against the oracle directly
    j = jobs[1]
    ref = oracle.da_anneal(inst.sk_gaussian(128, 1).Q, j["beta"], R=j["replicas"], seed=j["seed"], inc=0.5,
                           recompute_every=128, trace=True, nthreads=NT)
    assert np.array_equal(outs[1]["trace"], ref["trace"])


@pytest.mark.parametrize("staging,wpb", [(0, 1), (0, 4), (1, 2), (1, 8), (1, 16), (2, 1), (2, 4), (-1, 0)])
def test_batched_configurations_match_single_instances(da, inst, staging, wpb):
    """Every configuration the batched launch's tuner can choose (rows of W from L2 at 1 or 4
    warps per block, in the plain or the one-warp row order; W staged in shared memory with
    groups of 2, 8 or 16 replicas; the tuner itself) gives each item the results of its own
    da_anneal run, bit for bit.  Sizes that stage (V = 4 and V = 8 classes up to N = 221) and
    that do not, ragged replica counts."""
    rng = np.random.default_rng(7)
    jobs, refs = [], []
    sizes = [64, 100, 128, 200, 221, 256, 40, 1024, 90, 520]
    for n, N in enumerate(sizes):
        q = inst.sk_bimodal(N, 50 + n) if n % 2 == 0 else inst.sk_gaussian(N, 50 + n)
        T = int(rng.integers(150, 600))
        beta = inst.beta_linear(0.1, 3.0, T)
        if n >= 8:   # the DA's 16-bit couplers (da_quantize), beta divided by the scale
            Qi, scale = da.binding.da_quantize(inst.sk_gaussian(N, 50 + n).Q)
            ctx = da.da_create(Qi, da.DA_INT16)
            beta = (beta / scale).astype(np.float32)
            P = 0
        else:
            ctx = da.da_create(q.Q)
            P = 0 if q.bimodal else 100
        R = int(rng.integers(3, 23))
        jobs.append(dict(ctx=ctx, beta=beta, offset_inc=0.5, replicas=R, seed=300 + n, recompute_every=P,
                         trace=True))
        refs.append(da.da_anneal(ctx, beta, 0.5, R, 300 + n, recompute_every=P, trace=True))
    da.binding.da_batch_force(staging, wpb)
    try:
        outs, el = da.binding.da_batch_anneal(jobs)
        desc = da.binding.da_batch_describe()
    finally:
        da.binding.da_batch_force(-1, 0)
    assert el > 0
    if staging == 1:
        assert "shared memory" in desc, desc
    if staging == 2:
        assert "one-warp row order" in desc, desc
    for o, r in zip(outs, refs):
        for k in ("trace", "final_x", "best_x", "flips", "final_E", "best_E", "max_drift"):
            assert np.array_equal(o[k], r[k]), (k, desc)


def test_batched_recompute_with_and_without_shift_only_conversion(da, inst):
    """The batched kernel's warp-level exact recompute converts couplings to the fixed-point
    grid by a shift alone when every entry allows it (checked on the host), else through the
    rounding path: instances of both kinds (a tiny normal coupling 1e-30 and a subnormal one
    make the second) give their da_anneal results bit for bit."""
    jobs, refs = [], []
    for n, (N, tiny) in enumerate([(200, None), (200, 1e-30), (700, 1e-40), (1024, None)]):
        q = inst.sk_gaussian(N, 80 + n).Q.copy()
        if tiny is not None:
            q[0, 5] = np.float32(tiny)
            q[3, 3] = np.float32(-tiny)
        beta = inst.beta_linear(0.1, 6.0, 700)
        ctx = da.da_create(q)
        jobs.append(dict(ctx=ctx, beta=beta, offset_inc=0.0, replicas=9, seed=40 + n, recompute_every=64))
        refs.append(da.da_anneal(ctx, beta, 0.0, 9, 40 + n, recompute_every=64))
    outs, _ = da.binding.da_batch_anneal(jobs)
    for o, r in zip(outs, refs):
        for k in ("final_x", "best_x", "flips", "final_E", "best_E", "max_drift"):
            assert np.array_equal(o[k], r[k]), k


@pytest.mark.parametrize("N,R,kind", [(300, 40, "f32"), (97, 9, "i8"), (1500, 16, "f32"), (2100, 8, "i8")])
def test_tuned_launch_shape_keeps_results(da, inst, N, R, kind):
    """da_tune_shape picks the fastest launch shape for (instance, replicas) and every later
    anneal of that class uses it: the trajectories stay those of the oracle, bit for bit."""
    import oracle
    q = inst.sk_bimodal(N, 9) if kind == "i8" else inst.sk_gaussian(N, 9)
    ctx = da.da_create(q.Q)
    shape = da.binding.da_tune_shape(ctx, R, 64)
    assert shape["G"] in (1, 2, 4, 8) and 32 * shape["V"] * shape["G"] >= N, shape
    beta = inst.beta_linear(0.1, 4.0, 300)
    P = 0 if kind == "i8" else 64
    inc = 1.0 if kind == "i8" else 0.25
    got = da.da_anneal(ctx, beta, inc, R, 21, recompute_every=P, trace=True)
    ref = oracle.da_anneal(q.Q, beta, R=R, seed=21, inc=inc, recompute_every=P, trace=True, nthreads=NT)
    assert np.array_equal(got["trace"], ref["trace"]), shape
    assert np.array_equal(got["final_x"], ref["x_final"]), shape
    # a second context of the same class picks the tuned shape up from the process cache
    ctx2 = da.da_create(q.Q)
    got2 = da.da_anneal(ctx2, beta, inc, R, 21, recompute_every=P, trace=True)
    assert np.array_equal(got2["trace"], got["trace"])


@pytest.mark.parametrize("dtype", ["i8", "f32"])
def test_move_energy_percentiles_match_brute_force(da, inst, dtype):
    """The temperature grid's input: percentiles of the energy rises of all single-flip
    moves, against E(x xor e_i) - E(x) from the oracle's energy of every neighbour."""
    import oracle
    from paper_1806_08815_gb300 import tuning
    q = inst.sk_bimodal(40, 4) if dtype == "i8" else inst.sk_gaussian(40, 4)
    ctx = da.da_create(q.Q)
    rng = np.random.default_rng(2)
    X = rng.integers(0, 2, (6, q.N))
    up = []
    for x in X:
        E0 = oracle.energy(q.Q, oracle.pack(x[None]))[0]
        for i in range(q.N):
            y = x.copy()
            y[i] ^= 1
            d = oracle.energy(q.Q, oracle.pack(y[None]))[0] - E0
            if d > 0:
                up.append(d)
    qs = [0, 5, 10, 50, 80, 85, 100]
    got = da.binding.da_move_energy_percentiles(ctx, oracle.pack(X), qs)
    ref = np.percentile(np.array(up, dtype=np.float64), qs)
    if dtype == "i8":
        assert np.array_equal(got, ref)
    else:
        assert np.allclose(got, ref, rtol=1e-6, atol=1e-6)
    grid = tuning.temperature_grid(ctx, n_states=16)
    assert 0 < grid["T_low"][0] <= grid["T_low"][1] <= grid["T_high"][0] <= grid["T_high"][1]


def _int16_instance(inst, N, seed):
    """An SK-Gaussian instance in the DA's fixed-point precision (16-bit couplers)."""
    from paper_1806_08815_gb300 import binding
    Qi, scale = binding.da_quantize(inst.sk_gaussian(N, seed).Q)
    return Qi, scale


@pytest.mark.parametrize("N,shape", [(100, (0, 0, 0)), (100, (4, 1, 4)), (100, (4, 2, 2)), (256, (8, 1, 2)),
                                     (1024, (0, 0, 0)), (1024, (8, 4, 1)), (2100, (0, 0, 0))])
def test_int16_fixed_point_trajectories(da, inst, N, shape):
    """The fixed-point DA mode (16-bit couplers, 26-bit biases): bit-exact
    trajectories against the oracle's integer mode, over launch shapes."""
    import oracle
    Qi, scale = _int16_instance(inst, N, 5)
    assert np.abs(np.triu(Qi, 1)).max() <= 2 ** 15 - 1
    beta = (inst.beta_linear(0.1, 10.0, 1200) / scale).astype(np.float32)
    ctx = da.da_create(Qi, da.DA_INT16)
    if shape[0]:
        da.da_set_launch_shape(ctx, *shape)
    R = 7 if N <= 1024 else 3
    got = da.da_anneal(ctx, beta, 0.0, R, 8, trace=True)
    ref = oracle.da_anneal(Qi, beta, R=R, seed=8, inc=0.0, trace=True, nthreads=NT)
    _compare_anneal(got, ref, Qi, True)


def test_int16_draw_warp_pt_and_energies(da, inst):
    import oracle
    Qi, scale = _int16_instance(inst, 200, 6)
    ctx = da.da_create(Qi, da.DA_INT16)
    beta = (inst.beta_linear(0.1, 10.0, 800) / scale).astype(np.float32)
    da.binding.da_set_draw_warp(ctx, True)
    got = da.da_anneal(ctx, beta, 0.5 * scale, 5, 2, trace=True)
    ref = oracle.da_anneal(Qi, beta, R=5, seed=2, inc=np.float32(0.5 * scale), trace=True, nthreads=NT)
    _compare_anneal(got, ref, Qi, True)
    betas = (inst.beta_geometric(0.2, 5.0, 6) / scale).astype(np.float32)
    g = da.da_pt(ctx, betas, 10, 3, 4, swap_trace=True)
    r = oracle.ptda(Qi, betas, 10, L=3, seed=4, nthreads=NT)
    assert np.array_equal(g["swap_trace"], r["swap_trace"]) and np.array_equal(g["best_x"], r["x_best"])
    rng = np.random.default_rng(1)
    xp = oracle.pack(rng.integers(0, 2, (9, 200)))
    assert np.array_equal(da.da_energy(ctx, xp), oracle.energy(Qi, xp).astype(float))
    h = da.da_field_recompute(ctx, xp)
    for k in range(9):
        assert np.array_equal(h[k].astype(np.int64), oracle.fields_int(Qi, xp[k]) + np.diag(Qi))
    with pytest.raises(da.DAError):
        da.da_anneal_plain(ctx, beta, 0.0, 2, 0)


def test_bounded_wait_gives_up_instead_of_hanging(da):
    """The mbarrier wait of the pipelined kernels returns failure after its time limit
    when the arrival never comes (and success when it does), so a lost arrival ends a
    kernel with an error flag rather than a hung GPU."""
    ok, abandoned, ns = da.binding.da_diag_bounded_wait(2_000_000)
    assert ok == 1 and abandoned == 0
    assert 2_000_000 <= ns < 200_000_000


@pytest.mark.parametrize("dtype,shape", [("i8", (0, 0, 0)), ("f32", (0, 0, 0)), ("f32", (32, 4, 1))])
def test_largest_instances(da, inst, dtype, shape):
    """N = 8192 (the largest the library takes; G = 8 warps of 32 variables per lane) and
    N = 4096 on G = 4: bit-exact trajectories with a recompute inside the run."""
    import oracle
    N = 8192 if shape[0] == 0 else 4096
    q = inst.sk_bimodal(N, 1) if dtype == "i8" else inst.sk_gaussian(N, 1)
    beta = inst.beta_linear(0.1, 3.0 if dtype == "i8" else 9.0, 700)
    ctx = da.da_create(q.Q)
    if shape[0]:
        da.da_set_launch_shape(ctx, *shape)
    rec = 0 if dtype == "i8" else 512
    got = da.da_anneal(ctx, beta, 0.0, 3, 21, recompute_every=rec, trace=True)
    ref = oracle.da_anneal(q.Q, beta, R=3, seed=21, inc=0.0, recompute_every=rec, trace=True, nthreads=NT)
    _compare_anneal(got, ref, q.Q, dtype == "i8")


def test_read_bandwidth_probe(da):
    """The read-bandwidth probe the step kernel's roofline is stated against: an L2-resident
    buffer (64 MB) reads faster than one four times the L2 (512 MB), both at plausible
    rates for this GPU, and misaligned or empty buffers are refused."""
    import torch
    small = torch.zeros(64 << 20, dtype=torch.uint8, device="cuda")
    large = torch.zeros(512 << 20, dtype=torch.uint8, device="cuda")
    bw_l2 = max(da.binding.da_diag_read_bandwidth(small, 32) for _ in range(3))
    bw_hbm = max(da.binding.da_diag_read_bandwidth(large, 4) for _ in range(3))
    assert bw_l2 > 1.2 * bw_hbm, (bw_l2, bw_hbm)
    assert 1e12 < bw_hbm < 2e13 and bw_l2 < 1e14
    with pytest.raises(da.binding.DAError):
        da.binding.da_diag_read_bandwidth(small[1:17], 1)
    with pytest.raises(da.binding.DAError):
        da.binding.da_diag_read_bandwidth(small[:0], 1)
