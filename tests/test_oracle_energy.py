"""Pins of the oracle's energies, Ising <-> QUBO map, brute force and field recompute.

Each check compares against something other than the oracle's own formula:
the Ising Hamiltonian of Eq. 4 evaluated directly, an independent numpy
enumeration, closed-form ground states, exact rational arithmetic.
"""
import itertools
from fractions import Fraction

import numpy as np
import pytest

from paper_1806_08815_gb300 import instances


def _E_numpy(Q, x):
    """x^T triu(Q) x, the QUBO energy by matrix algebra (fp64 / int64)."""
    Qu = np.triu(Q.astype(np.float64 if Q.dtype != np.int32 else np.int64))
    x = x.astype(Qu.dtype)
    return x @ Qu @ x


@pytest.mark.parametrize("N", [5, 9, 16])
def test_ising_to_qubo_constant(orc, N):
    rng = np.random.default_rng(N)
    J = np.triu(rng.standard_normal((N, N)), 1)
    hb = rng.standard_normal(N)
    Q, C = orc.ising_to_qubo(J, hb)
    assert np.all(np.tril(Q, -1) == 0)
    for _ in range(50):
        x = rng.integers(0, 2, N)
        s = 2 * x - 1
        H = orc.ising_energy(J, hb, s)
        # direct evaluation of Eq. 4
        H_direct = -sum(J[i, j] * s[i] * s[j] for i in range(N) for j in range(i + 1, N)) - hb @ s
        assert H == pytest.approx(H_direct, abs=1e-9)
        assert H == pytest.approx(_E_numpy(Q, x) + C, abs=1e-9)


def test_generator_qubo_matches_oracle_map(orc):
    for inst in [instances.sk_bimodal(12, 3), instances.sk_gaussian(12, 4), instances.lattice2d(4, 5, True),
                 instances.lattice2d(4, 6, False)]:
        Q, C = orc.ising_to_qubo(inst.J, np.zeros(inst.N))
        assert np.allclose(Q, inst.Q.astype(np.float64), rtol=1e-6, atol=1e-6)
        assert C == pytest.approx(inst.C, abs=1e-9)
        if inst.bimodal:
            assert np.array_equal(Q.astype(np.int64), inst.Q.astype(np.int64))


def test_energy_matches_numpy(orc):
    for inst in [instances.random_qubo(37, 1, True), instances.sk_bimodal(40, 2)]:
        rng = np.random.default_rng(7)
        X = rng.integers(0, 2, (20, inst.N))
        E = orc.energy(inst.Q, orc.pack(X))
        assert E.dtype == np.int64
        for e, x in zip(E, X):
            assert e == _E_numpy(inst.Q, x)
    inst = instances.sk_gaussian(33, 3)
    X = np.random.default_rng(8).integers(0, 2, (20, inst.N))
    E = orc.energy(inst.Q, orc.pack(X))
    for e, x in zip(E, X):
        assert e == pytest.approx(_E_numpy(inst.Q, x), rel=1e-12, abs=1e-12)


def test_delta_e_identity_and_fields(orc):
    """E(x xor e_k) - E(x) = (1 - 2 x_k)(Q_kk + h_k) with h = W x, for every k."""
    inst = instances.random_qubo(23, 11, True)
    rng = np.random.default_rng(3)
    W = np.triu(inst.Q.astype(np.int64), 1)
    W = W + W.T
    for _ in range(10):
        x = rng.integers(0, 2, inst.N)
        h = orc.fields_int(inst.Q, orc.pack(x)[0])
        assert np.array_equal(h, W @ x)
        E0 = _E_numpy(inst.Q, x)
        for k in range(inst.N):
            y = x.copy()
            y[k] ^= 1
            assert _E_numpy(inst.Q, y) - E0 == (1 - 2 * x[k]) * (inst.Q[k, k] + h[k])


@pytest.mark.parametrize("N", [4, 7, 11])
def test_brute_force_matches_enumeration(orc, N):
    for integer in (True, False):
        inst = instances.random_qubo(N, N, integer)
        Emin, cnt, arg = orc.brute_force(inst.Q.astype(np.float64))
        Es = [_E_numpy(inst.Q, np.array(b)) for b in itertools.product([0, 1], repeat=N)]
        ref = min(Es)
        assert Emin == pytest.approx(ref, abs=1e-9)
        assert cnt == sum(abs(e - ref) <= 1e-9 * (abs(ref) + 1) for e in Es)
        assert _E_numpy(inst.Q, arg) == pytest.approx(ref, abs=1e-9)


@pytest.mark.parametrize("N", [6, 13, 20])
def test_brute_force_ferromagnet_closed_form(orc, N):
    """All J_ij = +1: the ground states are all-up and all-down, H = -N(N-1)/2."""
    J = np.triu(np.ones((N, N)), 1)
    Q, C = orc.ising_to_qubo(J, np.zeros(N))
    Emin, cnt, arg = orc.brute_force(Q)
    assert Emin + C == -N * (N - 1) / 2
    assert cnt == 2
    assert arg.sum() in (0, N)


def test_brute_force_planted_state(orc):
    """Mattis glass J_ij = xi_i xi_j: the ground states are xi and -xi."""
    N = 14
    xi = np.random.default_rng(5).choice([-1, 1], N)
    J = np.triu(np.outer(xi, xi), 1).astype(np.float64)
    Q, C = orc.ising_to_qubo(J, np.zeros(N))
    Emin, cnt, arg = orc.brute_force(Q)
    assert cnt == 2 and Emin + C == -N * (N - 1) / 2
    s = 2 * arg.astype(int) - 1
    assert np.array_equal(s, xi) or np.array_equal(s, -xi)


def _exact_recompute(Q, x, S):
    """The fixed-point recompute of the effective fields from its definition, in
    exact integers: round(Q_ii 2^S) + sum_{x_j = 1} round(W_ij 2^S)."""
    N = Q.shape[0]
    W = np.triu(Q.astype(np.float32), 1)
    W = W + W.T
    scale = Fraction(2) ** S
    out = []
    for i in range(N):
        s = round(Fraction(float(Q[i, i])) * scale)      # Python round: half to even, as llrintf
        for j in range(N):
            if x[j]:
                s += round(Fraction(float(W[i, j])) * scale)
        out.append(s)
    return out


def test_recompute_exact_definition(orc):
    inst = instances.sk_gaussian(40, 9)
    rng = np.random.default_rng(2)
    x = rng.integers(0, 2, inst.N)
    g, sums, S = orc.recompute_f32(inst.Q, orc.pack(x)[0])
    # the scale: max(|W|, |Q_ii|) < 2^e, 2^L >= N + 1, S = 62 - L - e
    amax = np.abs(inst.Q).max()
    e = int(np.frexp(amax)[1])
    L = int(np.ceil(np.log2(inst.N + 1)))
    assert S == 62 - L - e
    assert list(sums) == _exact_recompute(inst.Q, x, S)
    # g is the fp32 rounding of the exact fixed-point value
    for i in range(inst.N):
        assert g[i] == np.float32(float(Fraction(int(sums[i])) / (Fraction(2) ** S)))
    # and the fixed-point value is within (N + 1) 2^-(S+1) of the real Q_ii + sum_j W_ij x_j
    W = np.triu(inst.Q, 1).astype(np.float64)
    real = np.diag(inst.Q).astype(np.float64) + (W + W.T) @ x
    assert np.all(np.abs(sums / 2.0 ** S - real) <= (inst.N + 1) * 2.0 ** -(S + 1) + 1e-15 * np.abs(real))


def test_recompute_integer_valued_is_exact(orc):
    inst = instances.random_qubo(50, 4, True, -100, 100)
    Qf = inst.Q.astype(np.float32)
    x = np.random.default_rng(6).integers(0, 2, inst.N)
    g, sums, S = orc.recompute_f32(Qf, orc.pack(x)[0])
    ref = orc.fields_int(inst.Q, orc.pack(x)[0]) + np.diag(inst.Q)
    assert np.array_equal(g.astype(np.int64), ref)
    E = orc.recompute_energy_f32(Qf, orc.pack(x)[0])
    assert E == orc.energy(inst.Q, orc.pack(x))[0]


def test_recompute_energy_matches_exact_energy(orc):
    inst = instances.sk_gaussian(60, 3)
    X = np.random.default_rng(7).integers(0, 2, (10, inst.N))
    for x in X:
        E = orc.recompute_energy_f32(inst.Q, orc.pack(x)[0])
        assert E == pytest.approx(orc.energy(inst.Q, orc.pack(x))[0], rel=1e-13, abs=1e-13)


def test_recompute_energy_is_the_rounded_exact_fixed_point_sum(orc):
    """E = sum_{x_i=1} (round(Q_ii 2^S) + sums_i) / 2^(S+1), rounded once to fp64."""
    for inst in (instances.sk_gaussian(50, 8), instances.lattice2d(6, 2, True)):
        rng = np.random.default_rng(11)
        for _ in range(5):
            x = rng.integers(0, 2, inst.N)
            _, sums, S = orc.recompute_f32(inst.Q, orc.pack(x)[0])
            scale = Fraction(2) ** S
            exact = sum(round(Fraction(float(inst.Q[i, i])) * scale) + int(sums[i])
                        for i in range(inst.N) if x[i])
            assert orc.recompute_energy_f32(inst.Q, orc.pack(x)[0]) == float(Fraction(exact) / (2 * scale))


@pytest.mark.parametrize("kind", ["sk", "lattice", "diag_binds"])
def test_quantize_scales_to_the_hardware_limits(orc, kind):
    """The DA's fixed-point scaling: the binding limit is reached exactly, every
    entry is within 1/2 of the scaled value, and the quantized energy is the
    scaled energy up to the summed rounding (exact bound, on random states)."""
    from paper_1806_08815_gb300 import instances
    if kind == "sk":
        Q = instances.sk_gaussian(200, 1).Q
    elif kind == "lattice":
        Q = instances.lattice2d(12, 1, True).Q
    else:
        Q = instances.sk_gaussian(60, 2).Q.copy()
        np.fill_diagonal(Q, np.diag(Q) * 3000)
    Qi, s = orc.quantize(Q)
    off = np.triu(np.ones(Q.shape, bool), 1)
    qmax = np.abs(Qi[off]).max()
    dmax = np.abs(np.diag(Qi)).max()
    assert qmax <= 2 ** 15 - 1 and dmax <= 2 ** 25 - 1
    assert qmax == 2 ** 15 - 1 or dmax == 2 ** 25 - 1
    err = Qi - s * np.triu(Q).astype(np.float64)
    assert np.abs(err).max() <= 0.5
    assert np.all(np.tril(Qi, -1) == 0)
    rng = np.random.default_rng(4)
    X = rng.integers(0, 2, (20, Q.shape[0]))
    xp = orc.pack(X)
    Ei = orc.energy(Qi, xp)
    Ef = orc.energy(Q, xp)
    bound = np.array([np.abs(err)[np.ix_(x == 1, x == 1)][np.triu_indices(x.sum())].sum() for x in X])
    assert np.all(np.abs(Ei - s * Ef) <= bound + 1e-6 * np.abs(s * Ef) + 1e-6)


def test_library_quantize_equals_oracle(orc):
    from paper_1806_08815_gb300 import build, binding, instances
    build.build()
    for Q in (instances.sk_gaussian(150, 3).Q, instances.random_qubo(70, 2, False).Q, np.zeros((5, 5), np.float32)):
        a, sa = binding.da_quantize(Q)
        b, sb = orc.quantize(Q)
        assert np.array_equal(a, b) and sa == sb
