"""The seeded input generators behind every parity case and workload: the
structure of each instance family (couplings, the Ising-to-QUBO diagonal,
graph degrees and densities, the SK scaling) and of the beta schedules, as the
benchmarking section's instance classes define them.  CPU only."""
import math

import numpy as np
import pytest

from paper_1806_08815_gb300 import instances


def _upper(J):
    return J[np.triu_indices(J.shape[0], 1)]


def test_sk_bimodal_couplings_and_diagonal():
    N = 97
    inst = instances.sk_bimodal(N, 4)
    assert inst.Q.dtype == np.int32 and inst.bimodal
    J = inst.J
    assert np.all(np.tril(J) == 0)
    assert set(np.unique(_upper(J))) == {-1.0, 1.0}
    Q = inst.Q.astype(np.int64)
    assert np.array_equal(np.triu(Q, 1), np.triu(-4 * J, 1).astype(np.int64))   # q_ij = -4 J_ij
    row = J.sum(1) + J.sum(0)
    assert np.array_equal(np.diag(Q), (2 * row).astype(np.int64))             # q_ii = 2 sum_j J_ij
    assert np.abs(np.diag(Q)).max() <= 2 * (N - 1)
    assert np.all(np.tril(Q, -1) == 0)


def test_sk_gaussian_scale_and_precision():
    N = 400
    inst = instances.sk_gaussian(N, 1)
    assert inst.Q.dtype == np.float32 and not inst.bimodal
    u = _upper(inst.J)
    # J ~ N(0, 1/N): the sample variance of N(N-1)/2 draws, within 5 standard errors
    n = u.size
    var = u.var()
    assert abs(var * N - 1.0) < 5 * math.sqrt(2.0 / n)
    assert abs(u.mean()) < 5 / math.sqrt(n * N)
    assert np.array_equal(u, u.astype(np.float32).astype(np.float64))          # fp32 values
    assert np.array_equal(_upper(inst.Q.astype(np.float64)), (-4.0 * u).astype(np.float32).astype(np.float64))


@pytest.mark.parametrize("L,gaussian", [(3, False), (8, True), (12, False)])
def test_lattice2d_is_a_four_neighbour_torus(L, gaussian):
    inst = instances.lattice2d(L, 2, gaussian)
    N = L * L
    J = inst.J
    S = (J != 0) | (J.T != 0)
    assert np.all(S.sum(1) == 4)                    # every site has 4 neighbours
    assert np.count_nonzero(np.triu(S, 1)) == 2 * N  # 2 L^2 edges
    for i in range(N):
        r, c = divmod(i, L)
        nb = {((r + 1) % L) * L + c, ((r - 1) % L) * L + c, r * L + (c + 1) % L, r * L + (c - 1) % L}
        assert set(np.flatnonzero(S[i])) == nb


@pytest.mark.parametrize("p", [0.1, 0.5, 0.9])
def test_erdos_renyi_density(p):
    N = 300
    inst = instances.erdos_renyi_bimodal(N, p, 3)
    u = _upper(inst.J)
    n = u.size
    k = np.count_nonzero(u)
    assert abs(k - p * n) < 5 * math.sqrt(n * p * (1 - p))
    assert set(np.unique(u[u != 0])) == {-1.0, 1.0}


def test_generators_are_seeded():
    a, b, c = instances.sk_gaussian(64, 7), instances.sk_gaussian(64, 7), instances.sk_gaussian(64, 8)
    assert np.array_equal(a.Q, b.Q) and not np.array_equal(a.Q, c.Q)
    a, b = instances.erdos_renyi_bimodal(64, 0.3, 1), instances.erdos_renyi_bimodal(64, 0.3, 1)
    assert np.array_equal(a.Q, b.Q)


@pytest.mark.parametrize("T", [1, 2, 1000])
def test_beta_schedules(T):
    lin = instances.beta_linear(0.1, 10.0, T)
    geo = instances.beta_geometric(0.2, 5.0, T)
    assert lin.dtype == np.float32 and lin.size == T and geo.size == T
    assert lin[0] == np.float32(0.1) and geo[0] == np.float32(0.2)
    if T > 1:
        assert lin[-1] == np.float32(10.0) and geo[-1] == np.float32(5.0)
        assert np.all(np.diff(lin) > 0) and np.all(np.diff(geo) > 0)
        # geometric: constant ratio between neighbours (up to fp32 rounding)
        r = geo[1:].astype(np.float64) / geo[:-1].astype(np.float64)
        assert np.allclose(r, (5.0 / 0.2) ** (1.0 / (T - 1)), rtol=1e-6)
