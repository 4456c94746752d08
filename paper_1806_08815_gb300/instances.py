"""Seeded synthetic inputs: spin-glass instances and inverse-temperature schedules.

This module is the one both the CUDA library's tests/benchmarks and the CPU
oracle draw their inputs from.  It holds none of the annealer's arithmetic:
it draws couplings, writes them in the QUBO form the library takes (the
substitution s = 2x - 1 of the "Benchmarking Problems" section), and tabulates
beta schedules.

Instance classes follow the paper's "Benchmarking Problems" section:
bimodal couplings J_ij in {-1, +1} with equal probability, Gaussian couplings
N(0, 1), zero biases; complete graphs (SK) or a 2D torus with 4 neighbours.
The paper's own instances (Spin Glass Server, Biq Mac) are not available, so
these seeded draws stand in for them.

QUBO layout: an N x N row-major matrix whose upper triangle is read; Q_ii are
the linear terms and Q_ij (i < j) the couplings, E(x) = sum_i Q_ii x_i +
sum_{i<j} Q_ij x_i x_j, and H(s) = E(x) + C.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


@dataclass
class Instance:
    name: str
    N: int
    Q: np.ndarray        # int32 (bimodal) or float32 (Gaussian), N x N, upper triangle
    C: float             # constant: H(s) = E(x) + C
    J: np.ndarray        # Ising couplings, N x N upper triangle (float64)

    @property
    def bimodal(self) -> bool:
        return self.Q.dtype == np.int32


def _qubo_from_ising(J: np.ndarray, integer: bool):
    """Upper-triangular QUBO of H = -sum_{i<j} J_ij s_i s_j with s = 2x - 1."""
    N = J.shape[0]
    Ju = np.triu(J, 1)
    row = Ju.sum(axis=1) + Ju.sum(axis=0)          # sum_{j != i} J_ij
    C = -float(Ju.sum())
    if integer:
        Q = (-4 * Ju).astype(np.int64)
        Q[np.arange(N), np.arange(N)] = (2 * row).astype(np.int64)
        return Q.astype(np.int32), C
    Q = (-4.0 * Ju).astype(np.float32)
    Q[np.arange(N), np.arange(N)] = (2.0 * row).astype(np.float32)
    return Q, C


def sk_bimodal(N: int, seed: int) -> Instance:
    """Fully connected Ising spin glass, J_ij = +-1 iid; integer QUBO."""
    rng = np.random.default_rng([seed, 1, N])
    J = np.triu(rng.choice(np.array([-1.0, 1.0]), size=(N, N)), 1)
    Q, C = _qubo_from_ising(J, integer=True)
    return Instance(f"sk_bimodal_N{N}_s{seed}", N, Q, C, J)


def sk_gaussian(N: int, seed: int, scale: float | None = None) -> Instance:
    """Fully connected Ising spin glass, J_ij ~ N(0, 1) * scale (default 1/sqrt(N)),
    rounded to fp32; fp32 QUBO."""
    if scale is None:
        scale = 1.0 / math.sqrt(N)
    rng = np.random.default_rng([seed, 2, N])
    J = np.triu(rng.standard_normal((N, N)) * scale, 1).astype(np.float32).astype(np.float64)
    Q, C = _qubo_from_ising(J, integer=False)
    return Instance(f"sk_gaussian_N{N}_s{seed}", N, Q, C, J)


def _torus_edges(L: int):
    idx = np.arange(L * L).reshape(L, L)
    right = np.stack([idx.ravel(), np.roll(idx, -1, axis=1).ravel()], 1)
    down = np.stack([idx.ravel(), np.roll(idx, -1, axis=0).ravel()], 1)
    return np.concatenate([right, down])


def lattice2d(L: int, seed: int, gaussian: bool) -> Instance:
    """2D spin glass on an L x L torus (4 neighbours, 2 L^2 edges), kept dense."""
    N = L * L
    rng = np.random.default_rng([seed, 3 if gaussian else 4, L])
    e = _torus_edges(L)
    if gaussian:
        w = rng.standard_normal(len(e)).astype(np.float32).astype(np.float64)
    else:
        w = rng.choice(np.array([-1.0, 1.0]), size=len(e))
    J = np.zeros((N, N))
    a, b = np.minimum(e[:, 0], e[:, 1]), np.maximum(e[:, 0], e[:, 1])
    np.add.at(J, (a, b), w)      # L = 2 would create double edges; they add
    Q, C = _qubo_from_ising(J, integer=not gaussian)
    kind = "gaussian" if gaussian else "bimodal"
    return Instance(f"lattice2d_{kind}_L{L}_s{seed}", N, Q, C, J)


def erdos_renyi_bimodal(N: int, density: float, seed: int) -> Instance:
    """Bimodal couplings on a G(N, p) graph (the density study of the appendix)."""
    rng = np.random.default_rng([seed, 5, N, int(density * 1e6)])
    mask = rng.random((N, N)) < density
    J = np.triu(np.where(mask, rng.choice(np.array([-1.0, 1.0]), size=(N, N)), 0.0), 1)
    Q, C = _qubo_from_ising(J, integer=True)
    return Instance(f"er_bimodal_N{N}_p{density}_s{seed}", N, Q, C, J)


def random_qubo(N: int, seed: int, integer: bool, lo: int = -4, hi: int = 4) -> Instance:
    """Unstructured QUBO with all entries random (diagonal included), for tests."""
    rng = np.random.default_rng([seed, 6, N])
    if integer:
        Q = np.triu(rng.integers(lo, hi + 1, size=(N, N))).astype(np.int32)
    else:
        Q = np.triu(rng.standard_normal((N, N))).astype(np.float32)
    return Instance(f"random_qubo_N{N}_s{seed}", N, Q, 0.0, np.zeros((N, N)))


def beta_linear(b0: float, b1: float, T: int) -> np.ndarray:
    """beta_t = b0 + (b1 - b0) t / (T - 1) in fp64, stored as fp32."""
    if T == 1:
        return np.array([b0], dtype=np.float32)
    t = np.arange(T, dtype=np.float64)
    return (b0 + (b1 - b0) * t / (T - 1)).astype(np.float32)


def beta_geometric(b0: float, b1: float, T: int) -> np.ndarray:
    """beta_t = b0 (b1 / b0)^(t / (T - 1)) in fp64, stored as fp32."""
    if T == 1:
        return np.array([b0], dtype=np.float32)
    t = np.arange(T, dtype=np.float64)
    return (b0 * (b1 / b0) ** (t / (T - 1))).astype(np.float32)
