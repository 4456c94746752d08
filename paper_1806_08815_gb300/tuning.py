"""Parameter tuning of the DA (appendix "Parameters"; Sec. IV's time to solution).

- temperature_grid: the search ranges of the low and high temperatures from the
  distribution of the energy rises of proposed single-flip moves (the 5th-10th
  and 80th-85th percentiles), computed by da_move_energy_percentiles over
  uniformly random states.
- tts_distribution: Algorithm 3, the bootstrap distribution of TTS_q over a set
  of instances (da_tts_bootstrap).
- best_sweep_count: the number of sweeps whose TTS distribution has the lowest
  mean, with that distribution's mean and 5th / 95th percentiles per candidate.
Glue only: the statistics run in libda (host) and the fields on the GPU.
"""
from __future__ import annotations

import numpy as np

from . import binding


def temperature_grid(ctx, n_states: int = 64, seed: int = 0, low=(5.0, 10.0), high=(80.0, 85.0)) -> dict:
    """Search ranges (T_low, T_high) in energy units, from n_states uniformly random states."""
    rng = np.random.default_rng([seed, 7])
    w = binding.da_words(ctx.N)
    x = rng.integers(0, 2 ** 32, size=(n_states, w), dtype=np.uint64).astype(np.uint32)
    if ctx.N % 32:
        x[:, -1] &= np.uint32((1 << (ctx.N % 32)) - 1)
    p = binding.da_move_energy_percentiles(ctx, x, [*low, *high])
    return {"T_low": (float(p[0]), float(p[1])), "T_high": (float(p[2]), float(p[3])),
            "percentiles": {"low": tuple(low), "high": tuple(high)}}


def tts_distribution(hits, runs, tau: float, q: float = 50.0, B: int = 5000, seed: int = 0) -> np.ndarray:
    """B bootstrap samples of TTS_q (seconds if tau is the time per run in seconds)."""
    return binding.da_tts_bootstrap(hits, runs, tau, q, B, seed)


def best_sweep_count(results: dict, q: float = 50.0, B: int = 5000, seed: int = 0):
    """results: {sweeps: (hits[I], runs[I], tau)} for several sweep counts.  Returns
    (best sweep count, {sweeps: {"mean", "p5", "p95"}}) with the TTS_q distribution of each."""
    stats = {}
    for sweeps, (hits, runs, tau) in results.items():
        s = tts_distribution(hits, runs, tau, q, B, seed)
        p5, p95 = binding.da_percentiles(s, [5.0, 95.0])
        stats[sweeps] = {"mean": float(np.mean(s)), "p5": float(p5), "p95": float(p95)}
    best = min(stats, key=lambda k: stats[k]["mean"])
    return best, stats
