"""CPU oracle of the Digital Annealer method (arXiv:1806.08815).

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow, serial C reference
(``da_oracle.c``) that the CUDA library is checked against; only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may load
it.  It shares no code with ``paper_1806_08815_gb300``; the only module both
sides use is the seeded instance generator (``paper_1806_08815_gb300.instances``),
which holds none of the method's arithmetic.

The wrappers below only marshal numpy arrays to the C functions.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "da_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

MODE_INT, MODE_F32, MODE_F64 = 0, 1, 2

_lib = None


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (no fast-math, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "da_oracle.h"))):
        tmp = _LIB + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-O2", "-std=c11", "-Wall", "-ffp-contract=off", "-fno-fast-math",
               "-fopenmp", "-shared", "-fPIC", _SRC, "-o", tmp, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        i64, i32, u32, u64, f32 = (ctypes.c_int64, ctypes.c_int32, ctypes.c_uint32,
                                   ctypes.c_uint64, ctypes.c_float)
        L.orc_philox4x32_10.argtypes = [P, P, P]
        L.orc_expf.argtypes = [f32]
        L.orc_expf.restype = f32
        L.orc_expf_batch.argtypes = [P, P, i64]
        L.orc_uniform.argtypes = [u32]
        L.orc_uniform.restype = f32
        L.orc_energy_int.argtypes = [i64, P, P]
        L.orc_energy_int.restype = i64
        L.orc_energy_f64.argtypes = [i64, P, P]
        L.orc_energy_f64.restype = ctypes.c_double
        L.orc_ising_to_qubo.argtypes = [i64, P, P, P, P]
        L.orc_ising_energy.argtypes = [i64, P, P, P]
        L.orc_ising_energy.restype = ctypes.c_double
        L.orc_brute_force_f64.argtypes = [i64, P, P, P, P]
        L.orc_fields_int.argtypes = [i64, P, P, P]
        L.orc_recompute_f32.argtypes = [i64, P, P, P, P, P]
        L.orc_recompute_energy_f32.argtypes = [i64, P, P]
        L.orc_recompute_energy_f32.restype = ctypes.c_double
        L.orc_da_anneal.argtypes = [i64, ctypes.c_int, P, P, i64, f32, i32, u64, u32, i64,
                                    P, P, P, P, P, P, P, ctypes.c_int]
        L.orc_da_one_step.argtypes = [i64, ctypes.c_int, P, P, u32, f32, f32, u64, u32, u32, P]
        L.orc_sa_anneal.argtypes = [i64, P, P, i64, i32, u64, P, P, ctypes.c_int]
        L.orc_ptda.argtypes = [i64, ctypes.c_int, P, P, i32, i64, f32, i32, u64,
                               P, P, P, P, P, P, ctypes.c_int]
        L.orc_ptda_adaptive.argtypes = [i64, ctypes.c_int, P, P, i32, i64, f32, i32, u64, i64, i64, P,
                                        P, P, P, P, P, P, ctypes.c_int]
        L.orc_pt_adapt.argtypes = [i32, P, P, i64, P]
        L.orc_pt_adapt.restype = None
        L.orc_tts_bootstrap.argtypes = [P, P, i32, ctypes.c_double, ctypes.c_double, i32, u64, P]
        L.orc_beta_samples.argtypes = [ctypes.c_double, ctypes.c_double, i64, u64, P]
        L.orc_beta_samples.restype = None
        L.orc_quantize.argtypes = [i64, P, i32, i32, P, P]
        L.orc_percentile.argtypes = [P, i64, ctypes.c_double]
        L.orc_percentile.restype = ctypes.c_double
        _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _check(rc, name):
    if rc != 0:
        raise RuntimeError(f"{name} failed with status {rc}")


def words(N: int) -> int:
    return (N + 31) // 32


def pack(x: np.ndarray) -> np.ndarray:
    """Bit-pack a {0,1} vector (or the rows of a matrix): bit i%32 of word i//32."""
    x = np.atleast_2d(np.asarray(x, dtype=np.uint8))
    R, N = x.shape
    out = np.zeros((R, words(N)), dtype=np.uint32)
    for i in range(N):
        out[:, i // 32] |= x[:, i].astype(np.uint32) << np.uint32(i % 32)
    return out


def unpack(w: np.ndarray, N: int) -> np.ndarray:
    w = np.atleast_2d(np.asarray(w, dtype=np.uint32))
    i = np.arange(N)
    return ((w[:, i // 32] >> (i % 32).astype(np.uint32)) & 1).astype(np.uint8)


def philox(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def expf(x) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.float32).ravel()
    y = np.empty_like(x)
    lib().orc_expf_batch(_p(x), _p(y), x.size)
    return y


def uniform(r: int) -> float:
    return lib().orc_uniform(int(r) & 0xFFFFFFFF)


def energy(Q: np.ndarray, x: np.ndarray) -> float:
    """Exact energy of the bit-packed state(s) x: int64 for integer Q, fp64 otherwise."""
    N = Q.shape[0]
    xs = np.atleast_2d(np.ascontiguousarray(x, dtype=np.uint32))
    out = []
    if Q.dtype == np.int32:
        Qc = np.ascontiguousarray(Q)
        for row in xs:
            row = np.ascontiguousarray(row)
            out.append(lib().orc_energy_int(N, _p(Qc), _p(row)))
        return np.array(out, dtype=np.int64)
    Qc = np.ascontiguousarray(Q, dtype=np.float32)
    for row in xs:
        row = np.ascontiguousarray(row)
        out.append(lib().orc_energy_f64(N, _p(Qc), _p(row)))
    return np.array(out, dtype=np.float64)


def ising_to_qubo(J: np.ndarray, hb: np.ndarray):
    N = J.shape[0]
    Jc = np.ascontiguousarray(J, dtype=np.float64)
    hc = np.ascontiguousarray(hb, dtype=np.float64)
    Q = np.zeros((N, N), dtype=np.float64)
    C = ctypes.c_double()
    _check(lib().orc_ising_to_qubo(N, _p(Jc), _p(hc), _p(Q), ctypes.byref(C)), "ising_to_qubo")
    return Q, C.value


def ising_energy(J, hb, s) -> float:
    N = J.shape[0]
    Jc = np.ascontiguousarray(J, dtype=np.float64)
    hc = np.ascontiguousarray(hb, dtype=np.float64)
    sc = np.ascontiguousarray(s, dtype=np.int8)
    return lib().orc_ising_energy(N, _p(Jc), _p(hc), _p(sc))


def brute_force(Q: np.ndarray):
    """(E_min, number of minimisers, one minimiser as a {0,1} vector)."""
    N = Q.shape[0]
    Qc = np.ascontiguousarray(Q, dtype=np.float64)
    E = ctypes.c_double()
    cnt = ctypes.c_int64()
    arg = np.zeros(1, dtype=np.uint32)
    _check(lib().orc_brute_force_f64(N, _p(Qc), ctypes.byref(E), ctypes.byref(cnt), _p(arg)), "brute_force")
    return E.value, cnt.value, unpack(arg, N)[0]


def fields_int(Q: np.ndarray, x: np.ndarray) -> np.ndarray:
    N = Q.shape[0]
    Qc = np.ascontiguousarray(Q, dtype=np.int32)
    xc = np.ascontiguousarray(x, dtype=np.uint32)
    h = np.zeros(N, dtype=np.int64)
    _check(lib().orc_fields_int(N, _p(Qc), _p(xc), _p(h)), "fields_int")
    return h


def recompute_f32(Q: np.ndarray, x: np.ndarray):
    """(h fp32, exact int64 sums, scale S) of the fixed-point field recompute."""
    N = Q.shape[0]
    Qc = np.ascontiguousarray(Q, dtype=np.float32)
    xc = np.ascontiguousarray(x, dtype=np.uint32)
    h = np.zeros(N, dtype=np.float32)
    s = np.zeros(N, dtype=np.int64)
    S = ctypes.c_int32()
    _check(lib().orc_recompute_f32(N, _p(Qc), _p(xc), _p(h), _p(s), ctypes.byref(S)), "recompute_f32")
    return h, s, S.value


def recompute_energy_f32(Q: np.ndarray, x: np.ndarray) -> float:
    N = Q.shape[0]
    Qc = np.ascontiguousarray(Q, dtype=np.float32)
    xc = np.ascontiguousarray(x, dtype=np.uint32)
    return lib().orc_recompute_energy_f32(N, _p(Qc), _p(xc))


def da_anneal(Q: np.ndarray, beta: np.ndarray, R: int, seed: int, inc: float = 0.0,
              mode: int | None = None, replica_base: int = 0, recompute_every: int = 0,
              trace: bool = False, accepted: bool = False, nthreads: int = 1) -> dict:
    """Run Algorithm 2 R times from x = 0 (see da_oracle.h)."""
    N = Q.shape[0]
    if mode is None:
        mode = MODE_INT if Q.dtype == np.int32 else MODE_F32
    Qc = np.ascontiguousarray(Q, dtype=np.int32 if mode == MODE_INT else np.float32)
    b = np.ascontiguousarray(beta, dtype=np.float32)
    T = b.size
    W = words(N)
    out = dict(E_final=np.zeros(R), E_best=np.zeros(R),
               x_final=np.zeros((R, W), np.uint32), x_best=np.zeros((R, W), np.uint32),
               flips=np.zeros(R, np.int64))
    tr = np.zeros((R, T), np.int32) if trace else None
    ac = np.zeros((R, T), np.int32) if accepted else None
    rc = lib().orc_da_anneal(N, mode, _p(Qc), _p(b), T, float(inc), R, int(seed) & (2**64 - 1),
                             int(replica_base), int(recompute_every),
                             _p(out["E_final"]), _p(out["E_best"]), _p(out["x_final"]),
                             _p(out["x_best"]), _p(out["flips"]), _p(tr), _p(ac), int(nthreads))
    _check(rc, "da_anneal")
    if trace:
        out["trace"] = tr
    if accepted:
        out["accepted"] = ac
    return out


def da_one_step(Q, x, m, beta, inc, seed, t, replica, mode=None):
    N = Q.shape[0]
    if mode is None:
        mode = MODE_INT if Q.dtype == np.int32 else MODE_F32
    Qc = np.ascontiguousarray(Q, dtype=np.int32 if mode == MODE_INT else np.float32)
    xc = np.ascontiguousarray(x, dtype=np.uint32)
    na = ctypes.c_int32()
    k = lib().orc_da_one_step(N, mode, _p(Qc), _p(xc), int(m), float(beta), float(inc),
                              int(seed), int(t), int(replica), ctypes.byref(na))
    if k < -1:
        raise RuntimeError("da_one_step failed")
    return k, na.value


def sa_anneal(Q, beta, R, seed, nthreads=1):
    N = Q.shape[0]
    Qc = np.ascontiguousarray(Q, dtype=np.float32)
    b = np.ascontiguousarray(beta, dtype=np.float32)
    E = np.zeros(R)
    xb = np.zeros((R, words(N)), np.uint32)
    _check(lib().orc_sa_anneal(N, _p(Qc), _p(b), b.size, R, int(seed), _p(E), _p(xb), int(nthreads)),
           "sa_anneal")
    return dict(E_best=E, x_best=xb)


def pt_adapt(betas, accepted, proposals):
    """One update of the adaptive PTDA ladder (ends fixed, gaps towards equal acceptance)."""
    b = np.ascontiguousarray(betas, dtype=np.float32)
    a = np.ascontiguousarray(accepted, dtype=np.int64)
    out = np.zeros_like(b)
    lib().orc_pt_adapt(int(b.size), _p(b), _p(a), int(proposals), _p(out))
    return out


def ptda(Q, betas, sweeps, L, seed, inc=0.0, mode=None, nthreads=1, adapt_every=0, adapt_sweeps=0):
    """PTDA; with adapt_every > 0 the ladder adapts every adapt_every sweeps up to sweep
    adapt_sweeps, and out["betas"] is the final ladder."""
    N = Q.shape[0]
    if mode is None:
        mode = MODE_INT if Q.dtype == np.int32 else MODE_F32
    Qc = np.ascontiguousarray(Q, dtype=np.int32 if mode == MODE_INT else np.float32)
    b = np.ascontiguousarray(betas, dtype=np.float32)
    K = b.size
    out = dict(E_final=np.zeros((L, K)), E_best=np.zeros((L, K)),
               x_best=np.zeros((L, K, words(N)), np.uint32), temp_of=np.zeros((L, K), np.int32),
               swaps=np.zeros((L, max(K - 1, 0)), np.int64),
               swap_trace=np.zeros((L, sweeps, max(K - 1, 0)), np.uint8))
    out["betas"] = b.copy()
    rc = lib().orc_ptda_adaptive(N, mode, _p(Qc), _p(b), K, int(sweeps), float(inc), L, int(seed),
                                 int(adapt_every), int(adapt_sweeps), _p(out["betas"]),
                                 _p(out["E_final"]), _p(out["E_best"]), _p(out["x_best"]), _p(out["temp_of"]),
                                 _p(out["swaps"]), _p(out["swap_trace"]), int(nthreads))
    _check(rc, "ptda")
    return out


def tts_bootstrap(hits, runs, tau, q, B, seed):
    """Algorithm 3: B bootstrap samples of the q-th percentile of the TTS over instances."""
    y = np.ascontiguousarray(hits, dtype=np.int64)
    r = np.ascontiguousarray(runs, dtype=np.int64)
    out = np.zeros(int(B))
    _check(lib().orc_tts_bootstrap(_p(y), _p(r), int(y.size), float(tau), float(q), int(B), int(seed), _p(out)),
           "tts_bootstrap")
    return out


def beta_samples(a, b, n, seed):
    out = np.zeros(int(n))
    lib().orc_beta_samples(float(a), float(b), int(n), int(seed), _p(out))
    return out


def percentile(v, q):
    w = np.array(v, dtype=np.float64)
    return lib().orc_percentile(_p(w), int(w.size), float(q))


def quantize(Q, coupler_max=2 ** 15 - 1, bias_max=2 ** 25 - 1):
    """The DA's fixed-point scaling: (Qint int32, scale)."""
    Qc = np.ascontiguousarray(Q, dtype=np.float32)
    N = Qc.shape[0]
    out = np.zeros((N, N), np.int32)
    sc = np.zeros(1)
    _check(lib().orc_quantize(N, _p(Qc), int(coupler_max), int(bias_max), _p(out), _p(sc)), "quantize")
    return out, float(sc[0])
