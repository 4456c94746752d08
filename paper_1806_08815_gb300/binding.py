"""Thin ctypes binding of the C ABI in include/da.h (argument marshalling only).

Every function here calls the CUDA library libda.so; there is no CPU path.
If the library has not been built, importing raises at the first call with
instructions, and on a machine without a CUDA device the library returns
DA_ECUDA, which is raised as DAError.

Names follow the C ABI: da_create, da_anneal, da_anneal_async, da_pt,
da_energy, da_field_recompute, da_set_launch_shape, da_destroy.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libda.so")

DA_INT8, DA_FP32, DA_INT16 = 0, 1, 2
STATUS = {0: "DA_OK", 1: "DA_EINVAL", 2: "DA_ENOMEM", 3: "DA_EBUDGET", 4: "DA_EBUSY",
          5: "DA_ETIMEOUT", 6: "DA_ECUDA", 7: "DA_ENOTREADY", 8: "DA_ECANCELED"}


class DAError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


_P = ctypes.c_void_p


class da_checkpoint(ctypes.Structure):
    _fields_ = [("x", _P), ("best_x", _P), ("fields", _P), ("scalars", _P)]


class da_result(ctypes.Structure):
    _fields_ = [("final_E", _P), ("best_E", _P), ("final_x", _P), ("best_x", _P),
                ("max_drift", _P), ("flips", _P), ("trace", _P), ("elapsed_s", ctypes.c_double)]


class da_dev_result(ctypes.Structure):
    _fields_ = [("final_E", _P), ("best_E", _P), ("final_x", _P), ("best_x", _P),
                ("max_drift", _P), ("flips", _P), ("trace", _P)]


class da_batch_item(ctypes.Structure):
    _fields_ = [("ctx", _P), ("beta", _P), ("steps", ctypes.c_int64), ("offset_inc", ctypes.c_float),
                ("replicas", ctypes.c_int32), ("seed", ctypes.c_uint64), ("recompute_every", ctypes.c_int64),
                ("out", ctypes.POINTER(da_result))]


class da_job(ctypes.Structure):
    _fields_ = [("Q", _P), ("N", ctypes.c_int64), ("dtype", ctypes.c_int), ("beta", _P), ("steps", ctypes.c_int64),
                ("offset_inc", ctypes.c_float), ("replicas", ctypes.c_int32), ("seed", ctypes.c_uint64),
                ("recompute_every", ctypes.c_int64)]


class da_pt_result(ctypes.Structure):
    _fields_ = [("final_E", _P), ("best_E", _P), ("best_x", _P), ("temp_of", _P),
                ("swaps", _P), ("swap_trace", _P), ("elapsed_s", ctypes.c_double)]


_lib = None


def lib() -> ctypes.CDLL:
    """Load libda.so (built by __graft_entry__.build() / paper_1806_08815_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with "
                          "`python -c 'import __graft_entry__ as g; g.build()'`")
    L = ctypes.CDLL(LIB_PATH)
    i32, i64, u64, f32 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_float
    L.da_version.restype = ctypes.c_int
    L.da_words.argtypes = [i64]
    L.da_words.restype = i64
    L.da_last_error.restype = ctypes.c_char_p
    L.da_create.argtypes = [_P, i64, ctypes.c_int, ctypes.POINTER(_P)]
    L.da_destroy.argtypes = [_P]
    L.da_destroy.restype = None
    L.da_ctx_info.argtypes = [_P, ctypes.POINTER(i64), ctypes.POINTER(ctypes.c_int)]
    L.da_set_launch_shape.argtypes = [_P, i32, i32, i32]
    L.da_set_draw_warp.argtypes = [_P, i32]
    L.da_set_draw_warp.restype = ctypes.c_int
    L.da_anneal.argtypes = [_P, _P, i64, f32, i32, u64, i64, ctypes.POINTER(da_result)]
    L.da_anneal_async.argtypes = [_P, _P, i64, f32, i32, u64, i64, ctypes.POINTER(da_dev_result), _P]
    L.da_pt.argtypes = [_P, _P, i32, i64, i32, f32, u64, ctypes.POINTER(da_pt_result)]
    L.da_pt_adaptive.argtypes = [_P, _P, i32, i64, i32, f32, u64, i64, i64, ctypes.POINTER(da_pt_result)]
    L.da_pt_adaptive.restype = ctypes.c_int
    L.da_energy.argtypes = [_P, _P, i32, _P]
    L.da_field_recompute.argtypes = [_P, _P, i32, _P]
    L.da_profile_enable.argtypes = [_P, i32]
    L.da_profile_read.argtypes = [_P, ctypes.POINTER(i64), ctypes.POINTER(ctypes.c_double)]
    L.da_profile_enable.restype = ctypes.c_int
    L.da_profile_read.restype = ctypes.c_int
    L.da_server_create.argtypes = [i64, i32, ctypes.POINTER(_P)]
    L.da_submit.argtypes = [_P, ctypes.POINTER(da_job), ctypes.POINTER(_P)]
    L.da_poll.argtypes = [_P, i32, ctypes.POINTER(da_result)]
    L.da_req_free.argtypes = [_P]
    L.da_req_free.restype = None
    L.da_diag_read_bandwidth.argtypes = [_P, i64, i32, ctypes.POINTER(ctypes.c_double)]
    L.da_diag_read_bandwidth.restype = ctypes.c_int
    L.da_cancel.argtypes = [_P]
    L.da_cancel.restype = ctypes.c_int
    L.da_diag_fail_alloc.argtypes = [i32, i32]
    L.da_diag_fail_alloc.restype = ctypes.c_int
    L.da_diag_live_allocations.argtypes = [ctypes.POINTER(i64), ctypes.POINTER(i64), ctypes.POINTER(i64)]
    L.da_diag_live_allocations.restype = ctypes.c_int
    L.da_server_destroy.argtypes = [_P]
    L.da_server_destroy.restype = None
    L.da_server_resident.argtypes = [_P, i32]
    L.da_server_resident.restype = ctypes.c_int
    L.da_server_stats.argtypes = [_P, ctypes.POINTER(i64), ctypes.POINTER(i64), ctypes.POINTER(i64)]
    for name in ("da_server_create", "da_submit", "da_poll", "da_server_stats"):
        getattr(L, name).restype = ctypes.c_int
    L.da_batch_anneal.argtypes = [ctypes.POINTER(da_batch_item), i32, ctypes.POINTER(ctypes.c_double)]
    L.da_batch_anneal.restype = ctypes.c_int
    L.da_anneal_segment.argtypes = [_P, _P, i64, i64, i64, f32, i32, u64, i64, ctypes.POINTER(da_checkpoint),
                                    ctypes.POINTER(da_checkpoint), ctypes.POINTER(da_result)]
    L.da_anneal_segment.restype = ctypes.c_int
    L.da_tune_shape.argtypes = [_P, i32, i64] + [ctypes.POINTER(i32)] * 4
    L.da_tune_shape.restype = ctypes.c_int
    L.da_batch_describe.argtypes = [ctypes.c_char_p, i64]
    L.da_batch_describe.restype = ctypes.c_int
    L.da_batch_force.argtypes = [i32, i32]
    L.da_batch_force.restype = ctypes.c_int
    L.da_anneal_plain.argtypes = [_P, _P, i64, f32, i32, u64, ctypes.POINTER(da_result)]
    L.da_anneal_plain.restype = ctypes.c_int
    L.da_anneal_static.argtypes = [_P, _P, i64, i64, _P, i64, f32, i32, u64, ctypes.POINTER(da_dev_result), _P]
    L.da_anneal_static.restype = ctypes.c_int
    L.da_static_pitch.argtypes = [i64]
    L.da_static_pitch.restype = i64
    L.da_tts_bootstrap.argtypes = [_P, _P, i32, ctypes.c_double, ctypes.c_double, i32, u64, _P]
    L.da_tts_bootstrap.restype = ctypes.c_int
    L.da_move_energy_percentiles.argtypes = [_P, _P, i32, _P, i32, _P]
    L.da_move_energy_percentiles.restype = ctypes.c_int
    L.da_quantize.argtypes = [_P, i64, i32, i32, _P, ctypes.POINTER(ctypes.c_double)]
    L.da_quantize.restype = ctypes.c_int
    L.da_percentiles.argtypes = [_P, i64, _P, i32, _P]
    L.da_percentiles.restype = ctypes.c_int
    L.da_diag_bounded_wait.argtypes = [i64, _P]
    L.da_diag_bounded_wait.restype = ctypes.c_int
    L.da_diag_log_uniform.argtypes = [_P, _P, i64]
    L.da_diag_accept_log.argtypes = [_P, _P, _P, _P, i64]
    L.da_diag_log_uniform.restype = ctypes.c_int
    L.da_diag_accept_log.restype = ctypes.c_int
    L.da_diag_fixed.argtypes = [_P, _P, _P, _P, i64]
    L.da_diag_scaled.argtypes = [_P, _P, _P, _P, i64]
    L.da_diag_fixed.restype = ctypes.c_int
    L.da_diag_scaled.restype = ctypes.c_int
    L.da_diag_expf.argtypes = [_P, _P, i64]
    L.da_diag_philox.argtypes = [_P, _P, i64]
    for name in ("da_diag_expf", "da_diag_philox", "da_create", "da_ctx_info", "da_set_launch_shape", "da_anneal", "da_anneal_async", "da_pt",
                 "da_energy", "da_field_recompute"):
        getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def _check(status: int):
    if status != 0:
        raise DAError(status, lib().da_last_error().decode(errors="replace"))


def _ptr(a):
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data_as(_P)
    return _P(int(a.data_ptr()))      # torch tensor (device or host)


def da_words(N: int) -> int:
    return int(lib().da_words(int(N)))


class Context:
    """One QUBO instance resident on the device (wraps da_ctx*)."""

    def __init__(self, handle, N: int, dtype: int):
        self.handle = handle
        self.N = N
        self.dtype = dtype

    def __del__(self):
        try:
            da_destroy(self)
        except Exception:
            pass


def da_create(Q: np.ndarray, dtype: int | None = None) -> Context:
    """Q: N x N upper-triangular QUBO, integer (-> DA_INT8, or DA_INT16 when asked) or
    float32 (-> DA_FP32)."""
    Q = np.asarray(Q)
    N = Q.shape[0]
    if Q.ndim != 2 or Q.shape[1] != N:
        raise ValueError("Q must be N x N")
    if dtype is None:
        dtype = DA_INT8 if np.issubdtype(Q.dtype, np.integer) else DA_FP32
    Qc = np.ascontiguousarray(Q, dtype=np.float32 if dtype == DA_FP32 else np.int32)
    h = _P()
    _check(lib().da_create(_ptr(Qc), N, dtype, ctypes.byref(h)))
    return Context(h, N, dtype)


def da_destroy(ctx: Context):
    if ctx.handle:
        lib().da_destroy(ctx.handle)
        ctx.handle = None


def da_set_launch_shape(ctx: Context, V: int = 0, G: int = 0, rpb: int = 0):
    _check(lib().da_set_launch_shape(ctx.handle, V, G, rpb))


def da_anneal(ctx: Context, beta: np.ndarray, offset_inc: float, replicas: int, seed: int,
              recompute_every: int = 0, trace: bool = False) -> dict:
    """Blocking anneal; returns numpy arrays (see da_result in include/da.h)."""
    b = np.ascontiguousarray(beta, dtype=np.float32)
    R, T, W = int(replicas), b.size, da_words(ctx.N)
    out = dict(final_E=np.zeros(R), best_E=np.zeros(R), final_x=np.zeros((R, W), np.uint32),
               best_x=np.zeros((R, W), np.uint32), max_drift=np.zeros(R), flips=np.zeros(R, np.int64))
    if trace:
        out["trace"] = np.zeros((R, T), np.int32)
    res = da_result(*(_ptr(out.get(k)) for k in ("final_E", "best_E", "final_x", "best_x", "max_drift",
                                                  "flips", "trace")), 0.0)
    _check(lib().da_anneal(ctx.handle, _ptr(b), T, float(offset_inc), R, int(seed) & (2 ** 64 - 1),
                           int(recompute_every), ctypes.byref(res)))
    out["elapsed_s"] = res.elapsed_s
    return out


def da_anneal_plain(ctx: Context, beta: np.ndarray, offset_inc: float, replicas: int, seed: int,
                    trace: bool = False) -> dict:
    """The plain one-launch-per-step baseline form (see da_anneal_plain in include/da.h)."""
    b = np.ascontiguousarray(beta, dtype=np.float32)
    R, T, W = int(replicas), b.size, da_words(ctx.N)
    out = dict(final_E=np.zeros(R), best_E=np.zeros(R), final_x=np.zeros((R, W), np.uint32),
               best_x=np.zeros((R, W), np.uint32), max_drift=np.zeros(R), flips=np.zeros(R, np.int64))
    if trace:
        out["trace"] = np.zeros((R, T), np.int32)
    res = da_result(*(_ptr(out.get(k)) for k in ("final_E", "best_E", "final_x", "best_x", "max_drift",
                                                  "flips", "trace")), 0.0)
    _check(lib().da_anneal_plain(ctx.handle, _ptr(b), T, float(offset_inc), R, int(seed) & (2 ** 64 - 1),
                                 ctypes.byref(res)))
    out["elapsed_s"] = res.elapsed_s
    return out


def da_anneal_segment(ctx: Context, beta: np.ndarray, t0: int, t1: int, offset_inc: float, replicas: int,
                      seed: int, recompute_every: int = 0, checkpoint: dict | None = None):
    """Steps [t0, t1) of an anneal over the whole schedule `beta`, from `checkpoint` (None: from
    x = 0, t0 = 0).  Returns (results as da_anneal would give after step t1, checkpoint)."""
    b = np.ascontiguousarray(beta, dtype=np.float32)
    R, W, N = int(replicas), da_words(ctx.N), ctx.N
    out = dict(final_E=np.zeros(R), best_E=np.zeros(R), final_x=np.zeros((R, W), np.uint32),
               best_x=np.zeros((R, W), np.uint32), max_drift=np.zeros(R), flips=np.zeros(R, np.int64))
    res = da_result(*(_ptr(out.get(k)) for k in ("final_E", "best_E", "final_x", "best_x", "max_drift",
                                                  "flips", "trace")), 0.0)
    ck = dict(x=np.zeros((R, W), np.uint32), best_x=np.zeros((R, W), np.uint32),
              fields=np.zeros((R, N), np.float32 if ctx.dtype == DA_FP32 else np.int32),
              scalars=np.zeros((R, 4), np.int64))
    ck_out = da_checkpoint(_ptr(ck["x"]), _ptr(ck["best_x"]), _ptr(ck["fields"]), _ptr(ck["scalars"]))
    ck_in = None
    if checkpoint is not None:
        keep = {k: np.ascontiguousarray(checkpoint[k]) for k in ("x", "best_x", "fields", "scalars")}
        ck_in = da_checkpoint(*(_ptr(keep[k]) for k in ("x", "best_x", "fields", "scalars")))
    _check(lib().da_anneal_segment(ctx.handle, _ptr(b), b.size, int(t0), int(t1), float(offset_inc), R,
                                   int(seed) & (2 ** 64 - 1), int(recompute_every),
                                   ctypes.byref(ck_in) if ck_in is not None else None, ctypes.byref(ck_out),
                                   ctypes.byref(res)))
    out["elapsed_s"] = res.elapsed_s
    return out, ck


def da_anneal_async(ctx: Context, beta_dev, steps: int, offset_inc: float, replicas: int, seed: int,
                    recompute_every: int, out: dict, stream) -> None:
    """Queue an anneal on `stream` (torch.cuda.Stream or raw handle); `beta_dev` and the
    tensors in `out` (keys as da_dev_result) are device tensors owned by the caller."""
    res = da_dev_result(*(_ptr(out.get(k)) for k in ("final_E", "best_E", "final_x", "best_x", "max_drift",
                                                      "flips", "trace")))
    handle = getattr(stream, "cuda_stream", stream)
    _check(lib().da_anneal_async(ctx.handle, _ptr(beta_dev), int(steps), float(offset_inc), int(replicas),
                                 int(seed) & (2 ** 64 - 1), int(recompute_every), ctypes.byref(res),
                                 _P(int(handle) if handle else 0)))


def da_pt(ctx: Context, betas: np.ndarray, sweeps: int, ladders: int, seed: int, offset_inc: float = 0.0,
          swap_trace: bool = False, adapt_every: int = 0, adapt_sweeps: int = 0) -> dict:
    """PTDA; with adapt_every > 0 the ladder adapts (da_pt_adaptive) and out["betas"] is
    the final ladder."""
    b = np.array(betas, dtype=np.float32)
    K, L, W = b.size, int(ladders), da_words(ctx.N)
    out = dict(final_E=np.zeros((L, K)), best_E=np.zeros((L, K)), best_x=np.zeros((L, K, W), np.uint32),
               temp_of=np.zeros((L, K), np.int32), swaps=np.zeros((L, max(K - 1, 0)), np.int64))
    if swap_trace:
        out["swap_trace"] = np.zeros((L, sweeps, max(K - 1, 0)), np.uint8)
    res = da_pt_result(*(_ptr(out.get(k)) for k in ("final_E", "best_E", "best_x", "temp_of", "swaps",
                                                     "swap_trace")), 0.0)
    if adapt_every:
        _check(lib().da_pt_adaptive(ctx.handle, _ptr(b), K, int(sweeps), L, float(offset_inc),
                                    int(seed) & (2 ** 64 - 1), int(adapt_every), int(adapt_sweeps),
                                    ctypes.byref(res)))
    else:
        _check(lib().da_pt(ctx.handle, _ptr(b), K, int(sweeps), L, float(offset_inc), int(seed) & (2 ** 64 - 1),
                           ctypes.byref(res)))
    out["betas"] = b
    out["elapsed_s"] = res.elapsed_s
    return out


def da_set_draw_warp(ctx: Context, on: bool) -> None:
    _check(lib().da_set_draw_warp(ctx.handle, 1 if on else 0))


def da_energy(ctx: Context, x: np.ndarray) -> np.ndarray:
    xs = np.ascontiguousarray(np.atleast_2d(x), dtype=np.uint32)
    E = np.zeros(xs.shape[0])
    _check(lib().da_energy(ctx.handle, _ptr(xs), xs.shape[0], _ptr(E)))
    return E


def da_field_recompute(ctx: Context, x: np.ndarray) -> np.ndarray:
    xs = np.ascontiguousarray(np.atleast_2d(x), dtype=np.uint32)
    h = np.zeros((xs.shape[0], ctx.N), np.float32 if ctx.dtype == DA_FP32 else np.int32)
    _check(lib().da_field_recompute(ctx.handle, _ptr(xs), xs.shape[0], _ptr(h)))
    return h


def da_diag_expf(x: np.ndarray) -> np.ndarray:
    xs = np.ascontiguousarray(x, dtype=np.float32).ravel()
    y = np.empty_like(xs)
    _check(lib().da_diag_expf(_ptr(xs), _ptr(y), xs.size))
    return y


def da_diag_philox(ctr_key: np.ndarray) -> np.ndarray:
    """ctr_key: [n, 6] uint32 (c0..c3, k0, k1) -> [n, 4] uint32."""
    ck = np.ascontiguousarray(ctr_key, dtype=np.uint32).reshape(-1, 6)
    out = np.empty((ck.shape[0], 4), np.uint32)
    _check(lib().da_diag_philox(_ptr(ck), _ptr(out), ck.shape[0]))
    return out


def da_profile_enable(ctx: Context, on: bool = True):
    _check(lib().da_profile_enable(ctx.handle, 1 if on else 0))


def da_profile_read(ctx: Context):
    """(launches, summed device ms) of the step-kernel launches since the last read."""
    n = ctypes.c_int64()
    ms = ctypes.c_double()
    _check(lib().da_profile_read(ctx.handle, ctypes.byref(n), ctypes.byref(ms)))
    return n.value, ms.value


def da_tts_bootstrap(hits, runs, tau: float, q: float, B: int, seed: int) -> np.ndarray:
    """Algorithm 3: B bootstrap samples of TTS_q over the instances (hits/runs per instance)."""
    y = np.ascontiguousarray(hits, dtype=np.int64)
    r = np.ascontiguousarray(runs, dtype=np.int64)
    out = np.zeros(int(B))
    _check(lib().da_tts_bootstrap(_ptr(y), _ptr(r), int(y.size), float(tau), float(q), int(B),
                                  int(seed) & (2 ** 64 - 1), _ptr(out)))
    return out


def da_move_energy_percentiles(ctx: Context, x: np.ndarray, q) -> np.ndarray:
    """Percentiles of the energy rises of all single-flip moves from the states x."""
    xs = np.ascontiguousarray(np.atleast_2d(x), dtype=np.uint32)
    qs = np.ascontiguousarray(q, dtype=np.float64)
    out = np.zeros(qs.size)
    _check(lib().da_move_energy_percentiles(ctx.handle, _ptr(xs), xs.shape[0], _ptr(qs), qs.size, _ptr(out)))
    return out


def da_quantize(Q: np.ndarray, coupler_max: int = 2 ** 15 - 1, bias_max: int = 2 ** 25 - 1):
    """The DA's fixed-point scaling: (Qint int32 N x N upper triangle, scale)."""
    Qc = np.ascontiguousarray(Q, dtype=np.float32)
    N = Qc.shape[0]
    out = np.zeros((N, N), np.int32)
    sc = ctypes.c_double()
    _check(lib().da_quantize(_ptr(Qc), N, int(coupler_max), int(bias_max), _ptr(out), ctypes.byref(sc)))
    return out, sc.value


def da_percentiles(v, q) -> np.ndarray:
    vs = np.ascontiguousarray(v, dtype=np.float64)
    qs = np.ascontiguousarray(q, dtype=np.float64)
    out = np.zeros(qs.size)
    _check(lib().da_percentiles(_ptr(vs), vs.size, _ptr(qs), qs.size, _ptr(out)))
    return out


def da_diag_bounded_wait(ns: int) -> np.ndarray:
    out = np.zeros(3, np.int64)
    _check(lib().da_diag_bounded_wait(int(ns), _ptr(out)))
    return out


def da_diag_log_uniform(w: np.ndarray) -> np.ndarray:
    ws = np.ascontiguousarray(w, dtype=np.uint32).ravel()
    L = np.empty(ws.size, np.float32)
    _check(lib().da_diag_log_uniform(_ptr(ws), _ptr(L), ws.size))
    return L


def da_diag_accept_log(delta: np.ndarray, beta: np.ndarray, w: np.ndarray):
    """(decision, in_band) of the warp-specialised step for each trial."""
    d = np.ascontiguousarray(delta, dtype=np.float32).ravel()
    b = np.ascontiguousarray(np.broadcast_to(beta, d.shape), dtype=np.float32).ravel()
    ws = np.ascontiguousarray(w, dtype=np.uint32).ravel()
    out = np.empty(d.size, np.uint8)
    _check(lib().da_diag_accept_log(_ptr(d), _ptr(b), _ptr(ws), _ptr(out), d.size))
    return (out & 1).astype(bool), (out & 2).astype(bool)


def da_diag_fixed(w: np.ndarray, S: np.ndarray):
    """(integer-path, intrinsic-path) round(w 2^S) as the kernels compute it."""
    ws = np.ascontiguousarray(w, dtype=np.float32).ravel()
    Ss = np.ascontiguousarray(np.broadcast_to(S, ws.shape), dtype=np.int32).ravel()
    got = np.empty(ws.size, np.int64)
    ref = np.empty(ws.size, np.int64)
    _check(lib().da_diag_fixed(_ptr(ws), _ptr(Ss), _ptr(got), _ptr(ref), ws.size))
    return got, ref


def da_diag_scaled(v: np.ndarray, S: np.ndarray):
    """(integer-path, intrinsic-path) fl32(v) 2^-S as the kernels compute it."""
    vs = np.ascontiguousarray(v, dtype=np.int64).ravel()
    Ss = np.ascontiguousarray(np.broadcast_to(S, vs.shape), dtype=np.int32).ravel()
    got = np.empty(vs.size, np.float32)
    ref = np.empty(vs.size, np.float32)
    _check(lib().da_diag_scaled(_ptr(vs), _ptr(Ss), _ptr(got), _ptr(ref), vs.size))
    return got, ref


def da_static_pitch(N: int) -> int:
    return int(lib().da_static_pitch(int(N)))


def da_anneal_static(W_dev, diag_dev, N: int, ldw: int, beta_dev, steps: int, offset_inc: float, replicas: int,
                     seed: int, out: dict, stream) -> None:
    """The allocation-free integer anneal (see da_anneal_static in include/da.h); every
    argument that is an array is a device tensor owned by the caller."""
    res = da_dev_result(*(_ptr(out.get(k)) for k in ("final_E", "best_E", "final_x", "best_x", "max_drift",
                                                      "flips", "trace")))
    handle = getattr(stream, "cuda_stream", stream)
    _check(lib().da_anneal_static(_ptr(W_dev), _ptr(diag_dev), int(N), int(ldw), _ptr(beta_dev), int(steps),
                                  float(offset_inc), int(replicas), int(seed) & (2 ** 64 - 1), ctypes.byref(res),
                                  _P(int(handle) if handle else 0)))


def da_batch_anneal(jobs: list) -> tuple:
    """jobs: dicts with ctx, beta, offset_inc, replicas, seed, recompute_every (optional), trace
    (optional).  Returns (list of result dicts as from da_anneal, device seconds)."""
    n = len(jobs)
    arr = (da_batch_item * n)()
    keep = []
    outs = []
    for i, j in enumerate(jobs):
        ctx = j["ctx"]
        b = np.ascontiguousarray(j["beta"], dtype=np.float32)
        R, T, W = int(j["replicas"]), b.size, da_words(ctx.N)
        out = dict(final_E=np.zeros(R), best_E=np.zeros(R), final_x=np.zeros((R, W), np.uint32),
                   best_x=np.zeros((R, W), np.uint32), max_drift=np.zeros(R), flips=np.zeros(R, np.int64))
        if j.get("trace"):
            out["trace"] = np.zeros((R, T), np.int32)
        res = da_result(*(_ptr(out.get(k)) for k in ("final_E", "best_E", "final_x", "best_x", "max_drift",
                                                      "flips", "trace")), 0.0)
        keep += [b, res]
        outs.append(out)
        arr[i] = da_batch_item(ctx.handle, _ptr(b), T, float(j.get("offset_inc", 0.0)), R,
                               int(j["seed"]) & (2 ** 64 - 1), int(j.get("recompute_every", 0)),
                               ctypes.pointer(res))
    el = ctypes.c_double()
    _check(lib().da_batch_anneal(arr, n, ctypes.byref(el)))
    return outs, el.value


def da_tune_shape(ctx: Context, replicas: int, probe_steps: int = 256) -> dict:
    """Time every launch shape for this instance and replica count; the fastest is used from now
    on by every context of the process with the same coupling type, N and replica count."""
    v = [ctypes.c_int32() for _ in range(4)]
    _check(lib().da_tune_shape(ctx.handle, int(replicas), int(probe_steps), *(ctypes.byref(x) for x in v)))
    return dict(V=v[0].value, G=v[1].value, rpb=v[2].value, draw_warp=v[3].value)


def da_batch_describe() -> str:
    """The configuration each class of the last da_batch_anneal on this thread used."""
    buf = ctypes.create_string_buffer(8192)
    _check(lib().da_batch_describe(buf, len(buf)))
    return buf.value.decode()


def da_batch_force(staging: int = -1, warps_per_block: int = 0) -> None:
    """Override the batched launch's tuner (staging -1 auto / 0 L2 / 1 shared memory)."""
    _check(lib().da_batch_force(int(staging), int(warps_per_block)))


class Server:
    """A request loop on the current device (wraps da_server*)."""

    def __init__(self, hbm_budget_bytes: int, max_requests: int = 1024):
        h = _P()
        _check(lib().da_server_create(int(hbm_budget_bytes), int(max_requests), ctypes.byref(h)))
        self.handle = h

    def close(self):
        if self.handle:
            lib().da_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def resident(self, max_n: int) -> None:
        """Requests of at most max_n variables run as one resident launch (0: all chunked)."""
        _check(lib().da_server_resident(self.handle, int(max_n)))

    def stats(self):
        a, b, c = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _check(lib().da_server_stats(self.handle, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
        return dict(completed=a.value, kernel_launches=b.value, bytes_in_use=c.value)


class Request:
    def __init__(self, handle, keep, N, R, T, trace=False):
        self.handle, self.keep, self.N, self.R, self.T = handle, keep, N, R, T

    def __del__(self):
        try:
            if self.handle:
                lib().da_req_free(self.handle)
                self.handle = None
        except Exception:
            pass


def da_submit(srv: Server, Q: np.ndarray, beta: np.ndarray, offset_inc: float, replicas: int, seed: int,
              recompute_every: int = 0, dtype: int | None = None) -> Request:
    """Queue a request (integer Q -> DA_INT8, or DA_INT16 when asked; float32 Q -> DA_FP32)."""
    Q = np.asarray(Q)
    N = Q.shape[0]
    if dtype is None:
        dtype = DA_INT8 if np.issubdtype(Q.dtype, np.integer) else DA_FP32
    Qc = np.ascontiguousarray(Q, dtype=np.float32 if dtype == DA_FP32 else np.int32)
    b = np.ascontiguousarray(beta, dtype=np.float32)
    job = da_job(_ptr(Qc), N, dtype, _ptr(b), b.size, float(offset_inc), int(replicas), int(seed) & (2 ** 64 - 1),
                 int(recompute_every))
    h = _P()
    _check(lib().da_submit(srv.handle, ctypes.byref(job), ctypes.byref(h)))
    return Request(h, (Qc, b), N, int(replicas), b.size)


def da_poll(req: Request, timeout_us: int = 0):
    """Result dict once finished, None while not ready (or on timeout)."""
    R, W = req.R, da_words(req.N)
    out = dict(final_E=np.zeros(R), best_E=np.zeros(R), final_x=np.zeros((R, W), np.uint32),
               best_x=np.zeros((R, W), np.uint32), max_drift=np.zeros(R), flips=np.zeros(R, np.int64))
    res = da_result(*(_ptr(out.get(k)) for k in ("final_E", "best_E", "final_x", "best_x", "max_drift",
                                                  "flips", "trace")), 0.0)
    st = lib().da_poll(req.handle, int(timeout_us), ctypes.byref(res))
    if st in (5, 7):
        return None
    _check(st)
    out["latency_s"] = res.elapsed_s
    return out


def da_cancel(req: Request) -> None:
    """Cancel a queued or running request (da_poll then raises DA_ECANCELED)."""
    _check(lib().da_cancel(req.handle))


def da_diag_fail_alloc(after: int, count: int) -> None:
    """Make the library's device allocations after the next `after` fail, `count` times
    (host-side injection; count = 0 disarms)."""
    _check(lib().da_diag_fail_alloc(int(after), int(count)))


def da_diag_live_allocations() -> dict:
    a, b, c = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    _check(lib().da_diag_live_allocations(ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
    return dict(count=a.value, bytes=b.value, injected=c.value)


def da_diag_read_bandwidth(buf_dev, passes: int) -> float:
    """Read bandwidth in bytes/s of a device tensor (L2 for one that fits L2, else HBM)."""
    sec = ctypes.c_double()
    nbytes = int(buf_dev.numel() * buf_dev.element_size())
    _check(lib().da_diag_read_bandwidth(_ptr(buf_dev), nbytes, int(passes), ctypes.byref(sec)))
    return nbytes * int(passes) / sec.value
