"""Python binding of libqmccpw (C-ABI in include/qmccpw.h).

Argument marshalling only: every function forwards to the C entry point of the
same name; all computation runs in the library's CUDA kernels.  PyTorch is
used, where a caller wants it, for device memory and streams (pass
``torch.cuda.Stream.cuda_stream`` as a stream handle).

The library is loaded from ``paper_2209_11337_gb300/_lib/libqmccpw.so``
(built by ``paper_2209_11337_gb300.build``); importing this module does not
build it, and every call raises ``QmcCpwError`` if it is missing.  There is no
CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libqmccpw.so")

# ---- constants mirrored from include/qmccpw.h --------------------------------
QMCCPW_OK = 0
QMCCPW_ERR_INVALID_ARG = 1
QMCCPW_ERR_OOM = 2
QMCCPW_ERR_CUDA = 3
QMCCPW_ERR_TIMEOUT = 4
QMCCPW_NOT_READY = 5
QMCCPW_ERR_UNSUPPORTED = 6

QMCCPW_D_LIMIT = 1024
QMCCPW_R_LIMIT = 4096

QMCCPW_ARITH_ASIAN_CALL = 0
QMCCPW_BINARY_ASIAN = 1
QMCCPW_LOOKBACK_FIXED_CALL = 2
QMCCPW_GEOMETRIC_ASIAN_CALL = 3

QMCCPW_BB = 0
QMCCPW_PCA = 1
QMCCPW_STD = 2
QMCCPW_BB_LEAD = 3
QMCCPW_PCA_LEAD = 4

QMCCPW_FP64 = 0
QMCCPW_MIXED = 1
QMCCPW_MIXED_TC_BF16X3 = 2
QMCCPW_MIXED_TC_TF32X3 = 3

#: the symbols include/qmccpw.h declares
EXPORTS = (
    "qmccpw_plan", "qmccpw_greeks", "qmccpw_greeks_batch", "qmccpw_batch_create",
    "qmccpw_batch_launch", "qmccpw_batch_results", "qmccpw_batch_device_results",
    "qmccpw_batch_launch_count", "qmccpw_batch_set_timing", "qmccpw_batch_timing",
    "qmccpw_batch_use_graph", "qmccpw_batch_segment_timing", "qmccpw_batch_free",
    "qmccpw_selftest_bounded_wait", "qmccpw_sobol_points",
    "qmccpw_point_values", "qmccpw_greeks_noalloc", "qmccpw_server_start", "qmccpw_submit", "qmccpw_poll",
    "qmccpw_wait", "qmccpw_server_get_stats", "qmccpw_server_stop", "qmccpw_autotune", "qmccpw_tuning_get",
    "qmccpw_tuning_set", "qmccpw_free", "qmccpw_last_error",
    "qmccpw_version", "qmccpw_measure_pipe_peaks", "qmccpw_batch_scatter_replicates", "qmccpw_replicate_stats",
    "qmccpw_basket_greeks", "qmccpw_basket_point_values",
)


class QmcCpwError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"qmccpw error {code}: {msg}")
        self.code = code


# ---- structures ---------------------------------------------------------------
class qmccpw_plan_desc(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int32), ("d_max", ctypes.c_int32), ("r_max", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("seed", ctypes.c_uint64), ("stream", ctypes.c_void_p),
                ("workspace_bytes", ctypes.c_uint64)]


class qmccpw_option(ctypes.Structure):
    _fields_ = [("type", ctypes.c_int32), ("d", ctypes.c_int32), ("K", ctypes.c_double), ("T", ctypes.c_double)]


class qmccpw_market(ctypes.Structure):
    _fields_ = [("S0", ctypes.c_double), ("r", ctypes.c_double), ("sigma", ctypes.c_double)]


class qmccpw_result(ctypes.Structure):
    _fields_ = [("mean", ctypes.c_double * 4), ("se", ctypes.c_double * 4),
                ("per_replicate", ctypes.POINTER(ctypes.c_double))]


QMCCPW_ASSETS_MAX = 8


class qmccpw_basket(ctypes.Structure):
    _fields_ = [("type", ctypes.c_int32), ("d", ctypes.c_int32), ("m", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("K", ctypes.c_double), ("T", ctypes.c_double), ("S0", ctypes.c_double), ("r", ctypes.c_double),
                ("sigma", ctypes.c_double), ("weight", ctypes.c_double * QMCCPW_ASSETS_MAX),
                ("spot", ctypes.c_double * QMCCPW_ASSETS_MAX), ("vol", ctypes.c_double * QMCCPW_ASSETS_MAX),
                ("corr", ctypes.c_double * (QMCCPW_ASSETS_MAX * QMCCPW_ASSETS_MAX))]


def basket_struct(b) -> qmccpw_basket:
    """qmccpw_basket from an object with type, d, K, T, S0, r, sigma, w, a, v, corr (m x m)."""
    m = len(b.w)
    out = qmccpw_basket()
    out.type, out.d, out.m, out.reserved = b.type, b.d, m, 0
    out.K, out.T, out.S0, out.r, out.sigma = b.K, b.T, b.S0, b.r, b.sigma
    corr = np.asarray(b.corr, dtype=np.float64).reshape(m, m)
    for i in range(m):
        out.weight[i], out.spot[i], out.vol[i] = float(b.w[i]), float(b.a[i]), float(b.v[i])
        for k in range(m):
            out.corr[i * m + k] = float(corr[i, k])  # row stride m
    return out


class qmccpw_contract(ctypes.Structure):
    _fields_ = [("option", qmccpw_option), ("market", qmccpw_market), ("N", ctypes.c_uint64),
                ("R", ctypes.c_int32), ("construction", ctypes.c_int32), ("first_replicate", ctypes.c_int32),
                ("first_point", ctypes.c_uint32)]


class qmccpw_server_desc(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("max_inflight", ctypes.c_int32),
                ("idle_limit_us", ctypes.c_int32), ("constructions", ctypes.c_int32),
                ("max_inflight_bytes", ctypes.c_uint64)]


class qmccpw_server_stats(ctypes.Structure):
    _fields_ = [(name, ctypes.c_uint64) for name in (
        "submitted", "completed", "failed", "launches", "idle_exits", "point_dates", "pending", "inflight",
        "running")]


class qmccpw_pipe_peaks(ctypes.Structure):
    _fields_ = [(name, ctypes.c_double) for name in (
        "fp32_fma_tflops", "fp32_fma2_tflops", "fp64_fma_tflops", "sfu_ex2_gops", "sfu_lg2_gops",
        "sfu_rcp_gops", "tc_bf16_tflops", "tc_tf32_tflops")]


_lib = None
_lock = threading.Lock()


def library() -> ctypes.CDLL:
    """The loaded libqmccpw (raises QmcCpwError if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise QmcCpwError(QMCCPW_ERR_CUDA, f"{LIB_PATH} is missing: build it with "
                                                   "python -m paper_2209_11337_gb300.build")
            L = ctypes.CDLL(LIB_PATH)
            P = ctypes.POINTER
            vp, i32, u32, u64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_uint32, ctypes.c_uint64
            L.qmccpw_plan.argtypes = [P(vp), P(qmccpw_plan_desc)]
            L.qmccpw_greeks.argtypes = [vp, P(qmccpw_option), P(qmccpw_market), u64, i32, i32, i32, P(qmccpw_result)]
            L.qmccpw_greeks_batch.argtypes = [vp, P(qmccpw_contract), i32, i32, P(qmccpw_result)]
            L.qmccpw_batch_create.argtypes = [vp, P(qmccpw_contract), i32, i32, P(vp)]
            L.qmccpw_batch_launch.argtypes = [vp, vp]
            L.qmccpw_batch_results.argtypes = [vp, P(qmccpw_result)]
            L.qmccpw_batch_device_results.argtypes = [vp, P(vp), P(vp)]
            L.qmccpw_batch_launch_count.argtypes = [vp, P(i32)]
            L.qmccpw_batch_set_timing.argtypes = [vp, i32]
            L.qmccpw_batch_timing.argtypes = [vp, P(ctypes.c_float), P(i32)]
            L.qmccpw_batch_use_graph.argtypes = [vp, i32]
            L.qmccpw_selftest_bounded_wait.argtypes = [i32, i32, P(i32)]
            L.qmccpw_batch_segment_timing.argtypes = [vp, P(ctypes.c_float), P(i32)]
            L.qmccpw_batch_free.argtypes = [vp]
            L.qmccpw_measure_pipe_peaks.argtypes = [i32, P(qmccpw_pipe_peaks)]
            L.qmccpw_batch_scatter_replicates.argtypes = [vp, vp, P(ctypes.c_int64)]
            L.qmccpw_replicate_stats.argtypes = [vp, vp, vp, i32, vp, vp]
            L.qmccpw_sobol_points.argtypes = [vp, u32, i32, u64, u64, P(u32)]
            L.qmccpw_point_values.argtypes = [vp, P(qmccpw_option), P(qmccpw_market), i32, i32, u32, u64, u64,
                                              P(ctypes.c_double)]
            L.qmccpw_greeks_noalloc.argtypes = [vp, P(qmccpw_option), P(qmccpw_market), u64, i32, i32, i32,
                                                 ctypes.c_void_p, vp]
            L.qmccpw_basket_greeks.argtypes = [vp, P(qmccpw_basket), u64, i32, i32, P(qmccpw_result)]
            L.qmccpw_basket_point_values.argtypes = [vp, P(qmccpw_basket), i32, u32, u64, u64, P(ctypes.c_double)]
            L.qmccpw_server_start.argtypes = [vp, P(qmccpw_server_desc)]
            L.qmccpw_submit.argtypes = [vp, P(qmccpw_contract), P(u64)]
            L.qmccpw_poll.argtypes = [vp, u64, P(qmccpw_result)]
            L.qmccpw_wait.argtypes = [vp, u64, i32, P(qmccpw_result)]
            L.qmccpw_server_get_stats.argtypes = [vp, P(qmccpw_server_stats)]
            L.qmccpw_server_stop.argtypes = [vp]
            L.qmccpw_autotune.argtypes = [vp, P(qmccpw_contract), i32, i32]
            L.qmccpw_tuning_get.argtypes = [vp, i32, i32, i32, P(i32)]
            L.qmccpw_tuning_set.argtypes = [vp, i32, i32, i32, i32]
            L.qmccpw_free.argtypes = [vp]
            L.qmccpw_last_error.restype = ctypes.c_char_p
            L.qmccpw_version.restype = ctypes.c_char_p
            for name in EXPORTS:
                if name not in ("qmccpw_last_error", "qmccpw_version"):
                    getattr(L, name).restype = ctypes.c_int
            _lib = L
        return _lib


def _check(rc: int) -> int:
    if rc not in (QMCCPW_OK, QMCCPW_NOT_READY):
        msg = library().qmccpw_last_error().decode(errors="replace")
        raise QmcCpwError(rc, msg)
    return rc


# ---- thin functions with the C names ---------------------------------------------
def qmccpw_plan(device: int = 0, d_max: int = 366, r_max: int = 64, seed: int = 0x220911337,
                stream: Optional[int] = None, workspace_bytes: int = 0) -> ctypes.c_void_p:
    desc = qmccpw_plan_desc(device, d_max, r_max, 0, seed, stream, workspace_bytes)
    h = ctypes.c_void_p()
    _check(library().qmccpw_plan(ctypes.byref(h), ctypes.byref(desc)))
    return h


def qmccpw_free(plan) -> None:
    _check(library().qmccpw_free(plan))


def _result(R: int):
    per = np.zeros((R, 4))
    res = qmccpw_result()
    res.per_replicate = per.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    return res, per


def qmccpw_greeks(plan, type: int, d: int, K: float, T: float, S0: float, r: float, sigma: float,
                  N: int, R: int, construction: int = QMCCPW_BB, precision: int = QMCCPW_FP64):
    """One contract; returns (mean[4], se[4], per_replicate[R,4]) as numpy arrays."""
    res, per = _result(R)
    _check(library().qmccpw_greeks(plan, ctypes.byref(qmccpw_option(type, d, K, T)),
                                   ctypes.byref(qmccpw_market(S0, r, sigma)), N, R, construction, precision,
                                   ctypes.byref(res)))
    return np.array(res.mean[:]), np.array(res.se[:]), per


def qmccpw_basket_greeks(plan, basket, N: int, R: int, precision: int = QMCCPW_FP64):
    """A basket (see basket_struct); returns (mean[4], se[4], per_replicate[R,4])."""
    res, per = _result(R)
    _check(library().qmccpw_basket_greeks(plan, ctypes.byref(basket_struct(basket)), N, R, precision,
                                          ctypes.byref(res)))
    return np.array(res.mean[:]), np.array(res.se[:]), per


def qmccpw_basket_point_values(plan, basket, precision: int, replicate: int, k0: int, count: int) -> np.ndarray:
    out = np.zeros((count, 4))
    _check(library().qmccpw_basket_point_values(plan, ctypes.byref(basket_struct(basket)), precision, replicate,
                                                k0, count, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
    return out


def contract_array(contracts: Sequence) -> ctypes.Array:
    """ctypes array of qmccpw_contract from objects with type, d, K, T, S0, r, sigma, N, R, construction
    (and optionally first_replicate and first_point, 0 when absent)."""
    arr = (qmccpw_contract * len(contracts))()
    for i, c in enumerate(contracts):
        arr[i] = qmccpw_contract(qmccpw_option(c.type, c.d, c.K, c.T), qmccpw_market(c.S0, c.r, c.sigma),
                                 c.N, c.R, c.construction, getattr(c, "first_replicate", 0),
                                 getattr(c, "first_point", 0))
    return arr


def qmccpw_greeks_batch(plan, contracts: Sequence, precision: int = QMCCPW_FP64):
    """Returns a list of (mean[4], se[4], per_replicate[R,4])."""
    arr = contract_array(contracts)
    results = (qmccpw_result * len(contracts))()
    pers = []
    for i, c in enumerate(contracts):
        per = np.zeros((c.R, 4))
        pers.append(per)
        results[i].per_replicate = per.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    _check(library().qmccpw_greeks_batch(plan, arr, len(contracts), precision, results))
    return [(np.array(results[i].mean[:]), np.array(results[i].se[:]), pers[i]) for i in range(len(contracts))]


class Batch:
    """Prepared batch (qmccpw_batch_create / _launch / _results / _free)."""

    def __init__(self, plan, contracts: Sequence, precision: int):
        self.contracts = list(contracts)
        self._arr = contract_array(self.contracts)
        self.handle = ctypes.c_void_p()
        _check(library().qmccpw_batch_create(plan, self._arr, len(self.contracts), precision,
                                             ctypes.byref(self.handle)))

    def launch(self, stream: Optional[int] = None) -> None:
        _check(library().qmccpw_batch_launch(self.handle, stream))

    def launch_count(self) -> int:
        n = ctypes.c_int32()
        _check(library().qmccpw_batch_launch_count(self.handle, ctypes.byref(n)))
        return n.value

    def set_timing(self, capacity: int) -> None:
        _check(library().qmccpw_batch_set_timing(self.handle, capacity))

    def segment_timing(self):
        """([bridge, standard, streamed tensor-core PCA, other PCA, leading-coordinate bridge,
        leading-coordinate PCA] milliseconds, launches), record kept."""
        ms, n = (ctypes.c_float * 6)(), ctypes.c_int32()
        _check(library().qmccpw_batch_segment_timing(self.handle, ms, ctypes.byref(n)))
        return list(ms), n.value

    def scatter_replicates(self, dst_ptr: Optional[int], first_row: Sequence[int]) -> None:
        """qmccpw_batch_scatter_replicates: rows of a device array receive the replicate estimates."""
        qmccpw_batch_scatter_replicates(self.handle, dst_ptr, first_row)

    def use_graph(self, enable: bool = True) -> None:
        """Replay the launch sequence as one CUDA graph (qmccpw_batch_use_graph)."""
        _check(library().qmccpw_batch_use_graph(self.handle, 1 if enable else 0))

    def timing(self):
        """(summed fused-kernel milliseconds, launches covered) since the last call."""
        ms, n = ctypes.c_float(), ctypes.c_int32()
        _check(library().qmccpw_batch_timing(self.handle, ctypes.byref(ms), ctypes.byref(n)))
        return ms.value, n.value

    def device_results(self):
        per, st = ctypes.c_void_p(), ctypes.c_void_p()
        _check(library().qmccpw_batch_device_results(self.handle, ctypes.byref(per), ctypes.byref(st)))
        return per.value, st.value

    def results(self):
        results = (qmccpw_result * len(self.contracts))()
        pers = []
        for i, c in enumerate(self.contracts):
            per = np.zeros((c.R, 4))
            pers.append(per)
            results[i].per_replicate = per.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        _check(library().qmccpw_batch_results(self.handle, results))
        return [(np.array(results[i].mean[:]), np.array(results[i].se[:]), pers[i])
                for i in range(len(self.contracts))]

    def free(self) -> None:
        if self.handle:
            _check(library().qmccpw_batch_free(self.handle))
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def qmccpw_sobol_points(plan, replicate: int, ndims: int, k0: int, count: int) -> np.ndarray:
    out = np.zeros((count, ndims), dtype=np.uint32)
    _check(library().qmccpw_sobol_points(plan, replicate, ndims, k0, count,
                                         out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))))
    return out


def qmccpw_selftest_bounded_wait(device: int = 0, limit_us: int = 10000) -> int:
    """Status the probe kernel recorded (QMCCPW_ERR_TIMEOUT when the bounded wait gave up)."""
    st = ctypes.c_int32()
    _check(library().qmccpw_selftest_bounded_wait(device, limit_us, ctypes.byref(st)))
    return st.value


def qmccpw_point_values(plan, type: int, d: int, K: float, T: float, S0: float, r: float, sigma: float,
                        construction: int, precision: int, replicate: int, k0: int, count: int) -> np.ndarray:
    out = np.zeros((count, 4))
    _check(library().qmccpw_point_values(plan, ctypes.byref(qmccpw_option(type, d, K, T)),
                                         ctypes.byref(qmccpw_market(S0, r, sigma)), construction, precision,
                                         replicate, k0, count, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
    return out


def qmccpw_greeks_noalloc(plan, type: int, d: int, K: float, T: float, S0: float, r: float, sigma: float,
                          N: int, R: int, construction: int, precision: int, out_device_ptr: int,
                          stream: Optional[int] = None) -> None:
    """Allocation-free form: writes (R + 2) * 4 doubles to the caller's device buffer
    at ``out_device_ptr`` (per-replicate estimates, mean, se) on ``stream``."""
    _check(library().qmccpw_greeks_noalloc(plan, ctypes.byref(qmccpw_option(type, d, K, T)),
                                           ctypes.byref(qmccpw_market(S0, r, sigma)), N, R, construction,
                                           precision, ctypes.c_void_p(out_device_ptr), stream))


def qmccpw_server_start(plan, precision: int = QMCCPW_MIXED, max_inflight: int = 0, idle_limit_us: int = 0,
                        max_inflight_bytes: int = 0, constructions: Sequence[int] = ()) -> None:
    """Start the device-resident serving loop (0: the library's default for each limit; constructions:
    the accepted qmccpw_construction values, empty for all)."""
    mask = 0
    for cons in constructions:
        mask |= 1 << cons
    desc = qmccpw_server_desc(precision, max_inflight, idle_limit_us, mask, max_inflight_bytes)
    _check(library().qmccpw_server_start(plan, ctypes.byref(desc)))


def qmccpw_submit(plan, c) -> int:
    """Queue a contract (object with type, d, K, T, S0, r, sigma, N, R, construction); returns its ticket."""
    arr = contract_array([c])
    t = ctypes.c_uint64()
    _check(library().qmccpw_submit(plan, arr, ctypes.byref(t)))
    return t.value


def _server_result(R):
    per = np.zeros((R, 4))
    res = qmccpw_result()
    res.per_replicate = per.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    return res, per


def qmccpw_poll(plan, ticket: int, R: int):
    """(mean, se, per_replicate) when finished, None while not ready."""
    res, per = _server_result(R)
    rc = _check(library().qmccpw_poll(plan, ticket, ctypes.byref(res)))
    if rc == QMCCPW_NOT_READY:
        return None
    return np.array(res.mean[:]), np.array(res.se[:]), per


def qmccpw_wait(plan, ticket: int, R: int, timeout_ms: int = 60000):
    res, per = _server_result(R)
    _check(library().qmccpw_wait(plan, ticket, timeout_ms, ctypes.byref(res)))
    return np.array(res.mean[:]), np.array(res.se[:]), per


def qmccpw_server_get_stats(plan) -> dict:
    st = qmccpw_server_stats()
    _check(library().qmccpw_server_get_stats(plan, ctypes.byref(st)))
    return {k: getattr(st, k) for k, _ in qmccpw_server_stats._fields_}


def qmccpw_server_stop(plan) -> None:
    _check(library().qmccpw_server_stop(plan))


def qmccpw_autotune(plan, sample: Sequence, precision: int = QMCCPW_MIXED) -> None:
    arr = contract_array(sample)
    _check(library().qmccpw_autotune(plan, arr, len(sample), precision))


def qmccpw_tuning_get(plan, precision: int, construction: int, d: int) -> int:
    out = ctypes.c_int32()
    _check(library().qmccpw_tuning_get(plan, precision, construction, d, ctypes.byref(out)))
    return out.value


def qmccpw_tuning_set(plan, precision: int, construction: int, d: int, points_per_tile: int) -> None:
    _check(library().qmccpw_tuning_set(plan, precision, construction, d, points_per_tile))


def qmccpw_last_error() -> str:
    return library().qmccpw_last_error().decode(errors="replace")


def qmccpw_version() -> str:
    return library().qmccpw_version().decode()


def qmccpw_batch_scatter_replicates(batch, dst_ptr: Optional[int], first_row: Sequence[int]) -> None:
    """After each later launch, copy the batch's replicate estimates to rows of the device array at
    ``dst_ptr`` (e.g. ``tensor.data_ptr()``); ``None`` turns the copy off."""
    rows = (ctypes.c_int64 * max(1, len(first_row)))(*first_row)
    _check(library().qmccpw_batch_scatter_replicates(batch, dst_ptr, rows if dst_ptr else None))


def qmccpw_replicate_stats(per_replicate_ptr: int, first_row_ptr: int, R_ptr: int, count: int, stats_ptr: int,
                           stream=None) -> None:
    """Mean and SE over replicates of device-resident replicate estimates (all arguments device pointers)."""
    _check(library().qmccpw_replicate_stats(per_replicate_ptr, first_row_ptr, R_ptr, count, stats_ptr, stream))


def qmccpw_measure_pipe_peaks(device: int = 0) -> dict:
    """The pipe micro-benchmarks of ``device`` as a dict of the struct's fields."""
    out = qmccpw_pipe_peaks()
    _check(library().qmccpw_measure_pipe_peaks(device, ctypes.byref(out)))
    return {name: getattr(out, name) for name, _ in qmccpw_pipe_peaks._fields_}
