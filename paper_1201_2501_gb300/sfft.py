"""ctypes binding of ``libsfft.so`` (C ABI in ``include/sfft.h``): same names, argument marshalling only.

Every computation runs in the library's CUDA kernels.  There is no CPU fallback: if the library is
missing or fails to load, the first call raises ``RuntimeError``.  PyTorch supplies device memory and
the current stream; tensors are passed by ``data_ptr()``.
"""
from __future__ import annotations

import ctypes
import os
import threading

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libsfft.so")

SFFT_OK = 0
SFFT_ERR_INVALID_ARG = 1
SFFT_ERR_N_NOT_POW2 = 2
SFFT_ERR_K_RANGE = 3
SFFT_ERR_OOM = 4
SFFT_ERR_CUDA = 5
SFFT_ERR_TIMEOUT = 6
SFFT_ERR_CAPACITY = 7
SFFT_ERR_NOT_CONVERGED = 8
SFFT_ERR_BUSY = 9

SFFT_EXACT = 0
SFFT_GENERAL = 1
SFFT_FP32 = 0
SFFT_FP64 = 1


class SfftParams(ctypes.Structure):
    """Mirror of ``sfft_params`` (include/sfft.h)."""

    _fields_ = [
        ("n", ctypes.c_uint64),
        ("k", ctypes.c_uint32),
        ("mode", ctypes.c_uint32),
        ("precision", ctypes.c_uint32),
        ("delta", ctypes.c_double),
        ("alpha0", ctypes.c_double),
        ("bins_per_k", ctypes.c_double),
        ("B_min", ctypes.c_uint32),
        ("extra_rounds", ctypes.c_uint32),
        ("thr", ctypes.c_double),
        ("tau_dec", ctypes.c_double),
        ("iso_tol", ctypes.c_double),
        ("gmin", ctypes.c_double),
        ("prune", ctypes.c_double),
        ("ref_lo", ctypes.c_double),
        ("ref_hi", ctypes.c_double),
        ("ref_tol", ctypes.c_double),
        ("z_cap", ctypes.c_uint32),
        ("eps", ctypes.c_double),
        ("t_regions", ctypes.c_uint32),
        ("R_loc", ctypes.c_uint32),
        ("R_est", ctypes.c_uint32),
        ("s", ctypes.c_double),
        ("est_gmin", ctypes.c_double),
        ("streams", ctypes.c_uint32),
        ("gain", ctypes.c_uint32),
        ("chunk_taps", ctypes.c_uint32),
        ("permuted_copy", ctypes.c_uint32),
    ]


class SfftRequest(ctypes.Structure):
    """Mirror of ``sfft_request``."""

    _fields_ = [("d_x", ctypes.c_void_p), ("seed", ctypes.c_uint64), ("id", ctypes.c_uint32),
                ("period", ctypes.c_uint32)]


class SfftServerConfig(ctypes.Structure):
    """Mirror of ``sfft_server_config``."""

    _fields_ = [("mem_budget", ctypes.c_uint64), ("max_batch", ctypes.c_uint32), ("instances", ctypes.c_uint32),
                ("max_plans", ctypes.c_uint32), ("reserved", ctypes.c_uint32)]


class SfftJob(ctypes.Structure):
    """Mirror of ``sfft_job``."""

    _fields_ = [("x", ctypes.c_void_p), ("x_on_device", ctypes.c_uint32), ("id", ctypes.c_uint32),
                ("seed", ctypes.c_uint64), ("h_idx", ctypes.c_void_p), ("h_val", ctypes.c_void_p),
                ("cap", ctypes.c_uint32), ("period", ctypes.c_uint32)]


class SfftJobResult(ctypes.Structure):
    """Mirror of ``sfft_job_result``."""

    _fields_ = [("count", ctypes.c_uint32), ("flag", ctypes.c_int32), ("queued_us", ctypes.c_double),
                ("latency_us", ctypes.c_double)]


class SfftServerStats(ctypes.Structure):
    """Mirror of ``sfft_server_stats``."""

    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64), ("failed", ctypes.c_uint64),
                ("launches", ctypes.c_uint64), ("plans", ctypes.c_uint64), ("bytes_in_use", ctypes.c_uint64),
                ("bytes_peak", ctypes.c_uint64), ("mean_batch", ctypes.c_double), ("p50_us", ctypes.c_double),
                ("p99_us", ctypes.c_double)]


class SfftTuneEntry(ctypes.Structure):
    """Mirror of ``sfft_tune_entry``."""

    _fields_ = [("bins_per_k", ctypes.c_double), ("alpha0", ctypes.c_double), ("streams", ctypes.c_uint32),
                ("chunk_taps", ctypes.c_uint32), ("status", ctypes.c_int32), ("us_per_transform", ctypes.c_double), ("exact", ctypes.c_uint32),
                ("chosen", ctypes.c_uint32), ("rel_err", ctypes.c_double)]


class SfftGeneralTrace(ctypes.Structure):
    """Mirror of ``sfft_general_trace`` (device pointers of one traced general round)."""

    _fields_ = [("round", ctypes.c_uint32), ("reserved", ctypes.c_uint32), ("d_bins", ctypes.c_void_p),
                ("d_regions", ctypes.c_void_p), ("d_valid", ctypes.c_void_p), ("d_cand", ctypes.c_void_p),
                ("d_zidx_before", ctypes.c_void_p), ("d_zval_before", ctypes.c_void_p),
                ("d_zcount_before", ctypes.c_void_p), ("d_zidx_after", ctypes.c_void_p),
                ("d_zval_after", ctypes.c_void_p), ("d_zcount_after", ctypes.c_void_p)]


class SfftError(RuntimeError):
    def __init__(self, status, what):
        self.status = status
        super().__init__(f"{what}: {sfft_status_str(status)} ({status}) {sfft_last_error()}")


_lib = None
_lock = threading.Lock()
_P = ctypes.POINTER(SfftParams)
_vp = ctypes.c_void_p
_u32, _u64, _i32, _dbl = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int32, ctypes.c_double
_u32p = ctypes.POINTER(ctypes.c_uint32)
_u64p = ctypes.POINTER(ctypes.c_uint64)
_i64p = ctypes.POINTER(ctypes.c_int64)
_dblp = ctypes.POINTER(ctypes.c_double)

_SIGS = {
    "sfft_params_default": (None, [_P, _u64, _u32, _u32]),
    "sfft_status_str": (ctypes.c_char_p, [ctypes.c_int]),
    "sfft_last_error": (ctypes.c_char_p, []),
    "sfft_plan_create": (ctypes.c_int, [_P, _u32, ctypes.POINTER(_vp)]),
    "sfft_plan_destroy": (ctypes.c_int, [_vp]),
    "sfft_plan_rounds": (_u32, [_vp]),
    "sfft_plan_round_info": (ctypes.c_int, [_vp, _u32, _u64, _u32, _u32p, _dblp, _i64p, _u32p, _u64p, _u64p, _u64p]),
    "sfft_plan_taps": (ctypes.c_int, [_vp, _u32, _dblp, _u64]),
    "sfft_execute": (ctypes.c_int, [_vp, _vp, _u32, _u64, _vp, _vp, _vp, _u32, _vp, _vp]),
    "sfft_execute_host": (ctypes.c_int, [_vp, _vp, _u32, _u64, _vp, _vp, _vp, _u32, _vp, _vp]),
    "sfft_hash_to_bins": (ctypes.c_int, [_vp, _u32, _vp, _u64, _u64, _u64, _vp, _vp, _u32, _vp, _vp]),
    "sfft_exact_decode": (ctypes.c_int, [_vp, _u32, _u64, _u64, _vp, _vp, _u32, _vp, _vp, _vp, _vp, _vp, _vp]),
    "sfft_philox": (ctypes.c_int, [_u32, _u32, _u32p, _u32, _vp, _vp]),
    "sfft_hash_to_bins_static": (ctypes.c_int, [_u64, _u32, ctypes.c_int64, _vp, _vp, _vp, _u64, _u64, _u64, _vp, _vp,
                                                _u32, _vp, _vp]),
    "sfft_plan_general_round_info": (ctypes.c_int, [_vp, _u32, _u32p, _i64p, _u32p, _u32p, _u32p, _u64p, _u64p]),
    "sfft_locate_votes": (ctypes.c_int, [_vp, _u32, _u64, _u64, _u64, _u32, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "sfft_estimate_from_bins": (ctypes.c_int, [_vp, _u32, _u32, _vp, _vp, _vp, _vp, _vp, _u32, _u32, _vp, _vp, _vp,
                                               _vp]),
    "sfft_window_taps": (ctypes.c_int, [_u64, _u32, _dbl, _dbl, _i64p, _dblp, _u64]),
    "sfft_window_gains": (ctypes.c_int, [_u64, _u32, _dbl, _dbl, _u64, _dblp]),
    "sfft_twiddle_tables": (ctypes.c_int, [_u64, ctypes.POINTER(ctypes.c_uint64), _dblp, _u64]),
    "sfft_execute_requests": (ctypes.c_int, [_vp, ctypes.POINTER(SfftRequest), _u32, _vp, _vp, _vp, _u32, _vp, _vp]),
    "sfft_autotune": (ctypes.c_int, [_P, _u32, _dbl, _u64, _u32, _P, ctypes.POINTER(SfftTuneEntry), _u32, _u32p]),
    "sfft_graph_create": (ctypes.c_int, [_vp, _vp, _u32, _u64, _vp, _vp, _u32, _vp, _vp, ctypes.POINTER(_vp)]),
    "sfft_graph_launch": (ctypes.c_int, [_vp, _vp]),
    "sfft_graph_destroy": (ctypes.c_int, [_vp]),
    "sfft_plan_set_requests": (ctypes.c_int, [_vp, ctypes.POINTER(SfftRequest), _u32, _vp]),
    "sfft_batch_plan_create": (ctypes.c_int, [ctypes.POINTER(_vp), _u32, _u32, ctypes.POINTER(_vp)]),
    "sfft_batch_plan_destroy": (ctypes.c_int, [_vp]),
    "sfft_persistent_wait_check": (ctypes.c_int, [_vp]),
    "sfft_batch_execute": (ctypes.c_int, [_vp, _u32p, ctypes.POINTER(SfftRequest), _u32, _vp, _vp, _vp, _u32, _vp,
                                          _vp]),
    "sfft_server_create": (ctypes.c_int, [ctypes.POINTER(SfftServerConfig), ctypes.POINTER(_vp)]),
    "sfft_server_destroy": (ctypes.c_int, [_vp]),
    "sfft_submit": (ctypes.c_int, [_vp, _P, ctypes.POINTER(SfftJob), _u64p]),
    "sfft_submit_many": (ctypes.c_int, [_vp, _P, ctypes.POINTER(SfftJob), _u32, _u64p]),
    "sfft_wait_many": (ctypes.c_int, [_vp, _u64p, _u32, _u64, ctypes.POINTER(SfftJobResult),
                                      ctypes.POINTER(ctypes.c_int32)]),
    "sfft_poll": (ctypes.c_int, [_vp, _u64]),
    "sfft_wait": (ctypes.c_int, [_vp, _u64, _u64, ctypes.POINTER(SfftJobResult)]),
    "sfft_server_stats_get": (ctypes.c_int, [_vp, ctypes.POINTER(SfftServerStats)]),
    "sfft_execute_channels": (ctypes.c_int, [_vp, _vp, _u32, _u64, _u32, _vp, _vp, _vp, _u32, _vp, _vp]),
    "sfft_execute_channels_timed": (ctypes.c_int, [_vp, _vp, _u32, _u64, _u32, _vp, _vp, _vp, _u32, _vp, _vp, _vp,
                                                   _vp]),
    "sfft_gather_rate": (ctypes.c_int, [_vp, _u64, _u32, _vp, _u32, _vp, _vp]),
    "sfft_execute_trace": (ctypes.c_int, [_vp, _vp, _u32, _u64, _vp, _vp, _vp, _u32, _vp, _vp,
                                          ctypes.POINTER(SfftGeneralTrace)]),
}

SFFT_STATIC_SCRATCH_BYTES = 4 * 1024 * 1024

EXPORTED = tuple(_SIGS)


def lib():
    """Load libsfft.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -m paper_1201_2501_gb300.build`")
            L = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in _SIGS.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def sfft_status_str(status: int) -> str:
    return lib().sfft_status_str(int(status)).decode()


def sfft_last_error() -> str:
    return lib().sfft_last_error().decode()


def _check(status, what):
    if status != SFFT_OK:
        raise SfftError(status, what)


def _stream_ptr(stream):
    if stream is None:
        import torch

        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(int(stream.cuda_stream))


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def sfft_params_default(n: int, k: int, mode: int = SFFT_EXACT, **over) -> SfftParams:
    p = SfftParams()
    lib().sfft_params_default(ctypes.byref(p), n, k, mode)
    for key, v in over.items():
        if not hasattr(p, key):
            raise KeyError(key)
        setattr(p, key, v)
    return p


class Plan:
    """Owner of an ``sfft_plan`` (``sfft_plan_create`` / ``sfft_plan_destroy``)."""

    def __init__(self, params: SfftParams, max_batch: int = 1):
        self.params = params
        self.max_batch = int(max_batch)
        h = ctypes.c_void_p()
        _check(lib().sfft_plan_create(ctypes.byref(params), self.max_batch, ctypes.byref(h)), "sfft_plan_create")
        self.handle = h

    def close(self):
        if getattr(self, "handle", None):
            lib().sfft_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def rounds(self) -> int:
        return int(lib().sfft_plan_rounds(self.handle))

    def round_info(self, t: int, seed: int = 0, request: int = 0) -> dict:
        B, ns = ctypes.c_uint32(), ctypes.c_uint32()
        alpha, T = ctypes.c_double(), ctypes.c_int64()
        shifts = (ctypes.c_uint64 * 4)()
        sigma, b = ctypes.c_uint64(), ctypes.c_uint64()
        _check(lib().sfft_plan_round_info(self.handle, t, seed, request, ctypes.byref(B), ctypes.byref(alpha),
                                          ctypes.byref(T), ctypes.byref(ns), shifts, ctypes.byref(sigma),
                                          ctypes.byref(b)), "sfft_plan_round_info")
        return dict(B=B.value, alpha=alpha.value, T=T.value, shifts=[int(shifts[i]) for i in range(ns.value)],
                    sigma=sigma.value, b=b.value)

    def taps(self, t: int):
        import numpy as np

        T = general_round_info(self, t)["T"] if self.params.mode == SFFT_GENERAL else self.round_info(t)["T"]
        out = np.zeros(T + 1, dtype=np.float64)
        _check(lib().sfft_plan_taps(self.handle, t, out.ctypes.data_as(_dblp), T + 1), "sfft_plan_taps")
        return out


def sfft_execute(plan: Plan, x, seed: int, cap: int, outputs=None, stream=None):
    """Run the batch ``x`` (torch tensor [batch, n], complex64 or complex128 on the GPU).

    Returns (idx uint32->int32 view [batch, cap], val float64 [batch, cap, 2], count int32 [batch],
    flag int32 [batch]) as device tensors (allocated here unless ``outputs`` is given)."""
    import torch

    batch = x.shape[0] if x.dim() == 2 else 1
    if outputs is None:
        dev = x.device
        outputs = (torch.empty((batch, cap), dtype=torch.int32, device=dev),
                   torch.empty((batch, cap, 2), dtype=torch.float64, device=dev),
                   torch.empty((batch,), dtype=torch.int32, device=dev),
                   torch.empty((batch,), dtype=torch.int32, device=dev))
    idx, val, count, flag = outputs
    _check(lib().sfft_execute(plan.handle, _ptr(x), batch, seed, _stream_ptr(stream), _ptr(idx), _ptr(val), cap,
                              _ptr(count), _ptr(flag)), "sfft_execute")
    return outputs


def sfft_execute_host(plan: Plan, x, seed: int, cap: int, outputs=None, stream=None):
    """Same as sfft_execute from host (CPU, ideally pinned) tensors; returns CPU tensors."""
    import torch

    batch = x.shape[0] if x.dim() == 2 else 1
    if outputs is None:
        outputs = (torch.empty((batch, cap), dtype=torch.int32),
                   torch.empty((batch, cap, 2), dtype=torch.float64),
                   torch.empty((batch,), dtype=torch.int32),
                   torch.empty((batch,), dtype=torch.int32))
    idx, val, count, flag = outputs
    _check(lib().sfft_execute_host(plan.handle, _ptr(x), batch, seed, _stream_ptr(stream), _ptr(idx), _ptr(val), cap,
                                   _ptr(count), _ptr(flag)), "sfft_execute_host")
    return outputs


def sfft_window_taps(n: int, B: int, alpha: float, delta: float):
    """Host-only: the window taps g_0..g_T (numpy float64) every plan builds for (n, B, alpha, delta)."""
    import numpy as np

    T = ctypes.c_int64()
    _check(lib().sfft_window_taps(n, B, alpha, delta, ctypes.byref(T), None, 0), "sfft_window_taps")
    g = np.empty(T.value + 1, dtype=np.float64)
    _check(lib().sfft_window_taps(n, B, alpha, delta, ctypes.byref(T), g.ctypes.data_as(_dblp), g.size),
           "sfft_window_taps")
    return g


def sfft_twiddle_tables(n: int):
    """Host-only: the general mode's FP64 twiddle factor tables for n (numpy complex128)."""
    import numpy as np

    m = ctypes.c_uint64()
    _check(lib().sfft_twiddle_tables(n, ctypes.byref(m), None, 0), "sfft_twiddle_tables")
    tw = np.empty(2 * m.value, dtype=np.float64)
    _check(lib().sfft_twiddle_tables(n, ctypes.byref(m), tw.ctypes.data_as(_dblp), m.value), "sfft_twiddle_tables")
    return tw[0::2] + 1j * tw[1::2]


def sfft_window_gains(n: int, B: int, alpha: float, delta: float, length: int):
    """Host-only: W(o), o = 0..length-1, the exact response of those taps (numpy float64)."""
    import numpy as np

    W = np.empty(length, dtype=np.float64)
    _check(lib().sfft_window_gains(n, B, alpha, delta, length, W.ctypes.data_as(_dblp)), "sfft_window_gains")
    return W


def sfft_execute_requests(plan: Plan, xs, seeds, ids, cap: int, outputs=None, stream=None, periods=None):
    """Run independent requests: ``xs`` a list of device tensors (n values each, anywhere in memory,
    or periods[r] values of a periodic signal), request r drawing with (seeds[r], ids[r]).  Outputs as
    for sfft_execute, slot r = request r."""
    import torch

    batch = len(xs)
    if outputs is None:
        dev = xs[0].device
        outputs = (torch.empty((batch, cap), dtype=torch.int32, device=dev),
                   torch.empty((batch, cap, 2), dtype=torch.float64, device=dev),
                   torch.empty((batch,), dtype=torch.int32, device=dev),
                   torch.empty((batch,), dtype=torch.int32, device=dev))
    table = (SfftRequest * batch)()
    for r, (x, sd, i) in enumerate(zip(xs, seeds, ids)):
        table[r].d_x = _ptr(x)
        table[r].seed = int(sd)
        table[r].id = int(i)
        table[r].period = int(periods[r]) if periods is not None else 0
    idx, val, count, flag = outputs
    _check(lib().sfft_execute_requests(plan.handle, table, batch, _stream_ptr(stream), _ptr(idx), _ptr(val), cap,
                                       _ptr(count), _ptr(flag)), "sfft_execute_requests")
    return outputs


def sfft_autotune(base: SfftParams, batch: int = 16, snr_db: float = 20.0, seed: int = 1, reps: int = 5):
    """Runs the library's autotuner for ``base``; returns (best SfftParams, list of report dicts)."""
    best = SfftParams()
    rep = (SfftTuneEntry * 128)()
    nrep = ctypes.c_uint32()
    _check(lib().sfft_autotune(ctypes.byref(base), batch, snr_db, seed, reps, ctypes.byref(best), rep, 128,
                               ctypes.byref(nrep)), "sfft_autotune")
    out = [{f: getattr(rep[i], f) for f, _ in SfftTuneEntry._fields_} for i in range(min(nrep.value, 128))]
    return best, out


class Graph:
    """A whole transform of a fixed batch captured as a CUDA graph (``sfft_graph_*``).  x = None: the
    batch is the plan's request table (refill it with ``set_requests``)."""

    def __init__(self, plan: Plan, x, batch: int, seed: int, cap: int, outputs):
        idx, val, count, flag = outputs
        h = ctypes.c_void_p()
        _check(lib().sfft_graph_create(plan.handle, _ptr(x) if x is not None else None, batch, seed, _ptr(idx),
                                       _ptr(val), cap, _ptr(count), _ptr(flag), ctypes.byref(h)), "sfft_graph_create")
        self.handle = h
        self.plan = plan
        self.outputs = outputs

    def set_requests(self, xs, seeds, ids, stream=None, periods=None):
        nreq = len(xs)
        table = (SfftRequest * nreq)()
        for r in range(nreq):
            table[r].d_x = _ptr(xs[r])
            table[r].seed = int(seeds[r])
            table[r].id = int(ids[r])
            table[r].period = int(periods[r]) if periods is not None else 0
        _check(lib().sfft_plan_set_requests(self.plan.handle, table, nreq, _stream_ptr(stream)),
               "sfft_plan_set_requests")

    def launch(self, stream=None):
        _check(lib().sfft_graph_launch(self.handle, _stream_ptr(stream)), "sfft_graph_launch")
        return self.outputs

    def close(self):
        if self.handle:
            lib().sfft_graph_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class BatchPlan:
    """Exact-mode plans of any (n, k) run together in one persistent launch (``sfft_batch_*``)."""

    def __init__(self, plans, max_requests: int):
        self.plans = list(plans)  # the plans must outlive the batch plan
        arr = (_vp * len(self.plans))(*[p.handle for p in self.plans])
        h = ctypes.c_void_p()
        _check(lib().sfft_batch_plan_create(arr, len(self.plans), max_requests, ctypes.byref(h)),
               "sfft_batch_plan_create")
        self.handle = h
        self.max_requests = max_requests

    @staticmethod
    def prepare(plan_of, xs, seeds, ids, periods=None):
        """The host tables of a batch (plan indices and requests), reusable across calls."""
        nreq = len(xs)
        table = (SfftRequest * nreq)()
        for r in range(nreq):
            table[r].d_x = _ptr(xs[r])
            table[r].seed = int(seeds[r])
            table[r].id = int(ids[r])
            table[r].period = int(periods[r]) if periods is not None else 0
        po = (ctypes.c_uint32 * nreq)(*[int(p) for p in plan_of])
        return po, table, nreq, list(xs)

    def execute_prepared(self, prepared, cap: int, outputs, stream=None):
        po, table, nreq, _ = prepared
        idx, val, count, flag = outputs
        _check(lib().sfft_batch_execute(self.handle, po, table, nreq, _stream_ptr(stream), _ptr(idx), _ptr(val),
                                        cap, _ptr(count), _ptr(flag)), "sfft_batch_execute")
        return outputs

    def execute(self, plan_of, xs, seeds, ids, cap: int, outputs=None, stream=None, periods=None):
        """Request r uses plans[plan_of[r]] on device tensor xs[r] with (seeds[r], ids[r]); outputs as
        for sfft_execute."""
        import torch

        nreq = len(xs)
        if outputs is None:
            dev = xs[0].device
            outputs = (torch.empty((nreq, cap), dtype=torch.int32, device=dev),
                       torch.empty((nreq, cap, 2), dtype=torch.float64, device=dev),
                       torch.empty((nreq,), dtype=torch.int32, device=dev),
                       torch.empty((nreq,), dtype=torch.int32, device=dev))
        table = (SfftRequest * nreq)()
        for r in range(nreq):
            table[r].d_x = _ptr(xs[r])
            table[r].seed = int(seeds[r])
            table[r].id = int(ids[r])
            table[r].period = int(periods[r]) if periods is not None else 0
        po = (ctypes.c_uint32 * nreq)(*[int(p) for p in plan_of])
        idx, val, count, flag = outputs
        _check(lib().sfft_batch_execute(self.handle, po, table, nreq, _stream_ptr(stream), _ptr(idx), _ptr(val),
                                        cap, _ptr(count), _ptr(flag)), "sfft_batch_execute")
        return outputs

    def close(self):
        if self.handle:
            lib().sfft_batch_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching server (``sfft_server_*``, ``sfft_submit``, ``sfft_poll``, ``sfft_wait``).

    ``submit`` takes a signal tensor (host or device; it must stay alive and unchanged until the job
    completes, which this object ensures by holding a reference) and returns a ticket; ``wait``
    returns (indices int64, values complex128, result dict) with the host arrays the server wrote."""

    def __init__(self, mem_budget: int = 0, max_batch: int = 0, instances: int = 0, max_plans: int = 0):
        import numpy as np  # noqa: F401  (output arrays)

        cfg = SfftServerConfig(mem_budget, max_batch, instances, max_plans, 0)
        h = ctypes.c_void_p()
        _check(lib().sfft_server_create(ctypes.byref(cfg), ctypes.byref(h)), "sfft_server_create")
        self.handle = h
        self._live = {}
        self._mu = threading.Lock()

    def submit(self, params: SfftParams, x, seed: int, id: int = 0, cap: int = 0, period: int = 0) -> int:
        import numpy as np

        cap = cap or params.z_cap
        on_dev = bool(getattr(x, "is_cuda", False))
        if not on_dev and hasattr(x, "is_contiguous") and not x.is_contiguous():
            x = x.contiguous()
        idx = np.empty(cap, dtype=np.uint32)
        val = np.empty((cap, 2), dtype=np.float64)
        job = SfftJob(_ptr(x) if hasattr(x, "data_ptr") else x.ctypes.data, 1 if on_dev else 0, id, seed,
                      idx.ctypes.data, val.ctypes.data, cap, period)
        t = ctypes.c_uint64()
        _check(lib().sfft_submit(self.handle, ctypes.byref(params), ctypes.byref(job), ctypes.byref(t)),
               "sfft_submit")
        with self._mu:
            self._live[t.value] = (x, idx, val)
        return t.value

    def submit_many(self, params: SfftParams, xs, seed: int, ids, cap: int = 0) -> list:
        """sfft_submit_many: one job per signal of ``xs`` (device tensors, read in place), request
        indices ``ids``; returns the tickets in order."""
        import numpy as np

        cap = cap or params.z_cap
        xs, ids = list(xs), list(ids)
        if not xs or len(xs) != len(ids):
            raise SfftError(SFFT_ERR_INVALID_ARG, "submit_many: one request index per signal")
        if not all(getattr(x, "is_cuda", False) and x.is_contiguous() for x in xs):
            raise SfftError(SFFT_ERR_INVALID_ARG, "submit_many: contiguous device signals")
        m = len(xs)
        idx = np.empty((m, cap), dtype=np.uint32)
        val = np.empty((m, cap, 2), dtype=np.float64)
        # the job array built as one structured array (the layout of sfft_job), not m ctypes objects
        jobs = np.zeros(m, dtype=np.dtype({"names": [f for f, _ in SfftJob._fields_],
                                           "formats": [np.uint64, np.uint32, np.uint32, np.uint64, np.uint64,
                                                       np.uint64, np.uint32, np.uint32],
                                           "offsets": [getattr(SfftJob, f).offset for f, _ in SfftJob._fields_],
                                           "itemsize": ctypes.sizeof(SfftJob)}))
        jobs["x"] = [x.data_ptr() for x in xs]
        jobs["x_on_device"] = 1
        jobs["id"] = np.asarray(ids, dtype=np.uint32)
        jobs["seed"] = seed
        jobs["h_idx"] = idx.ctypes.data + np.arange(m, dtype=np.uint64) * (cap * 4)
        jobs["h_val"] = val.ctypes.data + np.arange(m, dtype=np.uint64) * (cap * 16)
        jobs["cap"] = cap
        t = (ctypes.c_uint64 * m)()
        _check(lib().sfft_submit_many(self.handle, ctypes.byref(params), jobs.ctypes.data_as(ctypes.POINTER(SfftJob)),
                                      m, t), "sfft_submit_many")
        tickets = [int(v) for v in t]
        with self._mu:
            for r, tk in enumerate(tickets):
                self._live[tk] = (xs[r], idx[r], val[r])
        return tickets

    def wait_many(self, tickets, timeout_s: float = 60.0, arrays: bool = False):
        """sfft_wait_many: [(indices, values, result dict)] in ticket order; raises TimeoutError if a
        job is still pending (its ticket stays valid) and SfftError if one failed.  arrays=True returns
        instead one dict of arrays for the whole call: the jobs' output rows "idx" (m x cap uint32) and
        "val" (m x cap x 2 float64), each valid up to "count", and "count", "flag", "latency_us"."""
        import numpy as np

        tickets = list(tickets)
        m = len(tickets)
        t = (ctypes.c_uint64 * m)(*tickets)
        res = (SfftJobResult * m)()
        status = (ctypes.c_int32 * m)()
        st = lib().sfft_wait_many(self.handle, t, m, int(timeout_s * 1e6), res, status)
        done = []
        with self._mu:
            for r, tk in enumerate(tickets):
                if status[r] == SFFT_ERR_TIMEOUT:
                    continue
                x, idx, val = self._live.pop(tk, (None, None, None))
                if status[r] == SFFT_OK and idx is not None:
                    done.append((r, idx, val))
        if st == SFFT_ERR_TIMEOUT:
            raise TimeoutError(f"sfft_wait_many: jobs still pending after {timeout_s} s")
        _check(st, "sfft_wait_many")
        if arrays:
            rb = np.frombuffer(res, dtype=np.dtype([("count", np.uint32), ("flag", np.int32), ("queued_us", np.float64),
                                                    ("latency_us", np.float64)]), count=m)
            return {"idx": np.stack([d[1] for d in done]), "val": np.stack([d[2] for d in done]),
                    "count": rb["count"].copy(), "flag": rb["flag"].copy(), "latency_us": rb["latency_us"].copy()}
        out = []
        for r, idx, val in done:
            c = res[r].count
            out.append((idx[:c].astype(np.int64), val[:c, 0] + 1j * val[:c, 1],
                        {"count": c, "flag": res[r].flag, "queued_us": res[r].queued_us,
                         "latency_us": res[r].latency_us}))
        return out

    def poll(self, ticket: int) -> int:
        return lib().sfft_poll(self.handle, ticket)

    def wait(self, ticket: int, timeout_s: float = 60.0):
        import numpy as np

        res = SfftJobResult()
        st = lib().sfft_wait(self.handle, ticket, int(timeout_s * 1e6), ctypes.byref(res))
        if st == SFFT_ERR_TIMEOUT:
            raise TimeoutError(f"sfft_wait: job {ticket} still pending after {timeout_s} s")
        with self._mu:
            x, idx, val = self._live.pop(ticket, (None, None, None))
        _check(st, "sfft_wait")
        c = res.count
        out = {"count": c, "flag": res.flag, "queued_us": res.queued_us, "latency_us": res.latency_us}
        return idx[:c].astype(np.int64), val[:c, 0] + 1j * val[:c, 1], out

    def stats(self) -> dict:
        st = SfftServerStats()
        _check(lib().sfft_server_stats_get(self.handle, ctypes.byref(st)), "sfft_server_stats_get")
        return {f: getattr(st, f) for f, _ in SfftServerStats._fields_}

    def close(self):
        if self.handle:
            lib().sfft_server_destroy(self.handle)
            self.handle = None
            self._live.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def sfft_hash_to_bins(plan: Plan, t: int, x, sigma: int, a: int, b: int, zidx=None, zval=None, out=None,
                      stream=None):
    """One HashToBins with round t's window; returns a float64 device tensor [B, 2]."""
    import torch

    B = plan.round_info(t)["B"]
    if out is None:
        out = torch.empty((B, 2), dtype=torch.float64, device=x.device)
    nz = 0 if zidx is None else int(zidx.numel())
    _check(lib().sfft_hash_to_bins(plan.handle, t, _ptr(x), sigma, a, b, _ptr(zidx), _ptr(zval), nz, _ptr(out),
                                   _stream_ptr(stream)), "sfft_hash_to_bins")
    return out


def sfft_exact_decode(plan: Plan, t: int, sigma: int, b: int, u, zidx=None, stream=None):
    """Decode of round t on device bins ``u`` (float64 [(1+L), B, 2]); returns (idx, val, count, nabove, nkept)."""
    import torch

    B = plan.round_info(t)["B"]
    dev = u.device
    widx = torch.empty((B,), dtype=torch.int32, device=dev)
    wval = torch.empty((B, 2), dtype=torch.float64, device=dev)
    aux = torch.zeros((3,), dtype=torch.int32, device=dev)
    nz = 0 if zidx is None else int(zidx.numel())
    _check(lib().sfft_exact_decode(plan.handle, t, sigma, b, _ptr(u), _ptr(zidx), nz, _ptr(widx), _ptr(wval),
                                   ctypes.c_void_p(aux.data_ptr()), ctypes.c_void_p(aux.data_ptr() + 4),
                                   ctypes.c_void_p(aux.data_ptr() + 8), _stream_ptr(stream)), "sfft_exact_decode")
    return widx, wval, aux


def sfft_philox(key0: int, key1: int, ctr, count: int, out, stream=None):
    c = (ctypes.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    _check(lib().sfft_philox(key0 & 0xFFFFFFFF, key1 & 0xFFFFFFFF, c, count, _ptr(out), _stream_ptr(stream)),
           "sfft_philox")
    return out


def _need(t, what, numel, dtypes):
    """A device tensor of at least ``numel`` elements of one of ``dtypes``, contiguous (the C side cannot
    check the sizes of raw pointers)."""
    ok = (t is not None and getattr(t, "is_cuda", False) and t.is_contiguous() and t.dtype in dtypes
          and t.numel() >= numel)
    if not ok:
        raise SfftError(SFFT_ERR_INVALID_ARG, f"{what}: need a contiguous CUDA tensor of >= {numel} "
                                              f"elements of {[str(d) for d in dtypes]}")


def sfft_hash_to_bins_static(n: int, B: int, T: int, taps, wtab, x, sigma: int, a: int, b: int, zidx=None, zval=None,
                             out=None, stream=None):
    """HashToBins that allocates nothing (``sfft_hash_to_bins_static`` in include/sfft.h).

    For callers that must not call the CUDA allocator: every buffer is the caller's device tensor
    (``taps`` float32 [T+1], ``wtab`` float64 [n/(2B)+1] or None when there is no zhat, ``x``
    complex64 [n], ``out`` float64 [B, 2]); scratch comes from an array compiled into the library.
    Calls that overlap on the GPU share that scratch and race: serialise them.  The tensors' devices,
    types, sizes and layouts are checked here (SfftError INVALID_ARG), since the C side only sees
    pointers."""
    import torch

    nz = 0 if zidx is None else int(zidx.numel())
    if B <= 0 or n <= 0 or T < 0 or n % (2 * B):
        raise SfftError(SFFT_ERR_INVALID_ARG, "sfft_hash_to_bins_static: bad n, B or T")
    _need(taps, "taps", T + 1, (torch.float32,))
    if x is not None and x.dtype == torch.float32:  # interleaved (re, im) pairs
        _need(x, "x", 2 * n, (torch.float32,))
    else:
        _need(x, "x", n, (torch.complex64,))
    _need(out, "out", 2 * B, (torch.float64,))
    if nz > 0:
        _need(wtab, "wtab", n // (2 * B) + 1, (torch.float64,))
        _need(zidx, "zidx", nz, (torch.int32,))
        _need(zval, "zval", 2 * nz, (torch.float64,))
    _check(lib().sfft_hash_to_bins_static(n, B, T, _ptr(taps), _ptr(wtab), _ptr(x), sigma, a, b, _ptr(zidx),
                                          _ptr(zval), nz, _ptr(out), _stream_ptr(stream)), "sfft_hash_to_bins_static")
    return out


def sfft_execute_channels(plan: Plan, x, seed: int, id: int, cap: int, outputs=None, stream=None, before=None,
                          after=None):
    """Multi-channel batch with shared hashing (sfft_execute_channels): ``x`` is a torch tensor [n, C]
    complex64 on the GPU (row m = sample m of every channel), every channel transformed with the draws
    of request ``id`` under ``seed``.  ``before`` / ``after`` (torch.cuda.Event, already recorded once
    so that torch has created them) are recorded around the gather kernel.
    Returns (idx [C, cap], val [C, cap, 2], count [C], flag [C]) device tensors, slot c = channel c."""
    import torch

    if x.dim() != 2 or x.dtype != torch.complex64 or not x.is_cuda or not x.is_contiguous():
        raise SfftError(SFFT_ERR_INVALID_ARG, "sfft_execute_channels: need a contiguous [n, C] complex64 CUDA tensor")
    C = x.shape[1]
    if outputs is None:
        dev = x.device
        outputs = (torch.empty((C, cap), dtype=torch.int32, device=dev),
                   torch.empty((C, cap, 2), dtype=torch.float64, device=dev),
                   torch.empty((C,), dtype=torch.int32, device=dev),
                   torch.empty((C,), dtype=torch.int32, device=dev))
    idx, val, count, flag = outputs
    if before is None and after is None:
        _check(lib().sfft_execute_channels(plan.handle, _ptr(x), C, seed, id, _stream_ptr(stream), _ptr(idx), _ptr(val),
                                           cap, _ptr(count), _ptr(flag)), "sfft_execute_channels")
    else:
        ev = lambda e: ctypes.c_void_p(e.cuda_event if e is not None else None)
        _check(lib().sfft_execute_channels_timed(plan.handle, _ptr(x), C, seed, id, _stream_ptr(stream), _ptr(idx),
                                                 _ptr(val), cap, _ptr(count), _ptr(flag), ev(before), ev(after)),
               "sfft_execute_channels_timed")
    return outputs


def sfft_gather_rate(x, row_elems: int, rows: int, idx, per_row: int, sink, stream=None):
    """Measurement: read x[r][idx[r][i]] in the order given (sfft_gather_rate); ``x`` and ``idx`` (int32
    [rows, per_row]) and ``sink`` (int32 [64]) are device tensors."""
    _check(lib().sfft_gather_rate(_ptr(x), row_elems, rows, _ptr(idx), per_row, _ptr(sink), _stream_ptr(stream)),
           "sfft_gather_rate")


def sfft_execute_trace(plan: Plan, x, seed: int, cap: int, round_: int, stream=None):
    """sfft_execute of a general-mode batch that also records round ``round_`` (sfft_execute_trace).

    Returns (outputs as sfft_execute, trace dict of device tensors: bins [batch, nhash, B, 2] float64,
    regions [batch, dmax, B] int64 (uint64 bits), valid [batch, dmax, B] uint8, cand [batch, B] int32
    (uint32 bits), zidx/zval/zcount before and after the round)."""
    import torch

    batch = x.shape[0] if x.dim() == 2 else 1
    dev = x.device
    g = general_round_info(plan, round_)
    B, dmax = g["B"], g["dmax"]
    nhash = 2 * dmax * plan.params.R_loc + plan.params.R_est
    zc = plan.params.z_cap
    tr = dict(bins=torch.zeros((batch, nhash, B, 2), dtype=torch.float64, device=dev),
              regions=torch.zeros((batch, dmax, B), dtype=torch.int64, device=dev),
              valid=torch.zeros((batch, dmax, B), dtype=torch.uint8, device=dev),
              cand=torch.zeros((batch, B), dtype=torch.int32, device=dev),
              zidx_before=torch.zeros((batch, zc), dtype=torch.int32, device=dev),
              zval_before=torch.zeros((batch, zc, 2), dtype=torch.float64, device=dev),
              zcount_before=torch.zeros((batch,), dtype=torch.int32, device=dev),
              zidx_after=torch.zeros((batch, zc), dtype=torch.int32, device=dev),
              zval_after=torch.zeros((batch, zc, 2), dtype=torch.float64, device=dev),
              zcount_after=torch.zeros((batch,), dtype=torch.int32, device=dev))
    st = SfftGeneralTrace(round_, 0, *[tr[k].data_ptr() for k in ("bins", "regions", "valid", "cand", "zidx_before",
                                                                  "zval_before", "zcount_before", "zidx_after",
                                                                  "zval_after", "zcount_after")])
    outputs = (torch.empty((batch, cap), dtype=torch.int32, device=dev),
               torch.empty((batch, cap, 2), dtype=torch.float64, device=dev),
               torch.empty((batch,), dtype=torch.int32, device=dev),
               torch.empty((batch,), dtype=torch.int32, device=dev))
    idx, val, count, flag = outputs
    _check(lib().sfft_execute_trace(plan.handle, _ptr(x), batch, seed, _stream_ptr(stream), _ptr(idx), _ptr(val), cap,
                                    _ptr(count), _ptr(flag), ctypes.byref(st)), "sfft_execute_trace")
    return outputs, tr


def general_round_info(plan: Plan, r: int) -> dict:
    B, kp, dmax, t = (ctypes.c_uint32() for _ in range(4))
    T = ctypes.c_int64()
    lo = (ctypes.c_uint64 * 16)()
    hi = (ctypes.c_uint64 * 16)()
    _check(lib().sfft_plan_general_round_info(plan.handle, r, ctypes.byref(B), ctypes.byref(T), ctypes.byref(kp),
                                              ctypes.byref(dmax), ctypes.byref(t), lo, hi), "sfft_plan_general_round_info")
    return dict(B=B.value, T=T.value, kprime=kp.value, dmax=dmax.value, t=t.value,
                beta_lo=[int(lo[i]) for i in range(dmax.value)], beta_hi=[int(hi[i]) for i in range(dmax.value)])


def sfft_locate_votes(plan: Plan, r: int, sigma: int, b: int, w_fp: int, beta, u, up, l_fp, valid, votes, stream=None):
    """One LocateInner level on device bins; l_fp / valid are updated in place, votes [B, t] filled."""
    _check(lib().sfft_locate_votes(plan.handle, r, sigma, b, w_fp, int(beta.numel()), _ptr(beta), _ptr(u), _ptr(up),
                                   _ptr(l_fp), _ptr(valid), _ptr(votes), _stream_ptr(stream)), "sfft_locate_votes")


def sfft_estimate_from_bins(plan: Plan, r: int, sig, bb, aa, u, L, kprime: int, widx, wval, count, stream=None):
    """EstimateValues on device bins; returns nothing (outputs in widx, wval, count)."""
    nL = 0 if L is None else int(L.numel())
    _check(lib().sfft_estimate_from_bins(plan.handle, r, int(sig.numel()), _ptr(sig), _ptr(bb), _ptr(aa), _ptr(u),
                                         _ptr(L), nL, kprime, _ptr(widx), _ptr(wval), _ptr(count),
                                         _stream_ptr(stream)), "sfft_estimate_from_bins")
