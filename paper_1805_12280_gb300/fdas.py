"""Thin ctypes binding of ``libfdas.so`` (include/fdas.h).

Argument marshalling only: every step of the computation runs in the library's
CUDA kernels.  The low-level functions keep the C names; ``Plan`` wraps them for
torch tensors (torch supplies device memory and streams).  There is no CPU
fallback: if the library cannot be built or loaded, ``load()`` raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import _build

FDAS_OK = 0
FDAS_ERR_INVALID_ARG = -1
FDAS_ERR_OOM = -2
FDAS_ERR_CUDA = -3
FDAS_ERR_TIMEOUT = -4
FDAS_ERR_BUSY = -5
FDAS_ERR_REJECTED = -6
FDAS_ERR_UNSUPPORTED = -7

FDAS_PREC_FP32 = 0
FDAS_PREC_TC_FP16 = 1
FDAS_PREC_TC_DFT2 = 2


class FdasError(RuntimeError):
    def __init__(self, code: int, where: str, message: str):
        super().__init__(f"{where}: {message} (code {code})")
        self.code = code


class fdas_opts(ctypes.Structure):
    _fields_ = [("seg_len", ctypes.c_int), ("tpl_per_cta", ctypes.c_int),
                ("precision", ctypes.c_int), ("autotune", ctypes.c_int), ("group_support", ctypes.c_int),
                ("tune_n_min", ctypes.c_int64)]


class fdas_plan_desc(ctypes.Structure):
    _fields_ = [("n_max", ctypes.c_int64), ("n_templates", ctypes.c_int), ("tpl_len", ctypes.c_int),
                ("frame_len", ctypes.c_int), ("seg_len", ctypes.c_int), ("seg_step", ctypes.c_int),
                ("tpl_per_cta", ctypes.c_int), ("precision", ctypes.c_int), ("device", ctypes.c_int),
                ("device_bytes", ctypes.c_int64), ("tuned", ctypes.c_int), ("tune_ms", ctypes.c_float * 12), ("tune_ms_tc", ctypes.c_float),
                ("batch_blocks", ctypes.c_int), ("groups", ctypes.c_int)]


class fdas_candidate(ctypes.Structure):
    _fields_ = [("tpl", ctypes.c_int32), ("power", ctypes.c_float), ("bin", ctypes.c_int64)]


CANDIDATE_DTYPE = np.dtype([("tpl", "<i4"), ("power", "<f4"), ("bin", "<i8")])


class fdas_harmonic_candidate(ctypes.Structure):
    _fields_ = [("tpl", ctypes.c_int32), ("power", ctypes.c_float), ("bin", ctypes.c_int64),
                ("nharm", ctypes.c_int32), ("reserved", ctypes.c_int32)]


HARMONIC_DTYPE = np.dtype([("tpl", "<i4"), ("power", "<f4"), ("bin", "<i8"), ("nharm", "<i4"),
                           ("reserved", "<i4")])


class fdas_server_opts(ctypes.Structure):
    _fields_ = [("budget_bytes", ctypes.c_int64), ("lanes", ctypes.c_int), ("max_batch", ctypes.c_int)]


class fdas_server_report(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("rejected", ctypes.c_int64),
                ("queued", ctypes.c_int64), ("in_flight", ctypes.c_int64), ("bytes_in_use", ctypes.c_int64),
                ("peak_bytes_in_use", ctypes.c_int64), ("admission_waits", ctypes.c_int64),
                ("launches", ctypes.c_int64), ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double),
                ("mean_ms", ctypes.c_double), ("max_ms", ctypes.c_double), ("arrays_per_s", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


# Every exported symbol with (restype, argtypes).  The CPU tests check that the
# library exports exactly what include/fdas.h declares.
_P = ctypes.c_void_p
_I = ctypes.c_int
_I64 = ctypes.c_int64
SIGNATURES = {
    "fdas_plan_create": (_I, [ctypes.POINTER(_P), _I64, _P, _I, _I, ctypes.POINTER(fdas_opts)]),
    "fdas_plan_describe": (_I, [_P, ctypes.POINTER(fdas_plan_desc)]),
    "fdas_plan_tpl_per_cta": (_I, [_P, _I64]),
    "fdas_convolve": (_I, [_P, _P, _I64, _P, _P]),
    "fdas_convolve_host": (_I, [_P, _P, _I64, _P, _P]),
    "fdas_convolve_batch": (_I, [_P, _I, ctypes.POINTER(_P), ctypes.POINTER(_I64), ctypes.POINTER(_P), _P]),
    "fdas_convolve_candidates": (_I, [_P, _P, _I64, ctypes.c_float, _P, _I64, _P, _P]),
    "fdas_convolve_direct": (_I, [_P, _P, _I64, _P, _P]),
    "fdas_convolve_batch_noalloc": (_I, [_P, _I, ctypes.POINTER(_P), ctypes.POINTER(_I64), ctypes.POINTER(_P), _P]),
    "fdas_plan_status": (_I, [_P, _P]),
    "fdas_selftest_wait_timeout": (_I, [_P, ctypes.c_double, _P]),
    "fdas_server_create": (_I, [ctypes.POINTER(_P), _P, ctypes.POINTER(fdas_server_opts)]),
    "fdas_server_submit": (_I, [_P, _P, _I64, ctypes.POINTER(_I64)]),
    "fdas_server_wait": (_I, [_P, _I64, _I64, ctypes.POINTER(_P)]),
    "fdas_server_release": (_I, [_P, _I64]),
    "fdas_server_stats": (_I, [_P, ctypes.POINTER(fdas_server_report)]),
    "fdas_server_reset_stats": (_I, [_P]),
    "fdas_server_destroy": (_I, [_P]),
    "fdas_destroy": (_I, [_P]),
    "fdas_fdfir_create": (_I, [ctypes.POINTER(_P), _I64, _P, _I, _I]),
    "fdas_fdfir_length": (_I, [_P, ctypes.POINTER(_I64)]),
    "fdas_fdfir_convolve": (_I, [_P, _P, _I64, _P, _P]),
    "fdas_fdfir_destroy": (_I, [_P]),
    "fdas_harmonic_sum": (_I, [_P, _I, _I64, _I64, _I, ctypes.POINTER(ctypes.c_float), _P, _I64, _P, _P]),
    "fdas_strerror": (ctypes.c_char_p, [_I]),
    "fdas_last_error": (ctypes.c_char_p, []),
    "fdas_version": (ctypes.c_char_p, []),
}

_lib = None
_lock = threading.Lock()


def library_path() -> str:
    return _build.LIB


def load(build_if_needed: bool = True) -> ctypes.CDLL:
    """Load (building first if needed) the CUDA library; raises if that is impossible."""
    global _lib
    with _lock:
        if _lib is None:
            if build_if_needed and not _build.up_to_date():
                _build.build()
            if not os.path.exists(_build.LIB):
                raise RuntimeError(f"CUDA library {_build.LIB} is missing; run paper_1805_12280_gb300._build.build()")
            lib = ctypes.CDLL(_build.LIB)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _check(rc: int, where: str) -> None:
    if rc != FDAS_OK:
        lib = load()
        raise FdasError(rc, where, lib.fdas_last_error().decode() or lib.fdas_strerror(rc).decode())


# ---- the C entry points, same names ---------------------------------------

def fdas_plan_create(n_max: int, templates_ptr: int, n_templates: int, tpl_len: int,
                     opts: fdas_opts | None = None) -> int:
    lib = load()
    h = _P()
    _check(lib.fdas_plan_create(ctypes.byref(h), int(n_max), _P(templates_ptr), int(n_templates), int(tpl_len),
                                ctypes.byref(opts) if opts is not None else None), "fdas_plan_create")
    return h.value


def fdas_plan_describe(plan: int) -> fdas_plan_desc:
    d = fdas_plan_desc()
    _check(load().fdas_plan_describe(_P(plan), ctypes.byref(d)), "fdas_plan_describe")
    return d


def fdas_plan_tpl_per_cta(plan: int, n: int) -> int:
    g = load().fdas_plan_tpl_per_cta(_P(plan), int(n))
    _check(min(g, 0), "fdas_plan_tpl_per_cta")
    return g


def fdas_selftest_wait_timeout(plan: int, limit_ms: float, stream: int = 0) -> None:
    _check(load().fdas_selftest_wait_timeout(_P(plan), float(limit_ms), _P(stream)), "fdas_selftest_wait_timeout")


def fdas_convolve(plan: int, in_ptr: int, n: int, out_ptr: int, stream: int = 0) -> None:
    _check(load().fdas_convolve(_P(plan), _P(in_ptr), int(n), _P(out_ptr), _P(stream)), "fdas_convolve")


def fdas_convolve_host(plan: int, in_ptr: int, n: int, out_ptr: int, stream: int = 0) -> None:
    _check(load().fdas_convolve_host(_P(plan), _P(in_ptr), int(n), _P(out_ptr), _P(stream)), "fdas_convolve_host")


def fdas_convolve_direct(plan: int, in_ptr: int, n: int, out_ptr: int, stream: int = 0) -> None:
    _check(load().fdas_convolve_direct(_P(plan), _P(in_ptr), int(n), _P(out_ptr), _P(stream)), "fdas_convolve_direct")


def fdas_convolve_candidates(plan: int, in_ptr: int, n: int, threshold: float, cand_ptr: int, max_cand: int,
                             count_ptr: int, stream: int = 0) -> None:
    _check(load().fdas_convolve_candidates(_P(plan), _P(in_ptr), int(n), float(threshold), _P(cand_ptr),
                                           int(max_cand), _P(count_ptr), _P(stream)), "fdas_convolve_candidates")


def fdas_convolve_batch(plan: int, in_ptrs, ns, out_ptrs, stream: int = 0) -> None:
    count = len(in_ptrs)
    if len(ns) != count or len(out_ptrs) != count:
        raise ValueError("in_ptrs, ns and out_ptrs must have the same length")
    ins = (_P * max(count, 1))(*[_P(int(v)) for v in in_ptrs])
    nn = (_I64 * max(count, 1))(*[int(v) for v in ns])
    outs = (_P * max(count, 1))(*[_P(int(v)) for v in out_ptrs])
    _check(load().fdas_convolve_batch(_P(plan), count, ins, nn, outs, _P(stream)), "fdas_convolve_batch")


def fdas_convolve_batch_noalloc(plan: int, in_ptrs, ns, out_ptrs, stream: int = 0) -> None:
    """Same as fdas_convolve_batch, for callers that cannot allocate GPU memory at call time."""
    count = len(in_ptrs)
    if len(ns) != count or len(out_ptrs) != count:
        raise ValueError("in_ptrs, ns and out_ptrs must have the same length")
    ins = (_P * max(count, 1))(*[_P(int(v)) for v in in_ptrs])
    nn = (_I64 * max(count, 1))(*[int(v) for v in ns])
    outs = (_P * max(count, 1))(*[_P(int(v)) for v in out_ptrs])
    _check(load().fdas_convolve_batch_noalloc(_P(plan), count, ins, nn, outs, _P(stream)),
           "fdas_convolve_batch_noalloc")


def fdas_plan_status(plan: int, stream: int = 0) -> None:
    _check(load().fdas_plan_status(_P(plan), _P(stream)), "fdas_plan_status")


def fdas_server_create(plan: int, budget_bytes: int, lanes: int = 0, max_batch: int = 0) -> int:
    h = _P()
    opts = fdas_server_opts(int(budget_bytes), int(lanes), int(max_batch))
    _check(load().fdas_server_create(ctypes.byref(h), _P(plan), ctypes.byref(opts)), "fdas_server_create")
    return h.value


def fdas_server_submit(server: int, in_ptr: int, n: int) -> int:
    t = _I64()
    _check(load().fdas_server_submit(_P(server), _P(in_ptr), int(n), ctypes.byref(t)), "fdas_server_submit")
    return t.value


def fdas_server_wait(server: int, ticket: int, timeout_ms: int = -1) -> int:
    ptr = _P()
    _check(load().fdas_server_wait(_P(server), int(ticket), int(timeout_ms), ctypes.byref(ptr)), "fdas_server_wait")
    return ptr.value


def fdas_server_release(server: int, ticket: int) -> None:
    _check(load().fdas_server_release(_P(server), int(ticket)), "fdas_server_release")


def fdas_server_stats(server: int) -> dict:
    r = fdas_server_report()
    _check(load().fdas_server_stats(_P(server), ctypes.byref(r)), "fdas_server_stats")
    return r.as_dict()


def fdas_server_reset_stats(server: int) -> None:
    _check(load().fdas_server_reset_stats(_P(server)), "fdas_server_reset_stats")


def fdas_server_destroy(server: int) -> None:
    _check(load().fdas_server_destroy(_P(server)), "fdas_server_destroy")


def fdas_destroy(plan: int) -> None:
    _check(load().fdas_destroy(_P(plan)), "fdas_destroy")


def fdas_version() -> str:
    return load().fdas_version().decode()


def fdas_fdfir_create(n_max: int, templates_ptr: int, n_templates: int, tpl_len: int) -> int:
    h = _P()
    _check(load().fdas_fdfir_create(ctypes.byref(h), int(n_max), _P(templates_ptr), int(n_templates), int(tpl_len)),
           "fdas_fdfir_create")
    return h.value


def fdas_fdfir_length(plan: int) -> int:
    p = _I64()
    _check(load().fdas_fdfir_length(_P(plan), ctypes.byref(p)), "fdas_fdfir_length")
    return p.value


def fdas_fdfir_convolve(plan: int, in_ptr: int, n: int, out_ptr: int, stream: int = 0) -> None:
    _check(load().fdas_fdfir_convolve(_P(plan), _P(in_ptr), int(n), _P(out_ptr), _P(stream)), "fdas_fdfir_convolve")


def fdas_fdfir_destroy(plan: int) -> None:
    _check(load().fdas_fdfir_destroy(_P(plan)), "fdas_fdfir_destroy")


# ---- convenience wrapper for torch tensors ---------------------------------

def fdas_harmonic_sum(plane_ptr: int, n_templates: int, n: int, bin0: int, max_harm: int, thresholds,
                      cand_ptr: int, max_cand: int, count_ptr: int, stream: int = 0) -> None:
    thr = (ctypes.c_float * len(thresholds))(*[float(t) for t in thresholds])
    _check(load().fdas_harmonic_sum(_P(plane_ptr), int(n_templates), int(n), int(bin0), int(max_harm), thr,
                                    _P(cand_ptr), int(max_cand), _P(count_ptr), _P(stream)), "fdas_harmonic_sum")


def harmonic_levels(max_harm: int) -> list:
    """The harmonic counts h = 1, 2, 4, .., max_harm whose sums are thresholded."""
    return [1 << j for j in range(int(max_harm).bit_length())]


def harmonic_thresholds(max_harm: int, sigmas: float = 6.0) -> list:
    """mu + sigmas * sd of a sum of h unit-exponential noise powers (mean h, sd sqrt(h)) for
    each level: at h = 1 this is the single-plane threshold 1 + 6 = 7."""
    return [h + sigmas * float(np.sqrt(h)) for h in harmonic_levels(max_harm)]


def harmonic_sum(plane, bin0: int, max_harm: int = 8, thresholds=None, max_cand: int = 1 << 20, stream=None,
                 buf=None, count=None):
    """Harmonic-sum crossings of a device float32 plane [n_templates, n] (rows z = -c .. c).

    Returns (buf, count): ``buf`` a device int64 tensor [max_cand, 3] holding
    fdas_harmonic_candidate records, ``count`` a device int64 tensor [1] with the number of
    crossings; ``harmonic_to_numpy`` decodes them.  ``thresholds`` defaults to
    ``harmonic_thresholds(max_harm)``.
    """
    import torch
    if plane.dtype != torch.float32 or not plane.is_cuda or not plane.is_contiguous() or plane.dim() != 2:
        raise ValueError("plane must be a contiguous 2-D float32 CUDA tensor")
    if thresholds is None:
        thresholds = harmonic_thresholds(max_harm)
    if len(thresholds) != len(harmonic_levels(max_harm)):
        raise ValueError(f"need {len(harmonic_levels(max_harm))} thresholds for max_harm={max_harm}")
    if buf is None:
        buf = torch.empty((max(max_cand, 1), 3), dtype=torch.int64, device=plane.device)
    if count is None:
        count = torch.empty(1, dtype=torch.int64, device=plane.device)
    with torch.cuda.device(plane.device):
        fdas_harmonic_sum(plane.data_ptr(), plane.shape[0], plane.shape[1], bin0, max_harm, thresholds,
                          buf.data_ptr(), min(max_cand, buf.shape[0]), count.data_ptr(), _stream_handle(stream))
    return buf, count


def harmonic_to_numpy(buf, count) -> np.ndarray:
    """Host copy of the stored harmonic-sum records as a structured array."""
    n = int(count.item()) if hasattr(count, "item") else int(count)
    n = min(n, buf.shape[0])
    return buf[:n].cpu().numpy().view(HARMONIC_DTYPE).reshape(-1)


def _stream_handle(stream) -> int:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream) if hasattr(stream, "cuda_stream") else int(stream)


class Plan:
    """A plan for arrays of up to ``n_max`` points and a fixed template bank.

    ``templates``: complex64 array [M, K] (host).  Options map to ``fdas_opts``.
    """

    def __init__(self, templates, n_max: int, seg_len: int = 2048, tpl_per_cta: int = 0,
                 precision: int = FDAS_PREC_FP32, autotune: int = 0, group_support: int = 0,
                 tune_n_min: int = 0):
        t = np.ascontiguousarray(np.atleast_2d(templates), dtype=np.complex64)
        self.n_templates, self.tpl_len = t.shape
        opts = fdas_opts(seg_len, tpl_per_cta, precision, autotune, group_support, tune_n_min)
        self.handle = fdas_plan_create(n_max, t.ctypes.data, self.n_templates, self.tpl_len, opts)
        self.desc = fdas_plan_describe(self.handle)

    def convolve(self, x, out=None, stream=None):
        """Power plane of device array ``x`` (torch complex64, [n]) into ``out`` ([M, n] float32)."""
        import torch
        if x.dtype != torch.complex64 or not x.is_cuda or not x.is_contiguous():
            raise ValueError("x must be a contiguous complex64 CUDA tensor")
        n = x.numel()
        if out is None:
            out = torch.empty((self.n_templates, n), dtype=torch.float32, device=x.device)
        if out.dtype != torch.float32 or not out.is_contiguous() or out.numel() != self.n_templates * n:
            raise ValueError("out must be a contiguous float32 tensor with M*n elements")
        fdas_convolve(self.handle, x.data_ptr(), n, out.data_ptr(), _stream_handle(stream))
        return out

    def convolve_direct(self, x, out=None, stream=None):
        """The same plane by the time-domain form (Eq. 1 term by term)."""
        import torch
        if x.dtype != torch.complex64 or not x.is_cuda or not x.is_contiguous():
            raise ValueError("x must be a contiguous complex64 CUDA tensor")
        n = x.numel()
        if out is None:
            out = torch.empty((self.n_templates, n), dtype=torch.float32, device=x.device)
        fdas_convolve_direct(self.handle, x.data_ptr(), n, out.data_ptr(), _stream_handle(stream))
        return out

    def candidates(self, x, threshold: float = 7.0, max_cand: int = 1 << 20, stream=None, buf=None, count=None):
        """Threshold crossings of the plane of device array ``x`` (the plane is not written).

        Returns (buf, count): ``buf`` a device int64 tensor [max_cand, 2] holding fdas_candidate
        records, ``count`` a device int64 tensor [1] with the number of crossings found.
        ``candidates_to_numpy`` decodes them on the host.
        """
        import torch
        if x.dtype != torch.complex64 or not x.is_cuda or not x.is_contiguous():
            raise ValueError("x must be a contiguous complex64 CUDA tensor")
        if buf is None:
            buf = torch.empty((max(max_cand, 1), 2), dtype=torch.int64, device=x.device)
        if count is None:
            count = torch.empty(1, dtype=torch.int64, device=x.device)
        fdas_convolve_candidates(self.handle, x.data_ptr(), x.numel(), threshold, buf.data_ptr(),
                                 min(max_cand, buf.shape[0]), count.data_ptr(), _stream_handle(stream))
        return buf, count

    def convolve_batch(self, xs, outs=None, stream=None):
        """Power planes of a list of device arrays in one persistent launch."""
        import torch
        for x in xs:
            if x.dtype != torch.complex64 or not x.is_cuda or not x.is_contiguous():
                raise ValueError("every input must be a contiguous complex64 CUDA tensor")
        if outs is None:
            outs = [torch.empty((self.n_templates, x.numel()), dtype=torch.float32, device=x.device) for x in xs]
        for x, o in zip(xs, outs):
            if o.dtype != torch.float32 or not o.is_contiguous() or o.numel() != self.n_templates * x.numel():
                raise ValueError("each output must be a contiguous float32 tensor with M*n elements")
        fdas_convolve_batch(self.handle, [x.data_ptr() for x in xs], [x.numel() for x in xs],
                            [o.data_ptr() for o in outs], _stream_handle(stream))
        return outs

    def convolve_host(self, x: np.ndarray, out: np.ndarray | None = None, stream=0) -> np.ndarray:
        """Synchronous host-to-host form (host input, host plane)."""
        x = np.ascontiguousarray(x, dtype=np.complex64)
        n = x.size
        if out is None:
            out = np.empty((self.n_templates, n), dtype=np.float32)
        if out.dtype != np.float32 or not out.flags.c_contiguous or out.size != self.n_templates * n:
            raise ValueError("out must be a C-contiguous float32 array with M*n elements")
        fdas_convolve_host(self.handle, x.ctypes.data, n, out.ctypes.data,
                           stream if isinstance(stream, int) else _stream_handle(stream))
        return out

    def status(self, stream=None) -> None:
        fdas_plan_status(self.handle, _stream_handle(stream))

    def close(self) -> None:
        if getattr(self, "handle", None):
            fdas_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class FdFir:
    """Full-length frequency-domain FIR (Eq. 2) over the same template bank: P-point transforms
    of the whole array, P = fdas_fdfir_length (the comparison the paper draws with overlap-save)."""

    def __init__(self, templates, n_max: int):
        t = np.ascontiguousarray(np.atleast_2d(templates), dtype=np.complex64)
        self.n_templates, self.tpl_len = t.shape
        self.handle = fdas_fdfir_create(n_max, t.ctypes.data, self.n_templates, self.tpl_len)
        self.length = fdas_fdfir_length(self.handle)

    def convolve(self, x, out=None, stream=None):
        import torch
        if x.dtype != torch.complex64 or not x.is_cuda or not x.is_contiguous():
            raise ValueError("x must be a contiguous complex64 CUDA tensor")
        n = x.numel()
        if out is None:
            out = torch.empty((self.n_templates, n), dtype=torch.float32, device=x.device)
        fdas_fdfir_convolve(self.handle, x.data_ptr(), n, out.data_ptr(), _stream_handle(stream))
        return out

    def close(self) -> None:
        if self.handle:
            fdas_fdfir_destroy(self.handle)
            self.handle = 0

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Server:
    """Continuous-batching request loop over a Plan (the plan must outlive the server)."""

    def __init__(self, plan: Plan, budget_bytes: int, lanes: int = 0, max_batch: int = 0):
        self.plan = plan
        self.handle = fdas_server_create(plan.handle, budget_bytes, lanes, max_batch)
        self._keep = {}

    def submit(self, x) -> int:
        """Queue device array ``x`` (torch complex64); returns a ticket.  ``x`` is kept alive."""
        t = fdas_server_submit(self.handle, x.data_ptr(), x.numel())
        self._keep[t] = x
        return t

    def wait(self, ticket: int, timeout_ms: int = -1, n: int | None = None):
        """Wait for the plane; returns its device address, or a torch view when ``n`` is given."""
        ptr = fdas_server_wait(self.handle, ticket, timeout_ms)
        if n is None:
            return ptr
        return _device_view(ptr, (self.plan.n_templates, n), self._keep[ticket].device)

    def release(self, ticket: int) -> None:
        fdas_server_release(self.handle, ticket)
        self._keep.pop(ticket, None)

    def stats(self) -> dict:
        return fdas_server_stats(self.handle)

    def reset_stats(self) -> None:
        fdas_server_reset_stats(self.handle)

    def close(self) -> None:
        if getattr(self, "handle", None):
            fdas_server_destroy(self.handle)
            self.handle = None
            self._keep.clear()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _device_view(ptr: int, shape, device):
    """A torch float32 tensor viewing device memory owned by the library (no copy)."""
    import torch

    class _Array:
        def __init__(self):
            self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": "<f4", "data": (int(ptr), False),
                                             "version": 3, "strides": None}
    with torch.cuda.device(device):
        return torch.as_tensor(_Array(), device=device)


def candidates_to_numpy(buf, count) -> np.ndarray:
    """Host copy of the stored candidates as a structured array (tpl, power, bin)."""
    n = int(count.item()) if hasattr(count, "item") else int(count)
    n = min(n, buf.shape[0])
    return buf[:n].cpu().numpy().view(CANDIDATE_DTYPE).reshape(-1)
