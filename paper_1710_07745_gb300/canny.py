"""Thin ctypes binding of libcanny's C ABI (``include/canny.h``).

The functions keep the C names and argument order; only marshalling happens
here (torch tensors and streams become raw pointers). Every step of the edge
detector runs in the CUDA library. There is no CPU fallback: if the library
is missing or no CUDA device is visible, calls raise.
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import Sequence

from . import build as _build

CANNY_OK, CANNY_EINVAL, CANNY_ENOMEM, CANNY_ECUDA, CANNY_ENOCONVERGE, CANNY_EUNSUPPORTED = range(6)
CANNY_PATH_INT, CANNY_PATH_F32 = 0, 1


class CannyError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {strerror(status)} (status {status})")


class canny_params(ctypes.Structure):
    _fields_ = [("path", ctypes.c_int), ("sigma", ctypes.c_float), ("ksize", ctypes.c_int),
                ("low", ctypes.c_float), ("high", ctypes.c_float), ("max_passes", ctypes.c_int)]


class canny_image(ctypes.Structure):
    _fields_ = [("d_in", ctypes.c_void_p), ("d_out", ctypes.c_void_p), ("w", ctypes.c_int),
                ("h", ctypes.c_int), ("in_pitch", ctypes.c_int), ("out_pitch", ctypes.c_int)]


class canny_stats(ctypes.Structure):
    _fields_ = [("images", ctypes.c_int64), ("pixels", ctypes.c_int64), ("tiles", ctypes.c_int64),
                ("hyst_passes", ctypes.c_int64), ("hyst_tiles_visited", ctypes.c_int64),
                ("pending_tiles", ctypes.c_int64), ("status", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}


class canny_timing(ctypes.Structure):
    _fields_ = [("runs", ctypes.c_int64), ("reset_ms", ctypes.c_double), ("stencil_ms", ctypes.c_double),
                ("local_ms", ctypes.c_double), ("global_ms", ctypes.c_double), ("total_ms", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class canny_tuning(ctypes.Structure):
    _fields_ = [("band", ctypes.c_int), ("ctas_per_sm", ctypes.c_int), ("ms", ctypes.c_double),
                ("from_cache", ctypes.c_int), ("direct_loads", ctypes.c_int), ("chase_budget", ctypes.c_int),
                ("batch_passes", ctypes.c_int)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class canny_request(ctypes.Structure):
    _fields_ = [("w", ctypes.c_int), ("h", ctypes.c_int), ("h_in", ctypes.c_void_p), ("h_pitch", ctypes.c_int),
                ("h_out", ctypes.c_void_p), ("out_pitch", ctypes.c_int), ("arrival_s", ctypes.c_double)]


class canny_serve_config(ctypes.Structure):
    _fields_ = [("memory_budget_bytes", ctypes.c_double), ("streams", ctypes.c_int),
                ("max_batch_images", ctypes.c_int), ("max_batch_pixels", ctypes.c_int64),
                ("serial", ctypes.c_int), ("low", ctypes.c_int), ("high", ctypes.c_int),
                ("band", ctypes.c_int), ("ctas_per_sm", ctypes.c_int)]


class canny_fault_injection(ctypes.Structure):
    _fields_ = [("device_allocations", ctypes.c_int), ("arena_admissions", ctypes.c_int),
                ("stalled_barriers", ctypes.c_int), ("host_driven_passes", ctypes.c_int)]


class canny_serve_report(ctypes.Structure):
    _fields_ = [("completed", ctypes.c_int64), ("wall_s", ctypes.c_double), ("delivered_mpx_s", ctypes.c_double),
                ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double), ("max_ms", ctypes.c_double),
                ("batches", ctypes.c_int64), ("mean_batch_images", ctypes.c_double), ("peak_bytes", ctypes.c_int64),
                ("deferrals", ctypes.c_int64)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None
_lock = threading.Lock()

# C name -> (argtypes, restype); every symbol include/canny.h declares
_P = ctypes.c_void_p
SIGNATURES = {
    "canny_params_default": ([ctypes.POINTER(canny_params)], ctypes.c_int),
    "canny_create": ([ctypes.c_int, ctypes.c_int, ctypes.POINTER(canny_params), ctypes.POINTER(_P)],
                     ctypes.c_int),
    "canny_destroy": ([_P], None),
    "canny_run": ([_P, _P, _P, _P], ctypes.c_int),
    "canny_run_pitched": ([_P, ctypes.POINTER(canny_image), _P], ctypes.c_int),
    "canny_run_batch": ([_P, ctypes.c_int, ctypes.POINTER(canny_image), _P], ctypes.c_int),
    "canny_run_host": ([_P, _P, ctypes.c_int, _P, ctypes.c_int, ctypes.c_int, ctypes.c_int, _P],
                       ctypes.c_int),
    "canny_run_frames": ([_P, ctypes.c_int, ctypes.POINTER(_P), ctypes.c_int, ctypes.POINTER(_P), ctypes.c_int,
                          ctypes.c_int, ctypes.c_int, _P], ctypes.c_int),
    "canny_classify": ([_P, ctypes.POINTER(canny_image), _P], ctypes.c_int),
    "canny_hysteresis": ([_P, ctypes.POINTER(canny_image), _P], ctypes.c_int),
    "canny_magnitude_f32": ([_P, ctypes.POINTER(canny_image), _P, ctypes.c_int, _P, _P],
                            ctypes.c_int),
    "canny_get_stats": ([_P, ctypes.POINTER(canny_stats)], ctypes.c_int),
    "canny_enable_timing": ([_P, ctypes.c_int], ctypes.c_int),
    "canny_set_tuning": ([_P, ctypes.POINTER(canny_tuning)], ctypes.c_int),
    "canny_get_tuning": ([_P, ctypes.POINTER(canny_tuning)], ctypes.c_int),
    "canny_autotune_batch": ([_P, ctypes.c_int, ctypes.POINTER(canny_image), _P, ctypes.c_char_p,
                              ctypes.POINTER(canny_tuning)], ctypes.c_int),
    "canny_serve": ([ctypes.POINTER(canny_serve_config), ctypes.c_int, ctypes.POINTER(canny_request), _P,
                     ctypes.POINTER(canny_serve_report)], ctypes.c_int),
    "canny_read_timing": ([_P, ctypes.POINTER(canny_timing)], ctypes.c_int),
    "canny_run_noalloc": ([_P, ctypes.c_int, _P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                           ctypes.c_int, _P], ctypes.c_int),
    "canny_strerror": ([ctypes.c_int], ctypes.c_char_p),
    "canny_inject_faults": ([ctypes.POINTER(canny_fault_injection)], ctypes.c_int),
}


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load libcanny.so (building it first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is None:
            if build_if_missing:
                _build.build()
            if not os.path.exists(_build.LIB):
                raise RuntimeError(f"libcanny.so not built ({_build.LIB}); run __graft_entry__.build()")
            L = ctypes.CDLL(_build.LIB)
            for name, (args, res) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.argtypes = args
                fn.restype = res
            _lib = L
        return _lib


_checked = None


def load_checked() -> ctypes.CDLL:
    """Load the checked build (-DCANNY_CHECKS: device-side bounds checks that set
    error bit 3, reported as CANNY_ECUDA, instead of faulting), building it first."""
    global _checked
    with _lock:
        if _checked is None:
            L = ctypes.CDLL(_build.build(checks=True))
            for name, (args, res) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.argtypes = args
                fn.restype = res
            _checked = L
        return _checked


def canny_inject_faults(device_allocations: int = 0, arena_admissions: int = 0, stalled_barriers: int = 0,
                        host_driven_passes: int = 0) -> None:
    """Test hook: make the library's next allocations, serving admissions or
    single-image hysteresis barriers fail, or the next single-image runs drive
    their global passes from the host (see include/canny.h)."""
    f = canny_fault_injection(device_allocations, arena_admissions, stalled_barriers, host_driven_passes)
    _check(load().canny_inject_faults(ctypes.byref(f)), "canny_inject_faults")


def strerror(status: int) -> str:
    return load().canny_strerror(status).decode()


def _check(status: int, where: str) -> None:
    if status != CANNY_OK:
        raise CannyError(status, where)


# ------------------------------------------------------------------ C-named calls
def canny_params_default() -> canny_params:
    p = canny_params()
    _check(load().canny_params_default(ctypes.byref(p)), "canny_params_default")
    return p


def canny_create(max_w: int, max_h: int, params: canny_params) -> int:
    ctx = _P()
    _check(load().canny_create(max_w, max_h, ctypes.byref(params), ctypes.byref(ctx)), "canny_create")
    return ctx.value


def canny_destroy(ctx: int) -> None:
    load().canny_destroy(ctx)


def canny_run(ctx: int, d_in: int, d_out: int, stream: int = 0) -> None:
    _check(load().canny_run(ctx, d_in, d_out, stream), "canny_run")


def canny_run_pitched(ctx: int, img: canny_image, stream: int = 0) -> None:
    _check(load().canny_run_pitched(ctx, ctypes.byref(img), stream), "canny_run_pitched")


def canny_run_batch(ctx: int, imgs: Sequence[canny_image], stream: int = 0) -> None:
    arr = (canny_image * len(imgs))(*imgs)
    _check(load().canny_run_batch(ctx, len(imgs), arr, stream), "canny_run_batch")


def canny_run_host(ctx: int, h_in: int, in_pitch: int, h_out: int, out_pitch: int, w: int, h: int,
                   stream: int = 0) -> None:
    _check(load().canny_run_host(ctx, h_in, in_pitch, h_out, out_pitch, w, h, stream), "canny_run_host")


def canny_run_frames(ctx: int, h_in: Sequence[int], in_pitch: int, h_out: Sequence[int], out_pitch: int,
                     w: int, h: int, stream: int = 0) -> None:
    """n frames on host buffers (addresses h_in[i] / h_out[i]), uploads, pipelines and
    downloads of consecutive frames overlapped."""
    n = len(h_in)
    if len(h_out) != n:
        raise ValueError("h_in and h_out differ in length")
    arr_in = (_P * max(n, 1))(*h_in)
    arr_out = (_P * max(n, 1))(*h_out)
    _check(load().canny_run_frames(ctx, n, arr_in, in_pitch, arr_out, out_pitch, w, h, stream), "canny_run_frames")


def canny_classify(ctx: int, img: canny_image, stream: int = 0) -> None:
    _check(load().canny_classify(ctx, ctypes.byref(img), stream), "canny_classify")


def canny_hysteresis(ctx: int, img: canny_image, stream: int = 0) -> None:
    _check(load().canny_hysteresis(ctx, ctypes.byref(img), stream), "canny_hysteresis")


def canny_magnitude_f32(ctx: int, img: canny_image, d_mag: int, d_mag_pitch: int, d_max: int,
                        stream: int = 0) -> None:
    _check(load().canny_magnitude_f32(ctx, ctypes.byref(img), d_mag, d_mag_pitch, d_max, stream),
           "canny_magnitude_f32")


def canny_get_stats(ctx: int) -> canny_stats:
    st = canny_stats()
    _check(load().canny_get_stats(ctx, ctypes.byref(st)), "canny_get_stats")
    return st


def canny_enable_timing(ctx: int, enable: bool) -> None:
    _check(load().canny_enable_timing(ctx, 1 if enable else 0), "canny_enable_timing")


def canny_read_timing(ctx: int) -> canny_timing:
    t = canny_timing()
    _check(load().canny_read_timing(ctx, ctypes.byref(t)), "canny_read_timing")
    return t


def canny_run_noalloc(d_in: int, in_pitch: int, d_out: int, out_pitch: int, w: int, h: int,
                      low: int, high: int, stream: int = 0) -> None:
    """Integer pipeline with no device allocation (fixed scratch, at most 16384 tiles)."""
    _check(load().canny_run_noalloc(d_in, in_pitch, d_out, out_pitch, w, h, low, high, stream),
           "canny_run_noalloc")


def canny_set_tuning(ctx: int, band: int, ctas_per_sm: int, direct_loads: int = 0, chase_budget: int = 0,
                     batch_passes: int = 0) -> None:
    t = canny_tuning(band, ctas_per_sm, 0.0, 0, direct_loads, chase_budget, batch_passes)
    _check(load().canny_set_tuning(ctx, ctypes.byref(t)), "canny_set_tuning")


def canny_get_tuning(ctx: int) -> canny_tuning:
    t = canny_tuning()
    _check(load().canny_get_tuning(ctx, ctypes.byref(t)), "canny_get_tuning")
    return t


def canny_autotune_batch(ctx: int, imgs: Sequence[canny_image], stream: int = 0,
                         cache_path: str | None = None) -> canny_tuning:
    arr = (canny_image * len(imgs))(*imgs)
    t = canny_tuning()
    cp = cache_path.encode() if cache_path else None
    _check(load().canny_autotune_batch(ctx, len(imgs), arr, stream, cp, ctypes.byref(t)),
           "canny_autotune_batch")
    return t


def canny_serve(cfg: canny_serve_config, reqs, latency_ms=None) -> canny_serve_report:
    """Serve a request trace (sequence of canny_request); latency_ms: optional float64 array."""
    arr = (canny_request * len(reqs))(*reqs)
    rep = canny_serve_report()
    lat = latency_ms.ctypes.data if latency_ms is not None else None
    _check(load().canny_serve(ctypes.byref(cfg), len(reqs), arr, lat, ctypes.byref(rep)), "canny_serve")
    return rep


# ------------------------------------------------------------------ torch marshalling
def _stream_ptr(stream) -> int:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def image_of(t_in, t_out, w: int | None = None, h: int | None = None) -> canny_image:
    """canny_image over two 2-D uint8 CUDA tensors (row stride = pitch)."""
    for t in (t_in, t_out):
        if not t.is_cuda or t.dtype.itemsize != 1 or t.dim() != 2:
            raise ValueError("expected 2-D uint8 CUDA tensors")
        if t.numel() and t.stride(1) != 1:
            raise ValueError("expected unit column stride")
    hh = t_in.shape[0] if h is None else h
    ww = t_in.shape[1] if w is None else w
    if ww == 0 or hh == 0:
        return canny_image(0, 0, ww, hh, 0, 0)
    return canny_image(t_in.data_ptr(), t_out.data_ptr(), ww, hh, t_in.stride(0), t_out.stride(0))


class Canny:
    """A context (``canny_create``) with torch-tensor convenience calls."""

    def __init__(self, max_w: int, max_h: int, *, path: int = CANNY_PATH_INT, low: float = 40.0,
                 high: float = 100.0, sigma: float = 1.4, ksize: int = 7, max_passes: int = 0):
        p = canny_params_default()
        p.path, p.low, p.high, p.sigma, p.ksize, p.max_passes = path, low, high, sigma, ksize, max_passes
        self.max_w, self.max_h, self.params = max_w, max_h, p
        self.ctx = canny_create(max_w, max_h, p)

    def close(self) -> None:
        if self.ctx:
            canny_destroy(self.ctx)
            self.ctx = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def run(self, t_in, t_out, stream=None) -> None:
        """Tight max_w x max_h image: canny_run."""
        canny_run(self.ctx, t_in.data_ptr(), t_out.data_ptr(), _stream_ptr(stream))

    def run_pitched(self, t_in, t_out, stream=None) -> None:
        canny_run_pitched(self.ctx, image_of(t_in, t_out), _stream_ptr(stream))

    def run_batch(self, pairs, stream=None) -> None:
        canny_run_batch(self.ctx, [image_of(a, b) for a, b in pairs], _stream_ptr(stream))

    def classify(self, t_in, t_cls, stream=None) -> None:
        canny_classify(self.ctx, image_of(t_in, t_cls), _stream_ptr(stream))

    def hysteresis(self, t_cls, t_out, stream=None) -> None:
        canny_hysteresis(self.ctx, image_of(t_cls, t_out), _stream_ptr(stream))

    def magnitude(self, t_in, t_mag, t_max, stream=None) -> None:
        img = canny_image(t_in.data_ptr(), 0, t_in.shape[1], t_in.shape[0], t_in.stride(0), 0)
        canny_magnitude_f32(self.ctx, img, t_mag.data_ptr(), t_mag.stride(0), t_max.data_ptr(),
                            _stream_ptr(stream))

    def autotune_batch(self, pairs, stream=None, cache_path: str | None = None) -> dict:
        return canny_autotune_batch(self.ctx, [image_of(a, b) for a, b in pairs], _stream_ptr(stream),
                                    cache_path).as_dict()

    def set_tuning(self, band: int, ctas_per_sm: int, direct_loads: int = 0, chase_budget: int = 0,
                   batch_passes: int = 0) -> None:
        canny_set_tuning(self.ctx, band, ctas_per_sm, direct_loads, chase_budget, batch_passes)

    def stats(self) -> dict:
        return canny_get_stats(self.ctx).as_dict()
