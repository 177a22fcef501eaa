"""Seeded synthetic inputs (the only code the oracle and the CUDA path share).

``synth.c`` draws the images: a linear-gradient background, filled rectangles
and disks of uniform random intensity, additive Gaussian-like noise, clamped
to [0, 255]. This module compiles it with gcc on first use and wraps it with
numpy. It contains none of the edge detector's arithmetic.

Workloads (the paper's unpublished photographs, Sec. 2.2 and Fig. 7, are
replaced by these images):

==========  ==========================  =====================  ==============
name        size                        objects per kind       noise sigma
==========  ==========================  =====================  ==============
small       512 x 512, seed 1000        20                     8
medium      4096 x 4096, seed 2000      200                    8
uhd         7680 x 4320, seed 3000      round(200 A / 4096^2)  12
huge        16384 x 16384, seed 3001    round(200 A / 4096^2)  12
batch       1024 images, seeds 4000+i,  max(2, round(200 A /   8
            sides log-uniform [64,2048]  4096^2))
serve       sides log-uniform           as batch               8
            [128, 4096]
==========  ==========================  =====================  ==============
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libcanny_synth.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    os.makedirs(_OUT_DIR, exist_ok=True)
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.run(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-pthread", _SRC,
                    "-o", tmp, "-lm"], check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _L() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            L.synth_image.argtypes = [ctypes.c_uint64, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                      ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                      ctypes.c_void_p]
            L.synth_image.restype = ctypes.c_int
            L.synth_log_uniform_sizes.argtypes = [ctypes.c_uint64, ctypes.c_int, ctypes.c_int,
                                                  ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
            L.synth_log_uniform_sizes.restype = None
            L.synth_poisson_arrivals.argtypes = [ctypes.c_uint64, ctypes.c_int, ctypes.c_double,
                                                 ctypes.c_void_p]
            L.synth_poisson_arrivals.restype = None
            _lib = L
        return _lib


def objects_for_area(w: int, h: int, minimum: int = 2) -> int:
    """Objects per kind scaled by area: 200 per 4096^2 pixels."""
    return max(minimum, int(round(200.0 * w * h / (4096.0 * 4096.0))))


def image(seed: int, w: int, h: int, n_rect: int | None = None, n_disk: int | None = None,
          noise_sigma: int = 8, pitch: int | None = None, threads: int | None = None,
          out: np.ndarray | None = None) -> np.ndarray:
    """One synthetic uint8 image of h rows and w columns.

    With ``pitch`` > w the result is a (h, pitch) array whose first w columns
    hold the image; the padding bytes are zero.
    """
    if n_rect is None:
        n_rect = objects_for_area(w, h)
    if n_disk is None:
        n_disk = n_rect
    if pitch is None:
        pitch = w
    if threads is None:
        threads = min(os.cpu_count() or 1, 64)
    if out is None:
        out = np.zeros((h, pitch), np.uint8)
    assert out.dtype == np.uint8 and out.flags.c_contiguous and out.shape == (h, pitch)
    if w and h:
        rc = _L().synth_image(seed, w, h, pitch, n_rect, n_disk, noise_sigma, threads,
                              out.ctypes.data)
        if rc != 0:
            raise ValueError("synth_image: bad arguments")
    return out


def log_uniform_sizes(seed: int, n: int, lo: int, hi: int) -> tuple[np.ndarray, np.ndarray]:
    ws = np.empty(n, np.int32)
    hs = np.empty(n, np.int32)
    _L().synth_log_uniform_sizes(seed, n, lo, hi, ws.ctypes.data, hs.ctypes.data)
    return ws, hs


def poisson_arrivals(seed: int, n: int, rate: float) -> np.ndarray:
    t = np.empty(n, np.float64)
    _L().synth_poisson_arrivals(seed, n, rate, t.ctypes.data)
    return t


# ----------------------------------------------------------------- named workloads
def small() -> np.ndarray:
    return image(1000, 512, 512, 20, 20, 8)


def medium() -> np.ndarray:
    return image(2000, 4096, 4096, 200, 200, 8)


def uhd() -> np.ndarray:
    n = objects_for_area(7680, 4320)
    return image(3000, 7680, 4320, n, n, 12)


def huge() -> np.ndarray:
    n = objects_for_area(16384, 16384)
    return image(3001, 16384, 16384, n, n, 12)


def batch_sizes(n: int = 1024, lo: int = 64, hi: int = 2048, seed: int = 4000):
    return log_uniform_sizes(seed, n, lo, hi)


def batch_image(i: int, w: int, h: int, seed_base: int = 4000) -> np.ndarray:
    n = objects_for_area(w, h)
    return image(seed_base + i, w, h, n, n, 8, threads=1)
