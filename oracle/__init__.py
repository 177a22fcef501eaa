"""CPU oracle for the Canny pipeline (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
legs import this package. It wraps ``canny_oracle.c`` (plain single-threaded
C, one function per step of the paper's Sec. 2.2.1 pipeline) with ctypes and
numpy; it shares nothing with the CUDA library.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "canny_oracle.c")
_HDR = os.path.join(_HERE, "canny_oracle.h")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

SECTOR_H, SECTOR_V, SECTOR_D, SECTOR_A = 0, 1, 2, 3
NONE, WEAK, STRONG = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile canny_oracle.c with gcc into oracle/_build/liboracle.so."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= newest:
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.run(
        ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
         "-shared", _SRC, "-o", tmp, "-lm"],
        check=True,
    )
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            P = ctypes.c_void_p
            i, i64, f = ctypes.c_int, ctypes.c_int64, ctypes.c_float
            sig = {
                "oracle_gauss5_u8": [P, i, i, i, P],
                "oracle_sobel_u8": [P, i, i, P, P],
                "oracle_mag2_i32": [P, P, i64, P],
                "oracle_sector_map_i": [P, P, i64, P],
                "oracle_nms_classify_u8": [P, P, P, i, i, i64, i64, P],
                "oracle_hysteresis": [P, i, i, P, i],
                "oracle_classify_u8": [P, i, i, i, i, i, P],
                "oracle_canny_u8": [P, i, i, i, i, i, P, i],
                "oracle_gauss_taps_f32": [f, i, P],
                "oracle_gauss_f32": [P, i, i, i, f, i, P],
                "oracle_sobel_f32": [P, i, i, P, P],
                "oracle_magnitude_f32": [P, P, i64, P],
                "oracle_nms_classify_f32": [P, P, P, i, i, f, f, P],
                "oracle_canny_f32": [P, i, i, i, f, i, f, f, P, i, P, P],
            }
            for name, args in sig.items():
                fn = getattr(L, name)
                fn.argtypes = args
                fn.restype = None
            L.oracle_sector_i.argtypes = [i, i]
            L.oracle_sector_i.restype = i
            L.oracle_sector_tan_q15.argtypes = []
            L.oracle_sector_tan_q15.restype = i
            L.oracle_sector_f.argtypes = [f, f]
            L.oracle_sector_f.restype = i
            L.oracle_max_f32.argtypes = [P, i64]
            L.oracle_max_f32.restype = f
            _lib = L
        return _lib


def _p(a: np.ndarray) -> int:
    return a.ctypes.data


def _img(img: np.ndarray) -> tuple[np.ndarray, int, int, int]:
    """Return (array, w, h, pitch) for a 2-D uint8 image with unit column stride."""
    img = np.asarray(img)
    assert img.dtype == np.uint8 and img.ndim == 2
    if img.strides[1] != 1 or img.strides[0] < img.shape[1]:
        img = np.ascontiguousarray(img)
    h, w = img.shape
    pitch = img.strides[0] if h > 0 else w
    return img, w, h, pitch


# ---------------------------------------------------------------- integer path
def gauss5_u8(img):
    img, w, h, pitch = _img(img)
    S = np.empty((h, w), np.uint8)
    if w * h:
        lib().oracle_gauss5_u8(_p(img), w, h, pitch, _p(S))
    return S


def sobel_u8(S):
    S = np.ascontiguousarray(S, dtype=np.uint8)
    h, w = S.shape
    gx = np.empty((h, w), np.int16)
    gy = np.empty((h, w), np.int16)
    if w * h:
        lib().oracle_sobel_u8(_p(S), w, h, _p(gx), _p(gy))
    return gx, gy


def mag2_i32(gx, gy):
    gx = np.ascontiguousarray(gx, dtype=np.int16)
    gy = np.ascontiguousarray(gy, dtype=np.int16)
    m2 = np.empty(gx.shape, np.int32)
    lib().oracle_mag2_i32(_p(gx), _p(gy), gx.size, _p(m2))
    return m2


def sector_tan_q15() -> int:
    return lib().oracle_sector_tan_q15()


def sector_i(gx: int, gy: int) -> int:
    return lib().oracle_sector_i(int(gx), int(gy))


def sector_map_i(gx, gy):
    gx = np.ascontiguousarray(gx, dtype=np.int32)
    gy = np.ascontiguousarray(gy, dtype=np.int32)
    out = np.empty(gx.shape, np.uint8)
    lib().oracle_sector_map_i(_p(gx), _p(gy), gx.size, _p(out))
    return out


def nms_classify_u8(gx, gy, m2, low: int, high: int):
    gx = np.ascontiguousarray(gx, dtype=np.int16)
    gy = np.ascontiguousarray(gy, dtype=np.int16)
    m2 = np.ascontiguousarray(m2, dtype=np.int32)
    h, w = m2.shape
    cls = np.empty((h, w), np.uint8)
    if w * h:
        lib().oracle_nms_classify_u8(_p(gx), _p(gy), _p(m2), w, h, low * low, high * high, _p(cls))
    return cls


def hysteresis(cls, out: np.ndarray | None = None):
    cls = np.ascontiguousarray(cls, dtype=np.uint8)
    h, w = cls.shape
    if out is None:
        out = np.zeros((h, w), np.uint8)
    assert out.dtype == np.uint8 and out.strides[1] == 1 and out.shape[1] >= w
    if w * h:
        lib().oracle_hysteresis(_p(cls), w, h, _p(out), out.strides[0])
    return out


def classify_u8(img, low: int = 40, high: int = 100):
    img, w, h, pitch = _img(img)
    cls = np.empty((h, w), np.uint8)
    if w * h:
        lib().oracle_classify_u8(_p(img), w, h, pitch, low, high, _p(cls))
    return cls


def canny_u8(img, low: int = 40, high: int = 100, out: np.ndarray | None = None):
    img, w, h, pitch = _img(img)
    if out is None:
        out = np.zeros((h, w), np.uint8)
    if w * h:
        lib().oracle_canny_u8(_p(img), w, h, pitch, low, high, _p(out), out.strides[0])
    return out


# ---------------------------------------------------------------- float32 variant
def gauss_taps_f32(sigma: float = 1.4, ksize: int = 7):
    t = np.empty(ksize, np.float32)
    lib().oracle_gauss_taps_f32(sigma, ksize, _p(t))
    return t


def gauss_f32(img, sigma: float = 1.4, ksize: int = 7):
    img, w, h, pitch = _img(img)
    S = np.empty((h, w), np.float32)
    if w * h:
        lib().oracle_gauss_f32(_p(img), w, h, pitch, sigma, ksize, _p(S))
    return S


def sobel_f32(S):
    S = np.ascontiguousarray(S, dtype=np.float32)
    h, w = S.shape
    gx = np.empty((h, w), np.float32)
    gy = np.empty((h, w), np.float32)
    if w * h:
        lib().oracle_sobel_f32(_p(S), w, h, _p(gx), _p(gy))
    return gx, gy


def magnitude_f32(gx, gy):
    gx = np.ascontiguousarray(gx, dtype=np.float32)
    gy = np.ascontiguousarray(gy, dtype=np.float32)
    M = np.empty(gx.shape, np.float32)
    lib().oracle_magnitude_f32(_p(gx), _p(gy), gx.size, _p(M))
    return M


def max_f32(M) -> float:
    M = np.ascontiguousarray(M, dtype=np.float32)
    return float(lib().oracle_max_f32(_p(M), M.size))


def sector_f(gx: float, gy: float) -> int:
    return lib().oracle_sector_f(float(gx), float(gy))


def nms_classify_f32(gx, gy, M, lo_t: float, hi_t: float):
    gx = np.ascontiguousarray(gx, dtype=np.float32)
    gy = np.ascontiguousarray(gy, dtype=np.float32)
    M = np.ascontiguousarray(M, dtype=np.float32)
    h, w = M.shape
    cls = np.empty((h, w), np.uint8)
    if w * h:
        lib().oracle_nms_classify_f32(_p(gx), _p(gy), _p(M), w, h, lo_t, hi_t, _p(cls))
    return cls


def canny_f32(img, sigma: float = 1.4, ksize: int = 7, lo_frac: float = 0.1,
              hi_frac: float = 0.3, out: np.ndarray | None = None, want_stages: bool = False):
    """Whole float32 pipeline. Returns the edge map, or (edges, M, class map)."""
    img, w, h, pitch = _img(img)
    if out is None:
        out = np.zeros((h, w), np.uint8)
    M = np.zeros((h, w), np.float32)
    cls = np.zeros((h, w), np.uint8)
    if w * h:
        lib().oracle_canny_f32(_p(img), w, h, pitch, sigma, ksize, lo_frac, hi_frac,
                               _p(out), out.strides[0], _p(M), _p(cls))
    return (out, M, cls) if want_stages else out
