"""The C-ABI library builds, loads and exports every symbol include/canny.h declares;
host-side argument checks reject bad input before any CUDA call (no GPU needed)."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

pytestmark = pytest.mark.skipif(shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"),
                                reason="CUDA toolkit not present")


def _declared_symbols(header):
    text = open(header).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(canny_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_1710_07745_gb300 import canny
    return canny.load()


def test_header_declares_the_boundary():
    syms = _declared_symbols(os.path.join(ROOT, "include", "canny.h"))
    for s in ("canny_create", "canny_run", "canny_run_batch", "canny_run_pitched", "canny_destroy",
              "canny_strerror", "canny_get_stats"):
        assert s in syms


def test_library_exports_every_declared_symbol(lib):
    from paper_1710_07745_gb300 import canny
    for header in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if header.endswith(".h"):
            for sym in _declared_symbols(os.path.join(ROOT, "include", header)):
                assert hasattr(lib, sym), f"{sym} declared in {header} but not exported"
    # and the binding knows every one of them
    for sym in _declared_symbols(os.path.join(ROOT, "include", "canny.h")):
        assert sym in canny.SIGNATURES, sym


def test_checked_build_exports_the_same_symbols():
    # the -DCANNY_CHECKS library (device bounds checks) is a drop-in copy of the ABI
    from paper_1710_07745_gb300 import canny
    checked = canny.load_checked()
    for sym in _declared_symbols(os.path.join(ROOT, "include", "canny.h")):
        assert hasattr(checked, sym), f"{sym} not exported by the checked build"
    assert checked.canny_strerror(canny.CANNY_OK) == canny.load().canny_strerror(canny.CANNY_OK)


def test_strerror_and_defaults(lib):
    from paper_1710_07745_gb300 import canny
    assert canny.strerror(canny.CANNY_OK) == "ok"
    assert "converge" in canny.strerror(canny.CANNY_ENOCONVERGE)
    p = canny.canny_params_default()
    assert (p.path, p.low, p.high, p.ksize, p.max_passes) == (0, 40.0, 100.0, 7, 0)
    assert abs(p.sigma - 1.4) < 1e-6


@pytest.mark.parametrize("field,value", [("path", 7), ("low", 120.0), ("low", -1.0), ("high", 40.5),
                                         ("high", 40000.0), ("max_passes", -3)])
def test_create_rejects_bad_params_without_cuda(lib, field, value):
    from paper_1710_07745_gb300 import canny
    p = canny.canny_params_default()
    setattr(p, field, value)
    ctx = ctypes.c_void_p()
    assert lib.canny_create(64, 64, ctypes.byref(p), ctypes.byref(ctx)) == canny.CANNY_EINVAL
    assert not ctx.value


@pytest.mark.parametrize("sigma,ksize", [(0.0, 7), (1.4, 6), (1.4, 1), (1.4, 33)])
def test_create_rejects_bad_float_params(lib, sigma, ksize):
    from paper_1710_07745_gb300 import canny
    p = canny.canny_params_default()
    p.path, p.sigma, p.ksize, p.low, p.high = canny.CANNY_PATH_F32, sigma, ksize, 0.1, 0.3
    ctx = ctypes.c_void_p()
    assert lib.canny_create(64, 64, ctypes.byref(p), ctypes.byref(ctx)) == canny.CANNY_EINVAL


def test_create_rejects_bad_sizes_and_nulls(lib):
    from paper_1710_07745_gb300 import canny
    p = canny.canny_params_default()
    ctx = ctypes.c_void_p()
    for w, h in [(0, 10), (10, 0), (-1, 5)]:
        assert lib.canny_create(w, h, ctypes.byref(p), ctypes.byref(ctx)) == canny.CANNY_EINVAL
    assert lib.canny_create(8, 8, None, ctypes.byref(ctx)) == canny.CANNY_EINVAL
    assert lib.canny_create(8, 8, ctypes.byref(p), None) == canny.CANNY_EINVAL
    assert lib.canny_run(None, None, None, None) == canny.CANNY_EINVAL
    assert lib.canny_get_stats(None, None) == canny.CANNY_EINVAL
    lib.canny_destroy(None)


def test_inject_faults_rejects_negative_counts(lib):
    import ctypes
    from paper_1710_07745_gb300 import canny
    for bad in [(-1, 0, 0, 0), (0, -2, 0, 0), (0, 0, -3, 0), (0, 0, 0, -4)]:
        f = canny.canny_fault_injection(*bad)
        assert lib.canny_inject_faults(ctypes.byref(f)) == canny.CANNY_EINVAL
    assert lib.canny_inject_faults(None) == canny.CANNY_EINVAL
    ok = canny.canny_fault_injection(0, 0, 0, 0)
    assert lib.canny_inject_faults(ctypes.byref(ok)) == canny.CANNY_OK


def test_serve_rejects_bad_configs_and_requests_without_cuda(lib):
    # canny_serve checks its configuration and the whole trace before it
    # allocates anything; an empty trace completes at once
    import numpy as np
    from paper_1710_07745_gb300 import canny
    img = np.zeros((40, 64), np.uint8)
    ptr = img.ctypes.data

    def serve(cfg, reqs):
        arr = (canny.canny_request * max(len(reqs), 1))(*reqs)
        rep = canny.canny_serve_report()
        return lib.canny_serve(ctypes.byref(cfg) if cfg is not None else None, len(reqs), arr, None,
                               ctypes.byref(rep)), rep

    def cfg(**kw):
        c = canny.canny_serve_config(float(1 << 24), 2, 64, 1 << 20, 0, 40, 100, 0, 0)
        for k, v in kw.items():
            setattr(c, k, v)
        return c

    good = canny.canny_request(64, 40, ptr, 64, None, 0, 0.0)
    assert serve(None, [good])[0] == canny.CANNY_EINVAL
    for bad in [dict(streams=0), dict(max_batch_images=0), dict(max_batch_images=65536),
                dict(max_batch_pixels=0), dict(memory_budget_bytes=0.0)]:
        assert serve(cfg(**bad), [good])[0] == canny.CANNY_EINVAL, bad
    for bad in [canny.canny_request(0, 40, ptr, 64, None, 0, 0.0),     # empty image
                canny.canny_request(64, 40, None, 64, None, 0, 0.0),   # no input
                canny.canny_request(64, 40, ptr, 63, None, 0, 0.0),    # pitch below the width
                canny.canny_request(64, 40, ptr, 64, ptr, 32, 0.0)]:   # output pitch below the width
        assert serve(cfg(), [bad])[0] == canny.CANNY_EINVAL
    late_first = [canny.canny_request(64, 40, ptr, 64, None, 0, 1.0), canny.canny_request(64, 40, ptr, 64, None, 0, 0.5)]
    assert serve(cfg(), late_first)[0] == canny.CANNY_EINVAL              # arrivals out of order
    assert serve(cfg(memory_budget_bytes=4096.0), [good])[0] == canny.CANNY_EINVAL   # buffers beyond the budget
    assert serve(cfg(max_batch_pixels=64 * 40 - 1), [good])[0] == canny.CANNY_EINVAL  # beyond one batch
    st, rep = serve(cfg(), [])
    assert st == canny.CANNY_OK and rep.completed == 0
