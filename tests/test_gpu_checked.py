"""The checked build (-DCANNY_CHECKS, in place of a sanitizer): every bounds
check in the device code holds on tiny, ragged, adversarial and batched inputs
(no check bit in the run's error word) and the edge maps stay equal to the
oracle's."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1710_07745_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1710_07745_gb300 import canny  # noqa: E402


@pytest.fixture(scope="module")
def lib():
    return canny.load_checked()


def create(lib, w, h, path=canny.CANNY_PATH_INT, low=40.0, high=100.0, max_passes=0):
    p = canny.canny_params()
    lib.canny_params_default(ctypes.byref(p))
    p.path, p.low, p.high, p.max_passes = path, low, high, max_passes
    ctx = ctypes.c_void_p()
    assert lib.canny_create(w, h, ctypes.byref(p), ctypes.byref(ctx)) == canny.CANNY_OK
    return ctx


def status(lib, ctx):
    st = canny.canny_stats()
    assert lib.canny_get_stats(ctx, ctypes.byref(st)) == canny.CANNY_OK
    return st.status


def serpentine(n, gap=32):
    """One weak path through every 32-row band of an n x n map, strong only at its start."""
    cls = np.zeros((n, n), np.uint8)
    rows = list(range(gap // 2, n, gap))
    for j, r in enumerate(rows):
        cls[r, :] = 1
        if j + 1 < len(rows):
            c = n - 1 if j % 2 == 0 else 0
            cls[r:rows[j + 1] + 1, c] = 1
    cls[rows[0], 0] = 2
    return cls


@pytest.mark.parametrize("h,w", [(1, 1), (1, 300), (300, 1), (3, 3), (17, 5), (31, 33), (64, 224), (65, 225),
                                 (200, 301), (129, 450), (300, 700), (520, 1000)])   # the last two hold interior units
def test_checked_build_integer_and_float_sizes(lib, h, w):
    img = synth.image(h * 7 + w, w, h, 4, 4, 10)
    for path in (canny.CANNY_PATH_INT, canny.CANNY_PATH_F32):
        ctx = create(lib, w, h, path, *((40.0, 100.0) if path == canny.CANNY_PATH_INT else (0.1, 0.3)))
        try:
            d_in = torch.from_numpy(img).cuda()
            out = torch.full((h, w), 7, dtype=torch.uint8, device="cuda")
            im = canny.image_of(d_in, out)
            assert lib.canny_run_pitched(ctx, ctypes.byref(im), None) == canny.CANNY_OK
            torch.cuda.synchronize()
            assert status(lib, ctx) == canny.CANNY_OK
            want = oracle.canny_u8(img) if path == canny.CANNY_PATH_INT else oracle.canny_f32(img, 1.4, 7, 0.1, 0.3)
            assert np.array_equal(out.cpu().numpy(), want)
        finally:
            lib.canny_destroy(ctx)


def test_checked_build_long_chains_and_pass_cap(lib):
    cls = serpentine(2048)
    h, w = cls.shape
    for cap, want_status in ((0, canny.CANNY_OK), (1, canny.CANNY_ENOCONVERGE)):
        ctx = create(lib, w, h, max_passes=cap)
        try:
            d = torch.from_numpy(cls).cuda()
            out = torch.zeros_like(d)
            im = canny.image_of(d, out)
            lib.canny_hysteresis(ctx, ctypes.byref(im), None)
            torch.cuda.synchronize()
            assert status(lib, ctx) == want_status
            if cap == 0:
                assert np.array_equal(out.cpu().numpy(), oracle.hysteresis(cls))
        finally:
            lib.canny_destroy(ctx)


def test_checked_build_batch(lib):
    rng = np.random.default_rng(21)
    imgs = [synth.image(2000 + i, int(w), int(h), 4, 4, 8) for i, (h, w) in enumerate(rng.integers(1, 400, (30, 2)))]
    ins = [torch.from_numpy(im).cuda() for im in imgs]
    outs = [torch.full(im.shape, 7, dtype=torch.uint8, device="cuda") for im in imgs]
    ctx = create(lib, sum(im.size for im in imgs), 1)
    try:
        arr = (canny.canny_image * len(imgs))(*[canny.image_of(a, b) for a, b in zip(ins, outs)])
        assert lib.canny_run_batch(ctx, len(imgs), arr, None) == canny.CANNY_OK
        torch.cuda.synchronize()
        assert status(lib, ctx) == canny.CANNY_OK
        for im, o in zip(imgs, outs):
            assert np.array_equal(o.cpu().numpy(), oracle.canny_u8(im))
    finally:
        lib.canny_destroy(ctx)
