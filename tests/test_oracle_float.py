"""Pins for the oracle's float32 variant: taps against scipy's Gaussian window,
smoothing and gradients against scipy's float64 filters within the float32
error bound, plus the invariants of the integer path."""
import numpy as np
import pytest
import scipy.ndimage as ndi
import scipy.signal

import oracle

RNG = np.random.default_rng(99)
EPS = 2.0 ** -24          # float32 unit roundoff


@pytest.mark.parametrize("sigma,ksize", [(1.4, 7), (1.0, 5), (2.0, 9), (0.8, 3)])
def test_taps_match_scipy_window(sigma, ksize):
    t = oracle.gauss_taps_f32(sigma, ksize)
    win = scipy.signal.windows.gaussian(ksize, std=sigma)
    win = win / win.sum()
    assert np.allclose(t, win, rtol=2 * EPS, atol=0)
    assert abs(float(t.astype(np.float64).sum()) - 1.0) <= ksize * EPS
    assert np.array_equal(t, t[::-1])


def _bound_gauss(ksize):
    # each pass: ksize products and ksize-1 sums of values <= 255, each rounded once,
    # plus the taps' own rounding; two passes
    return 2 * (2 * ksize + ksize) * 255 * EPS


@pytest.mark.parametrize("shape", [(1, 1), (1, 9), (9, 1), (12, 17), (64, 40)])
def test_gauss_f32_matches_scipy_float64(shape):
    img = RNG.integers(0, 256, shape, dtype=np.uint8)
    S = oracle.gauss_f32(img, 1.4, 7)
    ref = ndi.gaussian_filter(img.astype(np.float64), sigma=1.4, mode="nearest", truncate=3.0 / 1.4)
    assert np.abs(S - ref).max() <= _bound_gauss(7)


@pytest.mark.parametrize("c", [0, 1, 100, 255])
def test_gauss_f32_constant_image(c):
    S = oracle.gauss_f32(np.full((8, 8), c, np.uint8), 1.4, 7)
    assert np.abs(S - c).max() <= _bound_gauss(7)


@pytest.mark.parametrize("shape", [(1, 1), (3, 5), (30, 22)])
def test_sobel_f32_matches_scipy_on_same_input(shape):
    S = (RNG.random(shape) * 255).astype(np.float32)
    gx, gy = oracle.sobel_f32(S)
    rx = ndi.sobel(S.astype(np.float64), axis=1, mode="nearest")
    ry = ndi.sobel(S.astype(np.float64), axis=0, mode="nearest")
    bound = 6 * 1024 * EPS            # five roundings of values below 1024
    assert np.abs(gx - rx).max() <= bound
    assert np.abs(gy - ry).max() <= bound


def test_magnitude_f32_is_rounded_hypot():
    gx = (RNG.random(5000) * 2040 - 1020).astype(np.float32)
    gy = (RNG.random(5000) * 2040 - 1020).astype(np.float32)
    M = oracle.magnitude_f32(gx, gy)
    ref = np.hypot(gx.astype(np.float64), gy.astype(np.float64))
    assert (np.abs(M - ref) <= 3 * EPS * ref + 1e-30).all()
    assert oracle.max_f32(M) == M.max()


def test_sector_f_rotation_symmetry():
    g = (RNG.random((20000, 2)) * 2000 - 1000).astype(np.float32)
    rot = {0: 1, 1: 0, 2: 3, 3: 2}
    for gx, gy in g:
        s = oracle.sector_f(gx, gy)
        assert oracle.sector_f(-gy, gx) == rot[s]


def test_float_flat_image_has_no_edges():
    e, M, cls = oracle.canny_f32(np.full((16, 16), 90, np.uint8), want_stages=True)
    assert (e == 0).all() and (cls == 0).all()


@pytest.mark.parametrize("c", [6, 11, 20])
def test_float_step_edge_single_column(c):
    """Vertical step: exactly one edge column, next to the step (c-1 or c,
    which tie up to rounding)."""
    w, h = c + 10, 12
    img = np.full((h, w), 40, np.uint8)
    img[:, c:] = 210
    e = oracle.canny_f32(img) == 255
    cols = np.unique(np.nonzero(e)[1])
    assert len(cols) == 1 and cols[0] in (c - 1, c)
    assert e[:, cols[0]].all()


def test_float_thresholds_relative_to_max():
    img = np.zeros((24, 24), np.uint8)
    img[:, 12:] = 200
    img[5:9, 3:6] = 20          # a faint blob: weak only, not connected to the step
    e, M, cls = oracle.canny_f32(img, want_stages=True)
    mmax = float(M.max())
    assert (M[cls == 2] > np.float32(0.3) * np.float32(mmax)).all()
    assert (M[cls == 1] > np.float32(0.1) * np.float32(mmax)).all()
    assert e[:, :9].max() == 0  # the faint blob is not an edge
