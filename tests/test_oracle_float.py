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


# ---------------------------------------------------------------- sector pins (Step 2 direction, Step 3)
H, V, D, A = oracle.SECTOR_H, oracle.SECTOR_V, oracle.SECTOR_D, oracle.SECTOR_A


@pytest.mark.parametrize("gx,gy,want", [
    (100.0, 0.0, H), (-100.0, 3.0, H), (0.25, -0.1, H),
    (0.0, 100.0, V), (5.0, -100.0, V), (-0.1, 0.3, V),
    (100.0, 100.0, D), (-7.0, -7.0, D), (0.5, 0.5, D), (-3.5, -2.0, D),
    (100.0, -100.0, A), (-7.0, 7.0, A), (2.5, -2.5, A), (-2.0, 3.5, A),
])
def test_sector_f_examples(gx, gy, want):
    """One example per sector and sign pattern: D is the diagonal where Gx and
    Gy share a sign (the gradient points down-right or up-left, y downward),
    A the other one."""
    assert oracle.sector_f(gx, gy) == want


def test_sector_f_agrees_with_exact_boundary():
    """Away from a 1e-6 relative band around tan(22.5 deg) = sqrt(2) - 1, the
    float sector is the exact one: H iff (ax + ay)^2 < 2 ax^2, V iff
    (ax + ay)^2 < 2 ay^2, else D when Gx Gy > 0, A otherwise. float32 inputs
    in [2^-8, 1020] make every float64 operation here exact."""
    rng = np.random.default_rng(7)
    g = rng.uniform(-1020, 1020, (400000, 2)).astype(np.float32)
    r = np.arange(-40, 41, dtype=np.float32) * np.float32(0.75)
    gg = np.stack(np.meshgrid(r, r), -1).reshape(-1, 2)
    g = np.concatenate([g, gg])
    g = g[(np.abs(g) >= 2.0 ** -8).all(1)]
    gx, gy = g[:, 0].astype(np.float64), g[:, 1].astype(np.float64)
    ax, ay = np.abs(gx), np.abs(gy)
    t = np.sqrt(2.0) - 1.0
    ok = (np.abs(ay - ax * t) > 1e-6 * ax) & (np.abs(ax - ay * t) > 1e-6 * ay)
    assert ok.mean() > 0.999
    gx, gy, ax, ay = gx[ok], gy[ok], ax[ok], ay[ok]
    exact = np.where((ax + ay) ** 2 < 2 * ax ** 2, H,
                     np.where((ax + ay) ** 2 < 2 * ay ** 2, V, np.where(gx * gy > 0, D, A)))
    got = np.array([oracle.sector_f(a, b) for a, b in zip(gx.astype(np.float32), gy.astype(np.float32))])
    assert np.array_equal(got, exact)
    assert {H, V, D, A} <= set(got.tolist())


@pytest.mark.parametrize("anti", [False, True])
def test_float_diagonal_step_gives_the_two_central_diagonals(anti):
    """I = 224 where x + y >= n (or x >= y for the anti-diagonal step), else 32.
    The gradient lies in sector D (A), which compares pixels two diagonals
    apart across the step, so the two diagonals nearest the step both survive;
    the other diagonal sector would compare along the step and keep at most
    one pixel of it."""
    n = 40
    y, x = np.mgrid[0:n, 0:n]
    key = (x - y) if anti else (x + y)
    edge_at = 0 if anti else n
    img = np.where(key >= edge_at, 224, 32).astype(np.uint8)
    e = oracle.canny_f32(img) == 255
    inner, k = e[6:n - 6, 6:n - 6], key[6:n - 6, 6:n - 6]
    assert np.array_equal(inner, (k == edge_at - 1) | (k == edge_at))
    gx, gy = oracle.sobel_f32(oracle.gauss_f32(img))
    px = (20, 20) if anti else (20, 19)
    assert oracle.sector_f(gx[px], gy[px]) == (A if anti else D)
