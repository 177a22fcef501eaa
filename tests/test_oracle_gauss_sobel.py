"""Pins for the oracle's Steps 1-2 (Gaussian filter, Sobel gradient), integer path.

Each check compares the oracle with something it does not share code with:
Pascal's triangle, numpy/scipy routines, or the step-edge closed form.
"""
import math

import numpy as np
import pytest
import scipy.ndimage as ndi

import oracle

RNG = np.random.default_rng(12345)


def _numpy_gauss5(img):
    """Separable binomial smoothing with numpy: replicate border via np.pad(mode='edge')."""
    b = np.array([math.comb(4, k) for k in range(5)], np.int64)   # Pascal row 4
    h, w = img.shape
    P = np.pad(img.astype(np.int64), 2, mode="edge")
    H = sum(b[k] * P[:, k:k + w] for k in range(5))                # horizontal pass
    V = sum(b[k] * H[k:k + h, :] for k in range(5))                # vertical pass
    return ((V + 128) >> 8).astype(np.uint8)


def test_binomial_kernel_sums_to_256_constant_image_fixed():
    # sum of the 5x5 binomial weights is (2^4)^2 = 256, so (256 c + 128) >> 8 = c
    assert sum(math.comb(4, k) for k in range(5)) ** 2 == 256
    for c in (0, 1, 127, 128, 254, 255):
        img = np.full((9, 13), c, np.uint8)
        assert (oracle.gauss5_u8(img) == c).all()


def test_impulse_response_is_binomial_with_round_half_up():
    for v in (255, 128, 1):
        img = np.zeros((9, 9), np.uint8)
        img[4, 4] = v
        S = oracle.gauss5_u8(img)
        for i in range(-4, 5):
            for j in range(-4, 5):
                k = math.comb(4, i + 2) * math.comb(4, j + 2) if abs(i) <= 2 and abs(j) <= 2 else 0
                want = math.floor(v * k / 256 + 0.5)
                assert S[4 + i, 4 + j] == want, (v, i, j)


@pytest.mark.parametrize("shape", [(1, 1), (1, 7), (7, 1), (2, 3), (3, 2), (5, 5), (17, 33), (64, 48)])
def test_gauss_matches_separable_numpy_with_edge_padding(shape):
    img = RNG.integers(0, 256, shape, dtype=np.uint8)
    assert np.array_equal(oracle.gauss5_u8(img), _numpy_gauss5(img))


def test_gauss_reads_pitched_rows():
    base = RNG.integers(0, 256, (11, 40), dtype=np.uint8)
    view = base[:, :29]                       # pitch 40, width 29
    assert np.array_equal(oracle.gauss5_u8(view), _numpy_gauss5(np.ascontiguousarray(view)))


@pytest.mark.parametrize("shape", [(1, 1), (1, 6), (6, 1), (3, 3), (20, 31)])
def test_sobel_matches_scipy_nearest(shape):
    S = RNG.integers(0, 256, shape, dtype=np.uint8)
    gx, gy = oracle.sobel_u8(S)
    want_x = ndi.sobel(S.astype(np.int32), axis=1, mode="nearest")
    want_y = ndi.sobel(S.astype(np.int32), axis=0, mode="nearest")
    assert np.array_equal(gx, want_x)
    assert np.array_equal(gy, want_y)


def test_sobel_range_extremes():
    S = np.zeros((5, 6), np.uint8)
    S[:, 3:] = 255
    gx, gy = oracle.sobel_u8(S)
    assert gx.max() == 1020 and gx.min() == 0 and (gy == 0).all()
    gx, gy = oracle.sobel_u8(S.T.copy())
    assert gy.max() == 1020 and (gx == 0).all()


def test_mag2_is_squared_norm():
    gx = RNG.integers(-1020, 1021, 1000).astype(np.int16)
    gy = RNG.integers(-1020, 1021, 1000).astype(np.int16)
    m2 = oracle.mag2_i32(gx, gy)
    assert np.array_equal(m2, gx.astype(np.int64) ** 2 + gy.astype(np.int64) ** 2)
    assert oracle.mag2_i32(np.int16([1020]), np.int16([-1020]))[0] == 2080800


@pytest.mark.parametrize("c", [4, 7, 12])
def test_step_edge_closed_form_S_and_Gx(c):
    """I = 32 left of column c, 224 from c on: S and Gx follow from Pascal's row.

    S(c-2+k) = 32 + 192 * (1, 5, 11, 15)[k] / 16 for k = 0..3 (cumulative binomial
    weights), i.e. 44, 92, 164, 212, exactly; Gx = 4 * (S(x+1) - S(x-1)).
    """
    w, h = c + 8, 9
    img = np.full((h, w), 32, np.uint8)
    img[:, c:] = 224
    S = oracle.gauss5_u8(img)
    cum = np.cumsum([math.comb(4, k) for k in range(5)])[:4]       # 1, 5, 11, 15
    want = [32, 32] + [32 + 192 * int(q) // 16 for q in cum] + [224, 224]
    assert list(S[h // 2, c - 4:c + 4]) == want
    assert want[2:6] == [44, 92, 164, 212]
    gx, gy = oracle.sobel_u8(S)
    assert list(gx[h // 2, c - 3:c + 3]) == [48, 240, 480, 480, 240, 48]
    assert (gy == 0).all()
