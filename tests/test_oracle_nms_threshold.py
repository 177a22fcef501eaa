"""Pins for the oracle's Step 3 (direction sectors, non-maximum suppression) and
the double threshold of Step 4, integer path."""
import numpy as np
import pytest

import oracle

H, V, D, A = oracle.SECTOR_H, oracle.SECTOR_V, oracle.SECTOR_D, oracle.SECTOR_A
ROT90 = np.array([V, H, A, D], np.uint8)      # sector of the gradient turned by 90 degrees


def test_tan_q15_is_nearest_integer_to_exact_value():
    # T = round((sqrt(2)-1) 2^15) <=> T - 1/2 < (sqrt(2)-1) 2^15 < T + 1/2
    # <=> (2T + 1 + 65536)^2 > 2 * 65536^2 > (2T - 1 + 65536)^2, all in integers.
    T = oracle.sector_tan_q15()
    assert (2 * T - 1 + 65536) ** 2 < 2 * 65536 ** 2 < (2 * T + 1 + 65536) ** 2
    assert T == 13573


@pytest.fixture(scope="module")
def full_grid():
    r = np.arange(-1020, 1021, dtype=np.int32)
    gx, gy = np.meshgrid(r, r, indexing="xy")
    return gx.ravel(), gy.ravel()


def test_sector_rotation_symmetry_exhaustive(full_grid):
    gx, gy = full_grid
    keep = ~((gx == 0) & (gy == 0))
    gx, gy = gx[keep], gy[keep]
    s = oracle.sector_map_i(gx, gy)
    s_rot = oracle.sector_map_i(-gy, gx)
    assert np.array_equal(s_rot, ROT90[s])
    # mirror symmetry too: (gx, gy) -> (-gx, gy) keeps H/V and swaps D/A
    s_mir = oracle.sector_map_i(-gx, gy)
    assert np.array_equal(s_mir, np.array([H, V, A, D], np.uint8)[s])


def test_sector_agrees_with_exact_irrational_boundary(full_grid):
    gx, gy = full_grid
    ax, ay = np.abs(gx).astype(np.int64), np.abs(gy).astype(np.int64)
    s = oracle.sector_map_i(gx, gy)
    # exact: H <=> ay < ax (sqrt2 - 1) <=> (ax + ay)^2 < 2 ax^2 (ax > 0)
    exact_h = (ax > 0) & ((ax + ay) ** 2 < 2 * ax ** 2)
    exact_v = (ay > 0) & ((ax + ay) ** 2 < 2 * ay ** 2)
    t = np.sqrt(2.0) - 1.0
    near_h = np.abs(ay - ax * t) < ax * 2.0 ** -15
    near_v = np.abs(ax - ay * t) < ay * 2.0 ** -15
    ok = ~(near_h | near_v)
    assert ok.mean() > 0.999
    assert np.array_equal((s == H)[ok], exact_h[ok])
    assert np.array_equal((s == V)[ok], exact_v[ok])
    diag = ok & ~exact_h & ~exact_v & ((gx != 0) | (gy != 0))
    assert np.array_equal((s == D)[diag], (gx * gy > 0)[diag])


def test_sector_examples():
    assert oracle.sector_i(100, 0) == H and oracle.sector_i(-100, 3) == H
    assert oracle.sector_i(0, 100) == V and oracle.sector_i(5, -100) == V
    assert oracle.sector_i(100, 100) == D and oracle.sector_i(-7, -7) == D
    assert oracle.sector_i(100, -100) == A and oracle.sector_i(-7, 7) == A


def _cls(gx, gy, m2, low=40, high=100):
    return oracle.nms_classify_u8(np.int16(gx), np.int16(gy), np.int32(m2), low, high)


@pytest.mark.parametrize("gxy,want", [((40, 0), oracle.NONE), ((40, 1), oracle.WEAK),
                                      ((100, 0), oracle.WEAK), ((100, 1), oracle.STRONG),
                                      ((0, 0), oracle.NONE)])
def test_thresholds_are_strict(gxy, want):
    gx = np.zeros((3, 3), np.int16)
    gy = np.zeros((3, 3), np.int16)
    gx[1, 1], gy[1, 1] = gxy
    m2 = gx.astype(np.int32) ** 2 + gy.astype(np.int32) ** 2
    assert _cls(gx, gy, m2)[1, 1] == want


# (sector, gx, gy, negative-side offset (dy, dx), positive-side offset)
CASES = [(H, 300, 0, (0, -1), (0, 1)), (V, 0, 300, (-1, 0), (1, 0)),
         (D, 300, 300, (-1, -1), (1, 1)), (A, 300, -300, (1, -1), (-1, 1))]


@pytest.mark.parametrize("sec,gx0,gy0,neg,pos", CASES)
def test_nms_neighbours_and_tie_break(sec, gx0, gy0, neg, pos):
    assert oracle.sector_i(gx0, gy0) == sec
    gx = np.zeros((3, 3), np.int16)
    gy = np.zeros((3, 3), np.int16)
    gx[1, 1], gy[1, 1] = gx0, gy0
    m = gx0 * gx0 + gy0 * gy0
    for other, val in [((1 + neg[0], 1 + neg[1]), m), ((1 + pos[0], 1 + pos[1]), m)]:
        m2 = np.zeros((3, 3), np.int32)
        m2[1, 1] = m
        m2[other] = val
        c = _cls(gx, gy, m2)[1, 1]
        on_neg = other == (1 + neg[0], 1 + neg[1])
        # equal to the negative-side neighbour: suppressed; equal to the positive one: kept
        assert c == (oracle.NONE if on_neg else oracle.STRONG)
    # neighbours off the sector axis never suppress
    m2 = np.full((3, 3), m + 5, np.int32)
    m2[1, 1] = m
    m2[1 + neg[0], 1 + neg[1]] = 0
    m2[1 + pos[0], 1 + pos[1]] = 0
    assert _cls(gx, gy, m2)[1, 1] == oracle.STRONG


def test_plateau_keeps_first_pixel_along_positive_direction():
    gx = np.full((1, 5), 100, np.int16)
    gy = np.zeros((1, 5), np.int16)
    m2 = np.array([[0, 5000, 5000, 5000, 0]], np.int32)
    assert list(_cls(gx, gy, m2)[0]) == [0, 1, 0, 0, 0]


def test_outside_neighbours_count_as_zero():
    gx = np.full((1, 1), 100, np.int16)
    gy = np.zeros((1, 1), np.int16)
    assert _cls(gx, gy, np.int32([[10001]]))[0, 0] == oracle.STRONG


@pytest.mark.parametrize("shape", [(1, 1), (1, 9), (9, 1), (4, 4), (33, 17)])
@pytest.mark.parametrize("c", [0, 77, 255])
def test_constant_image_has_no_edges(shape, c):
    img = np.full(shape, c, np.uint8)
    assert (oracle.classify_u8(img) == 0).all()
    assert (oracle.canny_u8(img) == 0).all()


@pytest.mark.parametrize("w,h,c", [(8, 8, 4), (16, 5, 9), (40, 13, 36), (23, 2, 10)])
@pytest.mark.parametrize("lo_hi", [(32, 224), (224, 32)])
def test_step_edge_gives_single_column(w, h, c, lo_hi):
    """Vertical step at column c (4 <= c <= w-4): the edge is column c-1 only, in
    every row; the transposed image gives row c-1 only."""
    img = np.full((h, w), lo_hi[0], np.uint8)
    img[:, c:] = lo_hi[1]
    e = oracle.canny_u8(img)
    want = np.zeros((h, w), np.uint8)
    want[:, c - 1] = 255
    assert np.array_equal(e, want)
    assert np.array_equal(oracle.canny_u8(img.T.copy()), want.T)


def test_diagonal_step_gives_staircase_on_the_two_central_diagonals():
    """I = 224 where x + y >= n. The gradient lies in sector D, which compares
    pixels two diagonals apart, so the two diagonals nearest the step
    (x + y = n - 1 and n, equal strength by symmetry) both survive: a 4-connected
    staircase, two pixels per row. Sector A (the wrong sign) would compare
    along the edge and suppress everything."""
    n = 40
    y, x = np.mgrid[0:n, 0:n]
    img = np.where(x + y >= n, 224, 32).astype(np.uint8)
    e = oracle.canny_u8(img) == 255
    inner = e[6:n - 6, 6:n - 6]
    sums = x[6:n - 6, 6:n - 6] + y[6:n - 6, 6:n - 6]
    assert np.array_equal(inner, (sums == n - 1) | (sums == n))
    gx, gy = oracle.sobel_u8(oracle.gauss5_u8(img))
    assert oracle.sector_i(int(gx[20, 19]), int(gy[20, 19])) == D
