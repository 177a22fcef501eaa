"""The float variant's acceptance rule, pinned on the CPU against the oracle.

The rule must accept an edge map computed from strengths perturbed by 1e-6
(relative), far below its 1e-3 ambiguity margin, and reject maps with a
deliberate error at a pixel whose decisions are not close to any threshold.
"""
import numpy as np
import pytest

import oracle
from float_check import ambiguous_mask, check_float_edges


def blocky(seed, h, w):
    rng = np.random.default_rng(seed)
    small = rng.integers(0, 256, (h // 6 + 1, w // 6 + 1))
    big = np.kron(small, np.ones((6, 6)))[:h, :w]
    return np.clip(big + rng.normal(0, 6, (h, w)), 0, 255).astype(np.uint8)


def reference(img, lo=0.1, hi=0.3):
    S = oracle.gauss_f32(img, 1.4, 7)
    gx, gy = oracle.sobel_f32(S)
    M = oracle.magnitude_f32(gx, gy)
    e, _, cls = oracle.canny_f32(img, 1.4, 7, lo, hi, want_stages=True)
    return gx, gy, M, cls, e


def edges_from(gx, gy, M, lo=0.1, hi=0.3):
    mmax = np.float32(M.max())
    cls = oracle.nms_classify_f32(gx, gy, M, float(np.float32(lo) * mmax), float(np.float32(hi) * mmax))
    return oracle.hysteresis(cls)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_checker_accepts_a_map_from_slightly_perturbed_strengths(seed):
    img = blocky(seed, 90, 140)
    gx, gy, M, cls, e = reference(img)
    assert np.array_equal(edges_from(gx, gy, M), e)          # the split pipeline is the oracle's
    rng = np.random.default_rng(seed)
    Mp = (M * (1 + 1e-6 * rng.uniform(-1, 1, M.shape))).astype(np.float32)
    check_float_edges(edges_from(gx, gy, Mp), e, gx, gy, M, cls)


def test_checker_rejects_a_flipped_unambiguous_pixel():
    img = blocky(4, 90, 140)
    gx, gy, M, cls, e = reference(img)
    amb = ambiguous_mask(gx, gy, M, cls, 0.1, 0.3)
    strong = (cls == 2) & ~amb
    ys, xs = np.nonzero(strong)
    assert len(ys) > 0
    bad = e.copy()
    bad[ys[0], xs[0]] = 0                                      # a strong pixel dropped
    with pytest.raises(AssertionError):
        check_float_edges(bad, e, gx, gy, M, cls)
    none = (cls == 0) & ~amb
    ys, xs = np.nonzero(none)
    bad = e.copy()
    bad[ys[0], xs[0]] = 255                                    # an edge where nothing can be
    with pytest.raises(AssertionError):
        check_float_edges(bad, e, gx, gy, M, cls)


def test_checker_rejects_a_map_without_edges():
    img = blocky(5, 90, 140)
    gx, gy, M, cls, e = reference(img)
    assert (e == 255).sum() > 50
    with pytest.raises(AssertionError):
        check_float_edges(np.zeros_like(e), e, gx, gy, M, cls)
