"""The float variant's acceptance rule (the oracle is the reference).

An edge map may differ from the fp32 oracle's only at pixels where one of the
oracle's own float decisions lies within 1e-3 (relative) of a threshold, of the
sector boundary or of a suppression neighbour ("ambiguous"), and at pixels
connected to such a pixel through weak or strong pixels.
"""
import numpy as np
import scipy.ndimage as ndi


def ambiguous_mask(gx, gy, M, cls, lo, hi, tol=1e-3):
    """Pixels where one of the oracle's float decisions is within tol (relative)."""
    mmax = np.float32(M.max())
    lo_t, hi_t = np.float32(lo) * mmax, np.float32(hi) * mmax

    def near(a, b):
        return np.abs(a - b) <= tol * np.maximum(np.abs(a), np.abs(b))

    amb = near(M, lo_t) | near(M, hi_t)
    ax, ay = np.abs(gx), np.abs(gy)
    t = np.float32(0.41421356)
    amb |= near(ay, ax * t) | near(ax, ay * t)
    P = np.pad(M, 1)
    h, w = M.shape
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            if dy or dx:
                amb |= near(M, P[1 + dy:1 + dy + h, 1 + dx:1 + dx + w]) & (M > 0)
    return amb


def check_float_edges(got, want_e, gx, gy, M, cls, lo=0.1, hi=0.3):
    diff = got != want_e
    if not diff.any():
        return 0
    amb = ambiguous_mask(gx, gy, M, cls, lo, hi)
    lab, _ = ndi.label((cls > 0) | amb, structure=np.ones((3, 3), int))
    allowed = np.isin(lab, np.unique(lab[amb])) & (lab > 0) | amb
    assert not (diff & ~allowed).any(), int((diff & ~allowed).sum())
    return int(diff.sum())
