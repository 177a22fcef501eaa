"""Pins for the oracle's hysteresis (Step 4): exhaustive small maps against an
independent brute force, random larger maps against scipy's connected-component
labelling."""
import os
import subprocess

import numpy as np
import pytest
import scipy.ndimage as ndi

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))


def _scipy_hysteresis(cls):
    lab, n = ndi.label(cls > 0, structure=np.ones((3, 3), int))
    strong_labels = np.unique(lab[cls == 2])
    strong_labels = strong_labels[strong_labels > 0]
    return np.where(np.isin(lab, strong_labels), 255, 0).astype(np.uint8)


@pytest.fixture(scope="module")
def exhaustive_bin(tmp_path_factory):
    lib = oracle.build()
    exe = str(tmp_path_factory.mktemp("native") / "hyst_exhaustive")
    subprocess.run(["gcc", "-O2", os.path.join(HERE, "native", "hyst_exhaustive.c"), lib,
                    "-o", exe, f"-Wl,-rpath,{os.path.dirname(lib)}"], check=True)
    return exe


@pytest.mark.parametrize("w,h", [(1, 1), (3, 1), (1, 5), (3, 3), (4, 3), (3, 4), (2, 7), (7, 2)])
def test_hysteresis_exhaustive(exhaustive_bin, w, h):
    r = subprocess.run([exhaustive_bin, str(w), str(h)], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "0 mismatches" in r.stdout
    assert f"checked {3 ** (w * h)} maps" in r.stdout


@pytest.mark.slow
def test_hysteresis_exhaustive_4x4(exhaustive_bin):
    r = subprocess.run([exhaustive_bin, "4", "4"], capture_output=True, text=True)
    assert r.returncode == 0 and "0 mismatches" in r.stdout, r.stdout


@pytest.mark.parametrize("seed", range(6))
def test_hysteresis_random_vs_scipy_label(seed):
    rng = np.random.default_rng(seed)
    h, w = rng.integers(1, 97, 2)
    p = rng.dirichlet([4, 3, 1])
    cls = rng.choice(3, size=(h, w), p=p).astype(np.uint8)
    assert np.array_equal(oracle.hysteresis(cls), _scipy_hysteresis(cls))


def test_hysteresis_long_spiral_of_weak_pixels():
    """A 1-pixel-wide weak spiral with a single strong pixel at its inner end."""
    n = 41
    cls = np.zeros((n, n), np.uint8)
    x0, y0, x1, y1 = 0, 0, n - 1, n - 1
    path = []
    while x0 <= x1 and y0 <= y1:
        path += [(y0, x) for x in range(x0, x1 + 1)]
        path += [(y, x1) for y in range(y0 + 1, y1 + 1)]
        if y1 > y0:
            path += [(y1, x) for x in range(x1 - 1, x0 - 1, -1)]
        if x1 > x0:
            path += [(y, x0) for y in range(y1 - 1, y0 + 1, -1)]
        x0, y0, x1, y1 = x0 + 2, y0 + 2, x1 - 2, y1 - 2
        if path:
            path.append((y0 - 1, x0 - 1)) if (x0 - 1 <= x1 + 1) else None
    for (y, x) in path:
        if 0 <= y < n and 0 <= x < n:
            cls[y, x] = 1
    yy, xx = path[-1]
    cls[min(max(yy, 0), n - 1), min(max(xx, 0), n - 1)] = 2
    assert np.array_equal(oracle.hysteresis(cls), _scipy_hysteresis(cls))


def test_hysteresis_pitched_output_leaves_padding():
    rng = np.random.default_rng(7)
    cls = rng.integers(0, 3, (9, 13)).astype(np.uint8)
    out = np.full((9, 20), 77, np.uint8)
    oracle.hysteresis(cls, out)
    assert (out[:, 13:] == 77).all()
    assert np.array_equal(out[:, :13], _scipy_hysteresis(cls))
