"""The seeded input generator: determinism and the stated value distributions."""
import numpy as np

from paper_1710_07745_gb300 import synth


def test_same_seed_same_bytes_any_thread_count():
    a = synth.image(5, 300, 211, 10, 10, 8, threads=1)
    b = synth.image(5, 300, 211, 10, 10, 8, threads=7)
    c = synth.image(5, 300, 211, 10, 10, 8, threads=64)
    assert np.array_equal(a, b) and np.array_equal(a, c)
    assert not np.array_equal(a, synth.image(6, 300, 211, 10, 10, 8))


def test_pitched_output_pads_with_zero():
    a = synth.image(9, 50, 20, 3, 3, 8)
    p = synth.image(9, 50, 20, 3, 3, 8, pitch=64)
    assert np.array_equal(p[:, :50], a) and (p[:, 50:] == 0).all()


def test_noise_is_zero_mean_with_stated_sigma():
    clean = synth.image(11, 512, 512, 0, 0, 0).astype(np.float64)
    noisy = synth.image(11, 512, 512, 0, 0, 8).astype(np.float64)
    inside = (clean > 40) & (clean < 215)          # away from clamping
    d = (noisy - clean)[inside]
    assert abs(d.mean()) < 0.05
    assert abs(d.std() - 8.0) < 0.2


def test_background_gradient_spans_full_range():
    clean = synth.image(3, 200, 100, 0, 0, 0)
    assert clean.min() == 0 and clean.max() == 255


def test_objects_are_flat_regions():
    img = synth.image(4, 256, 256, 20, 20, 0)
    vals, counts = np.unique(img, return_counts=True)
    assert counts.max() > 256 * 256 // 50          # large uniform regions exist


def test_log_uniform_sizes_in_range_and_spread():
    ws, hs = synth.log_uniform_sizes(4000, 4096, 64, 2048)
    assert ws.min() >= 64 and ws.max() <= 2048 and hs.min() >= 64 and hs.max() <= 2048
    lw = np.log2(ws)
    assert abs(lw.mean() - 8.5) < 0.1            # log2 uniform on [6, 11]
    assert not np.array_equal(ws, hs)


def test_poisson_arrivals_mean_gap():
    t = synth.poisson_arrivals(1, 20000, 50.0)
    gaps = np.diff(t)
    assert (gaps > 0).all() and abs(gaps.mean() - 0.02) < 0.001


def test_object_count_scaling():
    assert synth.objects_for_area(4096, 4096) == 200
    assert synth.objects_for_area(16384, 16384) == 3200
    assert synth.objects_for_area(7680, 4320) == 396
    assert synth.objects_for_area(64, 64) == 2
