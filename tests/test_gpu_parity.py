"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Integer path: bit-exact edge maps and class maps on every case. Float path:
strength within 1e-5 relative, edge maps equal except where the oracle's own
decision is within 1e-3 of a threshold or neighbour (and what is connected to
such a pixel).
"""
import ctypes

import numpy as np
import pytest

import oracle
from float_check import check_float_edges
from paper_1710_07745_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1710_07745_gb300 import canny  # noqa: E402


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def run_int(img, low=40, high=100, ctx=None, stage="edges"):
    h, w = img.shape
    c = ctx or canny.Canny(max(w, 1), max(h, 1), low=low, high=high)
    d_in = dev(img)
    d_out = torch.full((h, w), 7, dtype=torch.uint8, device="cuda")
    if stage == "edges":
        c.run_pitched(d_in, d_out)
    else:
        c.classify(d_in, d_out)
    torch.cuda.synchronize()
    st = c.stats()
    out = d_out.cpu().numpy()
    if ctx is None:
        c.close()
    return out, st


def noise_image(seed, h, w):
    return np.random.default_rng(seed).integers(0, 256, (h, w), dtype=np.uint8)


def blocky_image(seed, h, w):
    """Smooth-ish random image: random values upsampled, plus noise (many weak/strong mixes)."""
    rng = np.random.default_rng(seed)
    small = rng.integers(0, 256, (max(1, h // 6 + 1), max(1, w // 6 + 1)))
    big = np.kron(small, np.ones((6, 6)))[:h, :w]
    return np.clip(big + rng.normal(0, 6, (h, w)), 0, 255).astype(np.uint8)


# ------------------------------------------------------------------ integer path
def test_small_workload_bit_exact():
    img = synth.small()
    out, st = run_int(img)
    assert st["status"] == canny.CANNY_OK
    assert np.array_equal(out, oracle.canny_u8(img))
    cls, _ = run_int(img, stage="classify")
    assert np.array_equal(cls, oracle.classify_u8(img))


# Sizes at the edge of the interior test: a unit (strip X0 = 480 k, band
# Y0 = 64 j) runs the stencil without border checks only when X0 >= 16,
# X0 + 496 <= w, Y0 >= 4 and Y0 + 68 <= h. Each size puts one strip or band
# exactly on either side of that line; all must stay bit-exact.
@pytest.mark.parametrize("h,w", [(132, 976), (133, 976), (132, 975), (133, 977), (197, 1456), (196, 1457),
                                 (261, 1936), (260, 1935), (69, 496), (68, 495), (132, 472), (133, 473)])
def test_interior_unit_boundaries(h, w):
    img = blocky_image(h * 3 + w, h, w)
    out, st = run_int(img)
    assert st["status"] == canny.CANNY_OK
    assert np.array_equal(out, oracle.canny_u8(img))
    cls, _ = run_int(img, stage="classify")
    assert np.array_equal(cls, oracle.classify_u8(img))


def test_medium_workload_bit_exact():
    img = synth.medium()
    out, st = run_int(img)
    assert st["status"] == canny.CANNY_OK
    want = oracle.canny_u8(img)
    assert np.array_equal(out, want), int((out != want).sum())


SIZES = [(1, 1), (1, 5), (5, 1), (2, 2), (3, 5), (5, 17), (17, 5), (7, 7), (31, 33), (32, 32),
         (33, 31), (64, 64), (37, 100), (257, 513), (999, 1000), (2, 700), (700, 3)]


@pytest.mark.parametrize("h,w", SIZES)
@pytest.mark.parametrize("kind", ["synth", "noise", "blocky"])
def test_sizes_bit_exact(h, w, kind):
    seed = h * 1009 + w
    if kind == "synth":
        img = synth.image(seed, w, h, 6, 6, 10)
    elif kind == "noise":
        img = noise_image(seed, h, w)
    else:
        img = blocky_image(seed, h, w)
    out, st = run_int(img)
    assert st["status"] == canny.CANNY_OK
    assert np.array_equal(out, oracle.canny_u8(img))
    cls, _ = run_int(img, stage="classify")
    assert np.array_equal(cls, oracle.classify_u8(img))


@pytest.mark.parametrize("low,high", [(0, 0), (40, 40), (10, 200), (100, 1000), (0, 1442), (1, 2)])
def test_thresholds_bit_exact(low, high):
    img = blocky_image(5, 300, 420)
    out, _ = run_int(img, low, high)
    assert np.array_equal(out, oracle.canny_u8(img, low, high))


def test_pitched_buffers_leave_padding_untouched():
    h, w, pin, pout = 150, 203, 256, 240
    img = synth.image(21, w, h, 5, 5, 8)
    base_in = np.full((h, pin), 99, np.uint8)
    base_in[:, :w] = img
    d_in = dev(base_in)
    d_out = torch.full((h, pout), 77, dtype=torch.uint8, device="cuda")
    with canny.Canny(w, h) as c:
        c.run_pitched(d_in[:, :w], d_out[:, :w])
        torch.cuda.synchronize()
    out = d_out.cpu().numpy()
    assert (out[:, w:] == 77).all()
    assert np.array_equal(out[:, :w], oracle.canny_u8(img))


def test_unaligned_input_base_and_pitch_are_staged():
    # inputs the TMA path cannot read (odd base address, odd pitch) are copied into
    # pitched staging first; results equal the oracle's, single and batched
    img = synth.image(77, 301, 203, 6, 6, 8)
    big = np.zeros((203, 320), np.uint8)
    big[:, 3:304] = img
    d_big = dev(big)
    d_view = d_big[:, 3:304]                       # base offset by 3 bytes, pitch 320
    out = torch.full((203, 301), 7, dtype=torch.uint8, device="cuda")
    with canny.Canny(301, 203) as c:
        c.run_pitched(d_view, out)
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy(), oracle.canny_u8(img))
    with canny.Canny(301, 203, path=canny.CANNY_PATH_F32, low=0.1, high=0.3) as c:
        c.run_pitched(d_view, out)
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy(), oracle.canny_f32(img, 1.4, 7, 0.1, 0.3))
    outs = [torch.full((203, 301), 7, dtype=torch.uint8, device="cuda") for _ in range(3)]
    ins = [d_view, dev(img), d_big[:, 1:302]]
    wants = [oracle.canny_u8(img), oracle.canny_u8(img), oracle.canny_u8(big[:, 1:302])]
    with canny.Canny(3 * 301 * 203, 1) as c:
        c.run_batch(list(zip(ins, outs)))
        torch.cuda.synchronize()
    for o, want in zip(outs, wants):
        assert np.array_equal(o.cpu().numpy(), want)


@pytest.mark.parametrize("direct", [0, 1])
def test_repitch_every_base_offset_and_narrow_width(direct):
    # repitching reads 16-byte granules funnel-shifted by the base offset, falling
    # back to byte loads where a granule would leave the image's bytes: every
    # offset 0..15, widths below, at and across one granule, pitches w..w+19
    rng = np.random.default_rng(77)
    cases = []
    for k in range(48):
        w = int([1, 3, 15, 16, 17, 31, 33, 47, 230, 449][k % 10])
        h = int(rng.integers(1, 40))
        off = k % 16
        pitch = w + int(rng.integers(0, 20))
        buf = np.zeros((h + 1) * pitch + 32, np.uint8)
        img = synth.image(3000 + k, w, h, 4, 4, 6)
        cases.append((img, buf, off, pitch))
    ins, outs, wants = [], [], []
    for img, buf, off, pitch in cases:
        h, w = img.shape
        d = dev(buf)
        view = d[off:off + (h - 1) * pitch + w].as_strided((h, w), (pitch, 1))
        view.copy_(dev(img))
        ins.append(view)
        outs.append(torch.full((h, w), 7, dtype=torch.uint8, device="cuda"))
        wants.append(oracle.canny_u8(img))
    total = sum(im.size for im, _, _, _ in cases)
    with canny.Canny(total, 1) as c:
        c.set_tuning(64, 12, direct)
        c.run_batch(list(zip(ins, outs)))
        torch.cuda.synchronize()
        for o, want in zip(outs, wants):
            assert np.array_equal(o.cpu().numpy(), want)
    with canny.Canny(449, 40) as c:
        c.set_tuning(64, 12, direct)
        for i, o, want in zip(ins, outs, wants):
            o.fill_(7)
            c.run_pitched(i, o)
            torch.cuda.synchronize()
            assert np.array_equal(o.cpu().numpy(), want)


def test_context_reuse_smaller_images_and_determinism():
    with canny.Canny(600, 400) as c:
        for (h, w, seed) in [(400, 600, 1), (17, 33, 2), (400, 600, 3), (1, 1, 4), (399, 599, 5)]:
            img = synth.image(seed, w, h, 8, 8, 8)
            outs = [run_int(img, ctx=c)[0] for _ in range(3)]
            assert all(np.array_equal(o, outs[0]) for o in outs)
            assert np.array_equal(outs[0], oracle.canny_u8(img))


def test_empty_image_is_a_no_op():
    with canny.Canny(16, 16) as c:
        img = canny.canny_image(0, 0, 0, 5, 0, 0)
        canny.canny_run_pitched(c.ctx, img, 0)
        canny.canny_run_batch(c.ctx, [], 0)


def test_rejects_oversize_and_overlap():
    with canny.Canny(64, 64) as c:
        a = torch.zeros((70, 70), dtype=torch.uint8, device="cuda")
        b = torch.zeros((70, 70), dtype=torch.uint8, device="cuda")
        with pytest.raises(canny.CannyError) as e:
            c.run_pitched(a, b)
        assert e.value.status == canny.CANNY_EINVAL
        with pytest.raises(canny.CannyError):
            c.run_pitched(a[:10, :10], a[5:15, :10])      # overlapping output


# ------------------------------------------------------------------ hysteresis alone
def spiral_map(n, gap=1):
    """1-pixel weak spiral (rings `gap` apart) with one strong pixel at its inner end."""
    cls = np.zeros((n, n), np.uint8)
    y0, x0, y1, x1 = 0, 0, n - 1, n - 1
    path = []
    step = gap + 1
    while y0 <= y1 and x0 <= x1:
        path += [(y0, x) for x in range(x0, x1 + 1)]
        path += [(y, x1) for y in range(y0 + 1, y1 + 1)]
        if y1 - y0 >= step:
            path += [(y1, x) for x in range(x1 - 1, x0 - 1, -1)]
        if x1 - x0 >= step:
            path += [(y, x0) for y in range(y1 - 1, y0 + step - 1, -1)]
        path += [(y0 + step, x) for x in range(x0, min(x0 + step, x1 + 1))]
        y0, x0, y1, x1 = y0 + step, x0 + step, y1 - step, x1 - step
    for (y, x) in path:
        if 0 <= y < n and 0 <= x < n:
            cls[y, x] = 1
    y, x = path[-1]
    cls[min(y, n - 1), min(x, n - 1)] = 2
    return cls


def run_hyst(cls, max_passes=0, ctx=None):
    h, w = cls.shape
    c = ctx or canny.Canny(w, h, max_passes=max_passes)
    d_in = dev(cls)
    d_out = torch.empty_like(d_in)
    c.hysteresis(d_in, d_out)
    torch.cuda.synchronize()
    out, st = d_out.cpu().numpy(), c.stats()
    if ctx is None:
        c.close()
    return out, st


@pytest.mark.parametrize("seed", range(8))
def test_hysteresis_random_maps(seed):
    rng = np.random.default_rng(seed)
    h, w = (int(v) for v in rng.integers(1, 300, 2))
    p = rng.dirichlet([3, 3, 0.3])
    cls = rng.choice(3, size=(h, w), p=p).astype(np.uint8)
    out, st = run_hyst(cls)
    assert st["status"] == canny.CANNY_OK
    assert np.array_equal(out, oracle.hysteresis(cls))


def serpentine_map(n, gap=32):
    """One weak path through every tile: horizontal runs every `gap` rows joined at
    alternate ends, strong only at its start."""
    cls = np.zeros((n, n), np.uint8)
    rows = list(range(gap // 2, n, gap))
    for j, r in enumerate(rows):
        cls[r, :] = 1
        if j + 1 < len(rows):
            c = n - 1 if j % 2 == 0 else 0
            cls[r:rows[j + 1] + 1, c] = 1
    cls[rows[0], 0] = 2
    return cls


def test_hysteresis_spiral_is_chased_in_few_passes():
    cls = spiral_map(300)
    out, st = run_hyst(cls)
    assert st["status"] == canny.CANNY_OK
    assert np.array_equal(out, oracle.hysteresis(cls))
    assert (out == 255).sum() == (cls > 0).sum()          # the whole spiral is reached
    # the pass that finds the first seed follows the chain tile to tile
    assert st["hyst_passes"] <= 3


def test_hysteresis_chain_longer_than_the_chase_budget():
    cls = serpentine_map(2048)                            # a chain through 4096+ tiles
    out, st = run_hyst(cls)
    assert st["status"] == canny.CANNY_OK
    assert np.array_equal(out, oracle.hysteresis(cls))
    assert (out == 255).sum() == (cls > 0).sum()
    assert st["hyst_passes"] > 1                          # the budget per entry spills to later passes


@pytest.mark.parametrize("tiles", [256, 1024, 4096, 16384])
def test_hysteresis_long_serpentines_resolve_in_two_passes(tiles):
    """One weak chain through every tile (strong only at its start): the first
    pass chases it for a budget of tiles, the union-find stage resolves the rest
    at once, so the pass count stays at two whatever the length."""
    n = 32 * int(round(tiles ** 0.5))
    cls = serpentine_map(n)
    out, st = run_hyst(cls)
    assert st["status"] == canny.CANNY_OK
    assert np.array_equal(out, oracle.hysteresis(cls))
    assert (out == 255).sum() == (cls > 0).sum()
    assert st["hyst_passes"] <= 2


def test_hysteresis_long_worklists_keep_to_passes():
    """More tiles with pending border pixels than the union-find stage takes
    (36864, one weak pixel at each tile's corner) and a chain through 100 tiles,
    longer than the chase budget: the passes alone finish it."""
    n = 6144
    cls = np.zeros((n, n), np.uint8)
    cls[::32, ::32] = 1
    cls[:320, :320] = serpentine_map(320)
    out, st = run_hyst(cls)
    assert st["status"] == canny.CANNY_OK
    assert np.array_equal(out, oracle.hysteresis(cls))
    assert st["hyst_passes"] > 2


def test_hysteresis_union_find_keeps_unreached_components_weak():
    """Long chains, one seeded at its start and one never seeded, plus pending
    blobs that touch tile borders without any edge: only the seeded chain's
    pixels become edges."""
    n = 1024
    cls = serpentine_map(n)
    cls[n // 2 + 7, :] = 0                              # cut the chain once: its far part stays weak
    rng = np.random.default_rng(5)
    for _ in range(40):
        y, x = (int(v) for v in rng.integers(0, n - 8, 2))
        cls[y:y + 6, x:x + 6] = np.maximum(cls[y:y + 6, x:x + 6], 1)
    out, st = run_hyst(cls)
    assert st["status"] == canny.CANNY_OK
    assert np.array_equal(out, oracle.hysteresis(cls))


def test_hysteresis_pass_cap_reports_no_convergence():
    cls = serpentine_map(2048)
    out, st = run_hyst(cls, max_passes=1)
    assert st["status"] == canny.CANNY_ENOCONVERGE
    assert st["hyst_passes"] == 1


def test_weak_chains_crossing_many_tiles():
    # long straight and diagonal weak lines, strong only at one end
    n = 700
    cls = np.zeros((n, n), np.uint8)
    cls[100, :] = 1
    cls[100, 0] = 2
    cls[:, 333] = 1
    np.fill_diagonal(cls, 1)
    cls[n - 1, n - 1] = 2
    cls[::37, 600] = 1
    out, _ = run_hyst(cls)
    assert np.array_equal(out, oracle.hysteresis(cls))


# ------------------------------------------------------------------ batch and host paths
def test_batch_equals_oracle_and_single_runs():
    sizes = [(64, 64), (1, 1), (0, 10), (33, 700), (257, 129), (512, 512), (5, 3), (100, 31)]
    imgs = [synth.image(100 + i, w, h, 5, 5, 8) if w * h else np.zeros((h, w), np.uint8)
            for i, (h, w) in enumerate(sizes)]
    total = sum(w * h for h, w in sizes)
    ins = [dev(im) for im in imgs]
    outs = [torch.full(im.shape, 3, dtype=torch.uint8, device="cuda") for im in imgs]
    with canny.Canny(total, 1) as c:
        c.run_batch(list(zip(ins, outs)))
        torch.cuda.synchronize()
        st = c.stats()
    assert st["status"] == canny.CANNY_OK and st["images"] == len(sizes)
    for im, o in zip(imgs, outs):
        if im.size:
            assert np.array_equal(o.cpu().numpy(), oracle.canny_u8(im))


def test_run_host_matches_device_path():
    img = synth.image(8, 640, 480, 10, 10, 8)
    out = np.zeros_like(img)
    with canny.Canny(640, 480) as c:
        canny.canny_run_host(c.ctx, img.ctypes.data, 640, out.ctypes.data, 640, 640, 480, 0)
    assert np.array_equal(out, oracle.canny_u8(img))


def pinned(a):
    t = torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    return t


def frames_run(ctx, frames, w, h, pin=True):
    outs = [np.full((h, w), 7, np.uint8) for _ in frames]
    if pin:
        ins_t = [pinned(f) for f in frames]
        outs_t = [pinned(o) for o in outs]
        canny.canny_run_frames(ctx.ctx, [t.data_ptr() for t in ins_t], w, [t.data_ptr() for t in outs_t], w, w, h)
        return [t.numpy().copy() for t in outs_t]
    canny.canny_run_frames(ctx.ctx, [f.ctypes.data for f in frames], w, [o.ctypes.data for o in outs], w, w, h)
    return outs


def test_frames_equal_single_runs_and_oracle():
    frames = [synth.image(600 + i, 300, 200, 8, 8, 8) for i in range(7)]
    with canny.Canny(320, 240) as c:
        got = frames_run(c, frames, 300, 200)
        assert c.stats()["images"] == 7
        # pageable host buffers: same results, copies do not overlap
        got_pageable = frames_run(c, frames, 300, 200, pin=False)
        for f, g, gp in zip(frames, got, got_pageable):
            want = oracle.canny_u8(f)
            assert np.array_equal(g, want)
            assert np.array_equal(gp, want)
            single = np.zeros_like(f)
            canny.canny_run_host(c.ctx, f.ctypes.data, 300, single.ctypes.data, 300, 300, 200, 0)
            assert np.array_equal(single, want)


def test_frames_new_size_and_new_tuning_rebuild_the_graphs():
    with canny.Canny(512, 512) as c:
        for (w, h) in [(512, 512), (97, 131), (512, 300)]:
            frames = [blocky_image(w * 3 + h + i, h, w) for i in range(3)]
            got = frames_run(c, frames, w, h)
            for f, g in zip(frames, got):
                assert np.array_equal(g, oracle.canny_u8(f))
        c.set_tuning(160, 12)
        frames = [blocky_image(77 + i, 300, 300) for i in range(4)]
        got = frames_run(c, frames, 300, 300)
        for f, g in zip(frames, got):
            assert np.array_equal(g, oracle.canny_u8(f))


def test_frames_single_frame_and_float_path():
    img = blocky_image(5, 150, 222)
    with canny.Canny(222, 150) as c:
        assert np.array_equal(frames_run(c, [img], 222, 150)[0], oracle.canny_u8(img))
    frames = [blocky_image(40 + i, 150, 222) for i in range(3)]
    with canny.Canny(222, 150, path=canny.CANNY_PATH_F32, low=0.1, high=0.3) as c:
        got = frames_run(c, frames, 222, 150)
    for f, g in zip(frames, got):
        assert np.array_equal(g, oracle.canny_f32(f, 1.4, 7, 0.1, 0.3))


def test_float_maps_grow_between_frames_and_single_runs():
    # the float path's strength/sector maps grow on demand; frame graphs that hold
    # the old maps are rebuilt, and every result stays equal to the oracle's
    small = [blocky_image(70 + i, 100, 130) for i in range(3)]
    large = blocky_image(80, 390, 517)
    want_small = [oracle.canny_f32(f, 1.4, 7, 0.1, 0.3) for f in small]
    with canny.Canny(517, 390, path=canny.CANNY_PATH_F32, low=0.1, high=0.3) as c:
        for f, g in zip(small, frames_run(c, small, 130, 100)):
            assert np.array_equal(g, oracle.canny_f32(f, 1.4, 7, 0.1, 0.3))
        out = torch.full(large.shape, 7, dtype=torch.uint8, device="cuda")
        c.run_pitched(dev(large), out)
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy(), oracle.canny_f32(large, 1.4, 7, 0.1, 0.3))
        for g, want in zip(frames_run(c, small, 130, 100), want_small):
            assert np.array_equal(g, want)


def test_batch_graph_variants_alternate():
    # all inputs TMA-readable (TMA-only kernel), then unaligned inputs repitched
    # (TMA-only kernel again), then direct loads (per-image kernel), then back
    imgs = [blocky_image(90 + i, h, w) for i, (h, w) in enumerate([(64, 128), (77, 301), (200, 33), (1, 16)])]
    wants = [oracle.canny_u8(im) for im in imgs]
    aligned_in, aligned_out = [], []
    for im in imgs:
        h, w = im.shape
        p = (w + 15) // 16 * 16
        t = torch.zeros((h, p), dtype=torch.uint8, device="cuda")
        t[:, :w] = dev(im)
        aligned_in.append(t[:, :w])
        aligned_out.append(torch.zeros((h, p), dtype=torch.uint8, device="cuda")[:, :w])
    tight_in = [dev(im) for im in imgs]
    total = sum(im.size for im in imgs) + 16 * 400
    with canny.Canny(total, 1) as c:
        for mode in ["aligned", "tight", "direct", "aligned", "tight"]:
            c.set_tuning(64, 12, 1 if mode == "direct" else 0)
            ins = aligned_in if mode == "aligned" else tight_in
            outs = aligned_out if mode == "aligned" else [torch.full(im.shape, 7, dtype=torch.uint8, device="cuda")
                                                          for im in imgs]
            for o in outs:
                o.fill_(7)
            c.run_batch(list(zip(ins, outs)))
            torch.cuda.synchronize()
            assert c.stats()["status"] == canny.CANNY_OK
            for o, want in zip(outs, wants):
                assert np.array_equal(o.cpu().numpy(), want), mode


def test_frames_argument_errors():
    lib = canny.load()
    with canny.Canny(64, 64) as c:
        P = ctypes.c_void_p
        one = (P * 1)(None)
        buf = np.zeros((64, 64), np.uint8)
        good = (P * 1)(buf.ctypes.data)
        assert lib.canny_run_frames(c.ctx, 1, one, 64, good, 64, 64, 64, None) == canny.CANNY_EINVAL
        assert lib.canny_run_frames(c.ctx, 1, good, 64, good, 64, 65, 64, None) == canny.CANNY_EINVAL
        assert lib.canny_run_frames(c.ctx, 1, good, 32, good, 64, 64, 64, None) == canny.CANNY_EINVAL
        assert lib.canny_run_frames(c.ctx, 0, None, 64, None, 64, 64, 64, None) == canny.CANNY_OK


# ------------------------------------------------------------------ float path
def float_reference(img, sigma=1.4, ksize=7, lo=0.1, hi=0.3):
    S = oracle.gauss_f32(img, sigma, ksize)
    gx, gy = oracle.sobel_f32(S)
    M = oracle.magnitude_f32(gx, gy)
    e, M2, cls = oracle.canny_f32(img, sigma, ksize, lo, hi, want_stages=True)
    assert np.array_equal(M, M2)
    return gx, gy, M, cls, e


@pytest.mark.parametrize("which", ["small", "blocky", "medium"])
def test_float_path(which):
    img = {"small": synth.small, "medium": synth.medium,
           "blocky": lambda: blocky_image(3, 333, 517)}[which]()
    h, w = img.shape
    gx, gy, M, cls, want = float_reference(img)
    with canny.Canny(w, h, path=canny.CANNY_PATH_F32, low=0.1, high=0.3) as c:
        d_in = dev(img)
        d_mag = torch.empty((h, w), dtype=torch.float32, device="cuda")
        d_max = torch.zeros(1, dtype=torch.float32, device="cuda")
        c.magnitude(d_in, d_mag, d_max)
        d_out = torch.empty_like(d_in)
        c.run_pitched(d_in, d_out)
        torch.cuda.synchronize()
        st = c.stats()
    Mg = d_mag.cpu().numpy()
    assert np.all(np.abs(Mg - M) <= 1e-5 * np.maximum(np.abs(M), 1.0))
    assert abs(float(d_max.item()) - float(M.max())) <= 1e-5 * float(M.max())
    assert st["status"] == canny.CANNY_OK
    check_float_edges(d_out.cpu().numpy(), want, gx, gy, M, cls)


def test_float_other_sigma():
    img = blocky_image(9, 200, 300)
    gx, gy, M, cls, want = float_reference(img, 2.0, 11, 0.05, 0.2)
    with canny.Canny(300, 200, path=canny.CANNY_PATH_F32, sigma=2.0, ksize=11, low=0.05, high=0.2) as c:
        d_in = dev(img)
        d_out = torch.empty_like(d_in)
        c.run_pitched(d_in, d_out)
        torch.cuda.synchronize()
    check_float_edges(d_out.cpu().numpy(), want, gx, gy, M, cls, 0.05, 0.2)


def run_float(img, sigma=1.4, ksize=7, lo=0.1, hi=0.3):
    h, w = img.shape
    with canny.Canny(max(w, 1), max(h, 1), path=canny.CANNY_PATH_F32, sigma=sigma, ksize=ksize,
                     low=lo, high=hi) as c:
        d_in = dev(img)
        d_out = torch.full((h, w), 7, dtype=torch.uint8, device="cuda")
        c.run_pitched(d_in, d_out)
        torch.cuda.synchronize()
        st = c.stats()
    return d_out.cpu().numpy(), st


# Two stencil passes, the second fused with the tile fill, in the definition's
# operation order: the edge maps are expected to equal the fp32 oracle's exactly
# (the tolerance check is the bar; equality is what the operation order gives).
@pytest.mark.parametrize("ksize,sigma", [(3, 0.8), (5, 1.0), (7, 1.4), (9, 2.0), (11, 2.0), (13, 2.5), (31, 6.0)])
@pytest.mark.parametrize("h,w", [(200, 300), (67, 131), (129, 257), (100, 512), (67, 400)])
def test_float_fused_every_kernel_size(ksize, sigma, h, w):
    img = blocky_image(ksize * 7 + h, h, w)
    gx, gy, M, cls, want = float_reference(img, sigma, ksize, 0.08, 0.25)
    got, st = run_float(img, sigma, ksize, 0.08, 0.25)
    assert st["status"] == canny.CANNY_OK
    check_float_edges(got, want, gx, gy, M, cls, 0.08, 0.25)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("h,w", [(1, 1), (1, 7), (5, 1), (3, 3), (31, 33), (64, 128), (65, 129)])
def test_float_fused_tiny_and_block_edges(h, w):
    img = noise_image(h * 1000 + w, h, w)
    gx, gy, M, cls, want = float_reference(img)
    got, st = run_float(img)
    assert st["status"] == canny.CANNY_OK
    check_float_edges(got, want, gx, gy, M, cls)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("seed", range(24))
def test_float_fused_exact_on_many_images(seed):
    # suppression ties between neighbours are decided by the last bit of the
    # strengths, so any rounding that differs from the definition shows up here
    # odd widths take the staged path; widths that are multiples of 16 and at least
    # 288 also take the register path for the blocks inside the image
    w = 130 + 3 * seed if seed % 2 else 288 + 16 * seed
    img = blocky_image(1000 + seed, 96 + seed, w)
    got, st = run_float(img)
    assert st["status"] == canny.CANNY_OK
    assert np.array_equal(got, oracle.canny_f32(img, 1.4, 7, 0.1, 0.3))


def test_float_fused_flat_image_has_no_edges():
    img = np.full((100, 150), 77, np.uint8)
    got, st = run_float(img)
    assert st["status"] == canny.CANNY_OK
    assert not got.any()


def test_float_batch_equals_single_runs_and_oracle():
    sizes = [(96, 130), (33, 47), (200, 64), (1, 9), (150, 150)]
    imgs = [blocky_image(50 + i, h, w) for i, (h, w) in enumerate(sizes)]
    total = sum(h * w for h, w in sizes)
    ins = [dev(im) for im in imgs]
    outs = [torch.full_like(x, 7) for x in ins]
    with canny.Canny(total, 1, path=canny.CANNY_PATH_F32, low=0.1, high=0.3) as c:
        c.run_batch(list(zip(ins, outs)))
        torch.cuda.synchronize()
        assert c.stats()["status"] == canny.CANNY_OK
    for im, o in zip(imgs, outs):
        gx, gy, M, cls, want = float_reference(im)
        got = o.cpu().numpy()
        check_float_edges(got, want, gx, gy, M, cls)
        assert np.array_equal(got, want)
        single, _ = run_float(im)
        assert np.array_equal(got, single)


# ------------------------------------------------------------------ full-size workloads
@pytest.mark.parametrize("which", ["uhd", "huge"])
def test_full_size_workloads_bit_exact(which):
    img = getattr(synth, which)()
    out, st = run_int(img)
    assert st["status"] == canny.CANNY_OK
    want = oracle.canny_u8(img)
    assert np.array_equal(out, want), int((out != want).sum())


# ------------------------------------------------------------------ batched integer path
def _batch_run(c, imgs):
    ins = [dev(im) for im in imgs]
    outs = [torch.full(im.shape, 3, dtype=torch.uint8, device="cuda") for im in imgs]
    c.run_batch(list(zip(ins, outs)))
    torch.cuda.synchronize()
    return [o.cpu().numpy() for o in outs], c.stats()


def test_batch_many_uneven_images_two_calls():
    rng = np.random.default_rng(31)
    sizes = [(int(h), int(w)) for h, w in rng.integers(1, 400, (150, 2))]
    imgs = [synth.image(500 + i, w, h, 4, 4, 8) for i, (h, w) in enumerate(sizes)]
    total = sum(w * h for h, w in sizes)
    with canny.Canny(total, 1) as c:
        for rep in range(2):           # two calls: alternate staging slots, reuse graphs
            outs, st = _batch_run(c, imgs if rep == 0 else imgs[::-1])
            assert st["status"] == canny.CANNY_OK
            src = imgs if rep == 0 else imgs[::-1]
            for im, o in zip(src, outs):
                assert np.array_equal(o, oracle.canny_u8(im))


@pytest.mark.parametrize("band,ctas,direct", [(32, 0, 0), (32, 12, 1), (64, 0, 0), (64, 8, 0), (160, 12, 0), (256, 4, 0), (256, 0, 1),
                                               (64, 16, 1), (160, 12, 1)])
def test_every_tuning_gives_identical_edges(band, ctas, direct):
    imgs = [synth.image(900 + i, w, h, 8, 8, 10) for i, (h, w) in
            enumerate([(300, 500), (1, 70), (257, 33), (700, 449)])]
    total = sum(im.size for im in imgs)
    with canny.Canny(max(total, 700 * 700), 1) as c:
        c.set_tuning(band, ctas, direct)
        assert canny.canny_get_tuning(c.ctx).direct_loads == direct
        outs, st = _batch_run(c, imgs)
        for im, o in zip(imgs, outs):
            assert np.array_equal(o, oracle.canny_u8(im))
    with canny.Canny(700, 700) as c:
        c.set_tuning(band, ctas, direct)
        for im in imgs:
            out, _ = run_int(im, ctx=c)
            assert np.array_equal(out, oracle.canny_u8(im))


def serpentine_u8(n, gap=32):
    """A 3-pixel bar of grey 32 on black through every 32 x 32 tile of an n x n
    image (runs every `gap` rows joined at alternate ends), its first 8 pixels
    at grey 80: with thresholds 40/100 the bar's edges are one weak chain whose
    only strong pixels sit at its start."""
    img = np.zeros((n, n), np.uint8)
    rows = list(range(gap // 2, n, gap))
    for j, r in enumerate(rows):
        img[r - 1:r + 2, 2:n - 2] = 32
        if j + 1 < len(rows):
            c = n - 3 if j % 2 == 0 else 2
            img[r:rows[j + 1] + 1, c - 1:c + 2] = 32
    img[rows[0] - 1:rows[0] + 2, 2:10] = 80
    return img


def test_serpentine_u8_is_one_long_weak_chain():
    img = serpentine_u8(256)
    cls = oracle.classify_u8(img, 40, 100)
    out = oracle.canny_u8(img, 40, 100)
    assert (cls == 2).sum() < 32 and (cls == 1).sum() > 4000
    assert (out == 255).sum() == (cls > 0).sum()          # every weak pixel is reached


@pytest.mark.parametrize("budget,passes", [(1, 0), (1, 1), (16, 0), (16, 1), (64, 1), (256, 0), (4096, 1)])
def test_every_pass_schedule_gives_identical_edges(budget, passes):
    """Chase budget x while-loop or cooperative node: batches holding a chain
    through 1024 tiles, images that end inside a tile and an empty-edged one,
    and single images through the same context."""
    imgs = [serpentine_u8(1024), synth.image(950, 300, 500, 8, 8, 10), serpentine_u8(320)[:, :301],
            synth.image(951, 70, 1, 8, 8, 10), np.zeros((33, 65), np.uint8)]
    total = sum(im.size for im in imgs)
    with canny.Canny(total, 1) as c:
        c.set_tuning(64, 0, 0, budget, passes)
        t = canny.canny_get_tuning(c.ctx)
        assert (t.chase_budget, t.batch_passes) == (budget, passes)
        for rep in range(2):
            outs, st = _batch_run(c, imgs)
            assert st["status"] == canny.CANNY_OK
            for im, o in zip(imgs, outs):
                assert np.array_equal(o, oracle.canny_u8(im))
    with canny.Canny(1024, 1024) as c:
        c.set_tuning(0, 0, 0, budget, passes)
        out, st = run_int(imgs[0], ctx=c)
        assert np.array_equal(out, oracle.canny_u8(imgs[0]))
        cls = serpentine_map(1024)
        h, _ = run_hyst(cls, ctx=c)
        assert np.array_equal(h, oracle.hysteresis(cls))


def test_tuning_rejects_out_of_range_schedules():
    with canny.Canny(64, 64) as c:
        for band, ctas, direct, budget, passes in [(64, 0, 0, -1, 0), (64, 0, 0, 4097, 0), (64, 0, 0, 0, 2),
                                                   (48, 0, 0, 0, 0), (64, 33, 0, 0, 0), (64, 0, 2, 0, 0)]:
            with pytest.raises(canny.CannyError):
                c.set_tuning(band, ctas, direct, budget, passes)
        c.set_tuning(32, 4, 1, 4096, 1)
        t = canny.canny_get_tuning(c.ctx)
        assert (t.band, t.ctas_per_sm, t.direct_loads, t.chase_budget, t.batch_passes) == (32, 4, 1, 4096, 1)


def test_autotune_picks_a_supported_config_and_caches_it(tmp_path):
    rng = np.random.default_rng(5)
    sizes = [(int(h), int(w)) for h, w in rng.integers(64, 300, (40, 2))]
    imgs = [synth.image(700 + i, w, h, 4, 4, 8) for i, (h, w) in enumerate(sizes)]
    total = sum(w * h for h, w in sizes)
    cache = str(tmp_path / "tune.jsonl")
    ins = [dev(im) for im in imgs]
    outs = [torch.empty_like(x) for x in ins]
    with canny.Canny(total, 1) as c:
        t1 = c.autotune_batch(list(zip(ins, outs)), cache_path=cache)
        assert t1["band"] in (32, 64, 160) and t1["ctas_per_sm"] in (0, 12, 16) and t1["from_cache"] == 0
        assert t1["chase_budget"] in (0, 4, 16, 64) and t1["batch_passes"] in (0, 1)
        assert t1["direct_loads"] in (0, 1)                 # widths not multiples of 16: both layouts timed
        t2 = c.autotune_batch(list(zip(ins, outs)), cache_path=cache)
        keys = ("band", "ctas_per_sm", "direct_loads", "chase_budget", "batch_passes")
        assert t2["from_cache"] == 1 and all(t2[k] == t1[k] for k in keys)
        assert all(getattr(canny.canny_get_tuning(c.ctx), k) == t1[k] for k in keys)
        c.run_batch(list(zip(ins, outs)))
        torch.cuda.synchronize()
    for im, o in zip(imgs, outs):
        assert np.array_equal(o.cpu().numpy(), oracle.canny_u8(im))


# ------------------------------------------------------------------ serving
def _trace(n, seed, spread_s):
    rng = np.random.default_rng(seed)
    sizes = [(int(h), int(w)) for h, w in rng.integers(16, 320, (n, 2))]
    imgs = [synth.image(1200 + i, w, h, 4, 4, 8) for i, (h, w) in enumerate(sizes)]
    arrivals = np.sort(rng.random(n) * spread_s)
    return imgs, arrivals


def _serve(imgs, arrivals, serial=0, budget=64 << 20, streams=2, max_batch_images=64):
    outs = [np.full(im.shape, 9, np.uint8) for im in imgs]
    reqs = [canny.canny_request(im.shape[1], im.shape[0], im.ctypes.data, im.strides[0],
                                o.ctypes.data, o.strides[0], float(t))
            for im, o, t in zip(imgs, outs, arrivals)]
    cfg = canny.canny_serve_config(float(budget), streams, max_batch_images, 1 << 24, serial, 40, 100, 0, 0)
    lat = np.zeros(len(imgs))
    rep = canny.canny_serve(cfg, reqs, lat).as_dict()
    return outs, rep, lat


def test_serving_results_equal_alone_and_in_the_mix():
    # half the requests arrive together (they must share batches), the rest spread
    # over 20 ms, arriving while earlier batches run
    imgs, arrivals = _trace(60, 11, 0.02)
    arrivals[:30] = 0.0
    outs, rep, lat = _serve(imgs, arrivals)
    assert rep["completed"] == len(imgs) and (lat > 0).all()
    outs_serial, rep_s, _ = _serve(imgs, arrivals, serial=1)
    for im, o, o1 in zip(imgs, outs, outs_serial):
        want = oracle.canny_u8(im)
        assert np.array_equal(o, want)        # in the mix
        assert np.array_equal(o1, want)       # alone
    assert rep["batches"] < len(imgs) and rep["mean_batch_images"] > 1.0


def test_serving_pinned_and_pageable_host_buffers():
    # pinned, tight and aligned buffers go through one gather / scatter kernel per
    # batch; pageable, unaligned or padded ones through copy-engine copies
    imgs, arrivals = _trace(40, 13, 0.02)
    reqs, keep, outs = [], [], []
    for i, (im, t) in enumerate(zip(imgs, arrivals)):
        h, w = im.shape
        kind = i % 4
        if kind == 0:                                  # pinned, tight: kernel path both ways
            src = torch.from_numpy(im.copy()).pin_memory()
            dst = torch.full((h, w), 9, dtype=torch.uint8).pin_memory()
            keep += [src, dst]
            reqs.append(canny.canny_request(w, h, src.data_ptr(), w, dst.data_ptr(), w, float(t)))
            outs.append(lambda d=dst: d.numpy())
        elif kind == 1:                                # pageable
            dst = np.full((h, w), 9, np.uint8)
            keep += [im, dst]
            reqs.append(canny.canny_request(w, h, im.ctypes.data, w, dst.ctypes.data, w, float(t)))
            outs.append(lambda d=dst: d)
        elif kind == 2:                                # pinned but one byte off 16-byte alignment
            buf = torch.zeros(h * w + 1, dtype=torch.uint8).pin_memory()
            buf[1:] = torch.from_numpy(im.reshape(-1))
            dbuf = torch.full((h * w + 1,), 9, dtype=torch.uint8).pin_memory()
            keep += [buf, dbuf]
            reqs.append(canny.canny_request(w, h, buf.data_ptr() + 1, w, dbuf.data_ptr() + 1, w, float(t)))
            outs.append(lambda d=dbuf, h=h, w=w: d[1:].numpy().reshape(h, w))
        else:                                          # pinned, padded rows
            src = torch.zeros((h, w + 7), dtype=torch.uint8).pin_memory()
            src[:, :w] = torch.from_numpy(im)
            dst = torch.full((h, w + 5), 9, dtype=torch.uint8).pin_memory()
            keep += [src, dst]
            reqs.append(canny.canny_request(w, h, src.data_ptr(), w + 7, dst.data_ptr(), w + 5, float(t)))
            outs.append(lambda d=dst, w=w: d.numpy()[:, :w])
    cfg = canny.canny_serve_config(float(64 << 20), 2, 64, 1 << 24, 0, 40, 100, 0, 0)
    rep = canny.canny_serve(cfg, reqs).as_dict()
    assert rep["completed"] == len(imgs)
    for i, (im, get) in enumerate(zip(imgs, outs)):
        assert np.array_equal(get(), oracle.canny_u8(im)), i
    # padding bytes of the padded output rows are untouched
    for i in range(3, len(imgs), 4):
        d = keep[2 * i + 1].numpy()
        assert (d[:, imgs[i].shape[1]:] == 9).all()


def test_serving_under_a_tight_memory_budget():
    imgs, arrivals = _trace(30, 12, 0.0)     # everything arrives at once
    biggest = max((((im.shape[1] + 15) // 16) * 16) * im.shape[0] for im in imgs)
    budget = 2 * (biggest + 256) * 3         # room for about three requests
    outs, rep, _ = _serve(imgs, arrivals, budget=budget)
    assert rep["completed"] == len(imgs) and rep["peak_bytes"] <= budget
    for im, o in zip(imgs, outs):
        assert np.array_equal(o, oracle.canny_u8(im))


def test_batch_tma_inputs_rewritten_between_calls():
    """Pitches that are multiples of 16 take the TMA path; the descriptors of a
    later batch reuse the device addresses of the earlier one's."""
    with canny.Canny(4 * 512 * 512, 1) as c:
        for rep in range(4):
            imgs = [synth.image(3000 + 10 * rep + i, w, h, 5, 5, 8)
                    for i, (h, w) in enumerate([(232, 32), (300, 480), (64, 16), (511, 496)])]
            outs, st = _batch_run(c, imgs)
            assert st["status"] == canny.CANNY_OK
            for im, o in zip(imgs, outs):
                assert np.array_equal(o, oracle.canny_u8(im))


@pytest.mark.parametrize("seed", [11, 12, 13])
def test_random_sizes_offsets_and_pitches_match_the_oracle(seed):
    # random widths 1..2999 and heights 1..599, input and output views at any
    # byte offset and with padded pitches (staging, unaligned stores, ragged
    # strips and bands), the float path on every third case
    rng = np.random.default_rng(seed)
    with canny.Canny(3000, 600) as ci, canny.Canny(3000, 600, path=canny.CANNY_PATH_F32, low=0.1, high=0.3) as cf:
        for k in range(50):
            w, h = int(rng.integers(1, 3000)), int(rng.integers(1, 600))
            img = synth.image(int(rng.integers(0, 1 << 30)), w, h, int(rng.integers(1, 40)), int(rng.integers(1, 40)),
                              int(rng.integers(0, 16)))
            views = []
            for _ in range(2):
                off, pitch = int(rng.integers(0, 16)), w + int(rng.integers(0, 40))
                buf = torch.full((off + h * pitch + 64,), 7, dtype=torch.uint8, device="cuda")
                views.append(buf[off:off + (h - 1) * pitch + w].as_strided((h, w), (pitch, 1)))
            src, dst = views
            src.copy_(dev(img))
            ci.run_pitched(src, dst)
            torch.cuda.synchronize()
            assert ci.stats()["status"] == canny.CANNY_OK
            assert np.array_equal(dst.cpu().numpy(), oracle.canny_u8(img)), (w, h)
            if k % 3 == 0 and w * h <= 400000:
                dst.fill_(7)
                cf.run_pitched(src, dst)
                torch.cuda.synchronize()
                assert np.array_equal(dst.cpu().numpy(), oracle.canny_f32(img, 1.4, 7, 0.1, 0.3)), (w, h)
