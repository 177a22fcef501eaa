"""canny_run_noalloc: the integer pipeline for callers that cannot allocate device
memory (a budget held by another allocator, or loops where cudaMalloc/cudaFree's
implicit synchronisation is not allowed). Its scratch is a fixed array in the
library, so these checks run it several times in a row (no call may see an
earlier call's leftovers) and compare every result with the oracle and with
canny_run_pitched on a context.

This file is collected last on purpose: it must pass both alone in a fresh
process and after every other test.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1710_07745_gb300 import synth


def test_noalloc_rejects_images_beyond_its_fixed_scratch():
    from paper_1710_07745_gb300 import canny
    lib = canny.load()
    # 4097 x 4096 needs 129 x 128 = 16512 tiles > 16384; rejected before any CUDA call
    rc = lib.canny_run_noalloc(ctypes.c_void_p(16), 4097, ctypes.c_void_p(1 << 40), 4097,
                               4097, 4096, 40, 100, None)
    assert rc == canny.CANNY_EUNSUPPORTED
    assert lib.canny_run_noalloc(None, 8, None, 8, 8, 8, 40, 100, None) == canny.CANNY_EINVAL
    assert lib.canny_run_noalloc(ctypes.c_void_p(16), 8, ctypes.c_void_p(4096), 8, 8, 8,
                                 50, 40, None) == canny.CANNY_EINVAL


def _device():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _noalloc(torch, img, in_off=0, in_pad=0, out_pad=0):
    """Run canny_run_noalloc on img placed at byte offset in_off of rows padded by
    in_pad bytes; the output rows are padded by out_pad bytes of sentinel 7."""
    from paper_1710_07745_gb300 import canny
    h, w = img.shape
    in_pitch, out_pitch = w + in_pad, w + out_pad
    buf = torch.zeros(in_off + h * in_pitch, dtype=torch.uint8, device="cuda")
    buf[in_off:].view(h, in_pitch)[:, :w] = torch.from_numpy(img).cuda()
    out = torch.full((h, out_pitch), 7, dtype=torch.uint8, device="cuda")
    canny.canny_run_noalloc(buf.data_ptr() + in_off, in_pitch, out.data_ptr(), out_pitch, w, h, 40, 100,
                            torch.cuda.current_stream().cuda_stream)
    got = out.cpu().numpy()
    assert (got[:, w:] == 7).all(), "padding bytes were written"
    return got[:, :w], buf, in_pitch


def _context(torch, img):
    from paper_1710_07745_gb300 import canny
    h, w = img.shape
    d_in = torch.from_numpy(img).cuda()
    d_ref = torch.full((h, w), 5, dtype=torch.uint8, device="cuda")
    with canny.Canny(w, h, low=40, high=100) as c:
        c.run_pitched(d_in, d_ref)
        torch.cuda.synchronize()
        assert c.stats()["status"] == canny.CANNY_OK
    return d_ref.cpu().numpy()


@pytest.mark.gpu
def test_noalloc_matches_the_oracle_and_canny_run_call_after_call():
    torch = _device()
    # unaligned widths (direct loads), a 16-byte pitch (the TMA instantiation),
    # the exact capacity (4096 x 4096 = 16384 tiles fills the array to its end),
    # then a small image right after the largest
    cases = [(synth.image(4242, 1500, 1100, 30, 30, 10), 0, 0, 0),
             (synth.image(4243, 613, 977, 12, 12, 8), 0, 0, 0),
             (synth.image(4244, 1024, 768, 20, 20, 8), 0, 0, 0),
             (synth.image(4245, 4096, 4096, 200, 200, 8), 0, 0, 0),
             (synth.image(4246, 333, 201, 6, 6, 8), 0, 0, 0),
             (synth.image(4247, 1000, 300, 10, 10, 8), 3, 5, 9)]
    for img, off, ipad, opad in cases:
        got, _, _ = _noalloc(torch, img, off, ipad, opad)
        want = oracle.canny_u8(img, 40, 100)
        assert np.array_equal(got, want), (img.shape, int((got != want).sum()))
        ref = _context(torch, img)
        assert np.array_equal(got, ref)
        assert (got == 255).any()


@pytest.mark.gpu
def test_noalloc_host_driven_passes_match_the_oracle():
    """The fallback taken when the device refuses the cooperative grid: the host
    launches one global pass at a time (forced here by the host-side test hook)."""
    torch = _device()
    from paper_1710_07745_gb300 import canny
    img = synth.image(4250, 900, 700, 14, 14, 10)
    want = oracle.canny_u8(img, 40, 100)
    canny.canny_inject_faults(host_driven_passes=1)
    try:
        got, _, _ = _noalloc(torch, img)
    finally:
        canny.canny_inject_faults()
    assert np.array_equal(got, want), int((got != want).sum())
    again, _, _ = _noalloc(torch, img)                  # and the cooperative launch after it
    assert np.array_equal(again, want)
