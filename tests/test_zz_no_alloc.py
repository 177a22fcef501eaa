"""canny_run_noalloc: the integer pipeline for callers that cannot allocate device
memory (a budget held by another allocator, or loops where cudaMalloc/cudaFree's
implicit synchronisation is not allowed). Its scratch is a fixed array in the
library, so these checks run it twice in a row (the second call must not see the
first call's leftovers) and compare each result with canny_run_pitched.

This file is collected last on purpose: it must pass both alone in a fresh
process and after every other test.
"""
import ctypes

import numpy as np
import pytest

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


@pytest.mark.gpu
def test_noalloc_matches_canny_run_on_two_calls_in_a_row():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1710_07745_gb300 import canny

    cases = [synth.image(4242, 1500, 1100, 30, 30, 10), synth.image(4243, 613, 977, 12, 12, 8)]
    for img in cases:
        h, w = img.shape
        d_in = torch.from_numpy(img).cuda()
        d_out = torch.full((h, w), 9, dtype=torch.uint8, device="cuda")
        canny.canny_run_noalloc(d_in.data_ptr(), w, d_out.data_ptr(), w, w, h, 40, 100,
                                torch.cuda.current_stream().cuda_stream)
        d_ref = torch.full((h, w), 5, dtype=torch.uint8, device="cuda")
        with canny.Canny(w, h, low=40, high=100) as c:
            c.run_pitched(d_in, d_ref)
            torch.cuda.synchronize()
            assert c.stats()["status"] == canny.CANNY_OK
        got, ref = d_out.cpu().numpy(), d_ref.cpu().numpy()
        assert np.array_equal(got, ref), int((got != ref).sum())
        assert (got == 255).any()
