"""Failure detection on the GPU path without a GPU fault: allocation failures
injected on the host (canny_inject_faults) must come back as CANNY_ENOMEM, or
be absorbed where a fallback exists, and leave the library usable; serving
admissions that find no room are deferred, not lost; a device-side wait that
can never complete (a grid-barrier arrival nobody makes) runs out, is reported
as CANNY_ECUDA, and the context stays usable."""
import numpy as np
import pytest

import oracle
from paper_1710_07745_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1710_07745_gb300 import canny  # noqa: E402


@pytest.fixture(autouse=True)
def no_injection_left():
    yield
    canny.canny_inject_faults()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_context_creation_reports_enomem_and_recovers():
    p = canny.canny_params_default()
    canny.canny_inject_faults(device_allocations=1)
    with pytest.raises(canny.CannyError) as ei:
        canny.canny_create(256, 256, p)
    assert ei.value.status == canny.CANNY_ENOMEM
    img = synth.image(5, 256, 200, 4, 4, 8)
    with canny.Canny(256, 200) as c:               # the next allocation succeeds
        out = torch.empty((200, 256), dtype=torch.uint8, device="cuda")
        c.run(dev(img), out)
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy(), oracle.canny_u8(img))


def test_staging_allocation_failure_falls_back_to_direct_loads():
    img = synth.image(6, 301, 203, 6, 6, 8)
    big = torch.zeros((203, 320), dtype=torch.uint8, device="cuda")
    big[:, 3:304] = dev(img)
    view = big[:, 3:304]                           # not TMA-readable: would be repitched
    out = torch.full((203, 301), 7, dtype=torch.uint8, device="cuda")
    with canny.Canny(301, 203) as c:
        canny.canny_inject_faults(device_allocations=1)    # the staging buffer cannot be had
        c.run_pitched(view, out)
        torch.cuda.synchronize()
        assert c.stats()["status"] == canny.CANNY_OK
        assert np.array_equal(out.cpu().numpy(), oracle.canny_u8(img))


def test_float_map_allocation_failure_is_enomem_then_recovers():
    img = synth.image(7, 208, 150, 4, 4, 8)      # a 16-byte pitch: no staging copy first
    out = torch.full((150, 208), 7, dtype=torch.uint8, device="cuda")
    with canny.Canny(208, 150, path=canny.CANNY_PATH_F32, low=0.1, high=0.3) as c:
        canny.canny_inject_faults(device_allocations=1)
        with pytest.raises(canny.CannyError) as ei:
            c.run_pitched(dev(img), out)
        assert ei.value.status == canny.CANNY_ENOMEM
        c.run_pitched(dev(img), out)
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy(), oracle.canny_f32(img, 1.4, 7, 0.1, 0.3))


def _requests(imgs, outs):
    return [canny.canny_request(im.shape[1], im.shape[0], im.ctypes.data, im.strides[0],
                                o.ctypes.data, o.strides[0], 0.0) for im, o in zip(imgs, outs)]


def test_serving_defers_admissions_that_find_no_room():
    rng = np.random.default_rng(3)
    imgs = [synth.image(1300 + i, int(w), int(h), 4, 4, 8) for i, (h, w) in enumerate(rng.integers(16, 200, (24, 2)))]
    outs = [np.full(im.shape, 9, np.uint8) for im in imgs]
    cfg = canny.canny_serve_config(float(64 << 20), 2, 64, 1 << 24, 0, 40, 100, 0, 0)
    canny.canny_inject_faults(arena_admissions=7)
    rep = canny.canny_serve(cfg, _requests(imgs, outs)).as_dict()
    assert rep["completed"] == len(imgs) and rep["deferrals"] >= 7
    for im, o in zip(imgs, outs):
        assert np.array_equal(o, oracle.canny_u8(im))


def test_serving_budget_allocation_failure_and_oversized_request():
    imgs = [synth.image(1400, 120, 90, 4, 4, 8)]
    outs = [np.full(imgs[0].shape, 9, np.uint8)]
    cfg = canny.canny_serve_config(float(64 << 20), 2, 64, 1 << 24, 0, 40, 100, 0, 0)
    canny.canny_inject_faults(device_allocations=1)       # the budget itself
    with pytest.raises(canny.CannyError) as ei:
        canny.canny_serve(cfg, _requests(imgs, outs))
    assert ei.value.status == canny.CANNY_ENOMEM
    small = canny.canny_serve_config(float(4096), 2, 64, 1 << 24, 0, 40, 100, 0, 0)
    with pytest.raises(canny.CannyError) as ei:     # 2 x 128 x 90 bytes cannot fit in 4 KB
        canny.canny_serve(small, _requests(imgs, outs))
    assert ei.value.status == canny.CANNY_EINVAL
    rep = canny.canny_serve(cfg, _requests(imgs, outs)).as_dict()
    assert rep["completed"] == 1 and np.array_equal(outs[0], oracle.canny_u8(imgs[0]))


def test_stalled_grid_barrier_times_out_and_is_reported():
    img = synth.image(8, 256, 192, 8, 8, 8)
    out = torch.full((192, 256), 7, dtype=torch.uint8, device="cuda")
    with canny.Canny(256, 192) as c:
        canny.canny_inject_faults(stalled_barriers=1)
        c.run(dev(img), out)
        torch.cuda.synchronize()
        assert c.stats()["status"] == canny.CANNY_ECUDA
        out.fill_(7)
        c.run(dev(img), out)                       # the next run is exact again
        torch.cuda.synchronize()
        assert c.stats()["status"] == canny.CANNY_OK
        assert np.array_equal(out.cpu().numpy(), oracle.canny_u8(img))



def test_host_driven_passes_give_the_oracle_edges():
    """The path taken when the device refuses the cooperative grid (forced by the
    host-side hook): one global pass per launch, driven from the host, on a weak
    serpentine through every tile with a strong pixel at its start (more passes
    than one: the chase budget per worklist entry runs out)."""
    n, gap = 1024, 32
    cls = np.zeros((n, n), np.uint8)
    rows = list(range(gap // 2, n, gap))
    for j, r in enumerate(rows):
        cls[r, :] = 1
        if j + 1 < len(rows):
            col = n - 1 if j % 2 == 0 else 0
            cls[r:rows[j + 1] + 1, col] = 1
    cls[rows[0], 0] = 2
    with canny.Canny(n, n) as c:
        out = torch.full((n, n), 7, dtype=torch.uint8, device="cuda")
        canny.canny_inject_faults(host_driven_passes=1)
        c.hysteresis(dev(cls), out)
        torch.cuda.synchronize()
        st = c.stats()
        assert st["status"] == canny.CANNY_OK and st["hyst_passes"] >= 1
        got = out.cpu().numpy()
        assert np.array_equal(got, oracle.hysteresis(cls))
        assert (got == 255).sum() == (cls > 0).sum()
