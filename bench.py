"""Throughput benchmark of the Canny pipeline on one GB300 (or N replicas).

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

One step = the whole pipeline (fused stencil, tile-local hysteresis, global
hysteresis passes) over one synthetic 16384 x 16384 uint8 image (3200
rectangles, 3200 disks, noise sigma 12; thresholds 40/100), inputs resident in
HBM. Inputs (268 MB) and outputs (268 MB) are larger than the 129 MB L2, so no
flush is needed between steps. Prints one JSON line.

--impl reference times the CPU oracle (single thread) on a bounded sample of
the same workload instead. Under torchrun (N > 1) each rank runs its own
replica of the image: the units (images) are independent, so the job scales
weakly with no collective on the data path; rank 0 prints the line with the
max-over-ranks time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

W = H = 16384
N_OBJ = 3200  # objects per kind at 16384^2 (200 per 4096^2 of area)
NOISE = 12
SEED = 3001
LOW, HIGH = 40, 100
METRIC = "Canny Mpixel/s & % of HBM roofline; batched vs plain loop; p50/p99 latency"
UNIT = "Mpixel/s"
WORKLOAD = "canny_int_16384x16384"
# algorithmic bytes per pixel of the stencil stage (fused stencil + tile fill): read the
# image byte, write the edge byte
K1_BYTES_PER_PX = 2
# the design's own traffic per pixel: the 2-bit class masks per pixel go from the
# stencil to the tile fill and back (0.25 B/px each way)
K1_DESIGN_BYTES_PER_PX = 2.5
# ncu DRAM traffic of the two stencil-stage kernels per 16384^2 image, valid only for
# the kernel sources it was measured on (a 16384 x 8192 capture, x2: both kernels'
# traffic is proportional to the pixels)
K1_TRAFFIC = {"sha256_prefix": "f8399db8212309d6", "bytes": 568.5e6}
# whole pipeline floor (the spec minimum): read the image, write the edge map
PIPE_BYTES_PER_PX = 2
# ncu smsp__inst_executed.sum of the two stencil-stage kernels per pixel (same
# capture and sources as K1_TRAFFIC)
K1_INST = {"sha256_prefix": "f8399db8212309d6", "warp_inst_per_px": 0.9740}
# ncu DRAM traffic of the global hysteresis passes per 16384^2 image (same capture,
# x2: an estimate, since the passes' work follows the image's chains, not its area)
K3_TRAFFIC = {"sha256_prefix": "ecd40c592ae66c79", "bytes": 9.46e6}
# warp instructions an SM can issue per clock (4 schedulers, one each)
ISSUE_PER_SM_CLK = 4


def measured_peaks() -> dict:
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return {"hbm_gbs": float(d["hbm_gbs"]), "source": "measured"}
    return {"hbm_gbs": 6800.0, "source": "fallback"}


def src_digest(names) -> str:
    """sha256 over the named kernel sources."""
    import hashlib
    h = hashlib.sha256()
    for name in names:
        with open(os.path.join(ROOT, "paper_1710_07745_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def k1_digest() -> str:
    """The stencil stage's sources: fused stencil, tile fill, the tile header."""
    return src_digest(("k1_fused.cu", "tile_fill.cu", "hyst_tile.cuh", "canny_internal.cuh"))


def k3_digest() -> str:
    """The global passes' sources."""
    return src_digest(("hysteresis.cu", "hyst_tile.cuh", "canny_internal.cuh"))


def k1_traffic(w: int, h: int):
    """Recorded ncu DRAM bytes per launch, if the kernel source is unchanged since."""
    if not K1_TRAFFIC["sha256_prefix"] or not k1_digest().startswith(K1_TRAFFIC["sha256_prefix"]) or \
            (w, h) != (16384, 16384):
        return None
    return K1_TRAFFIC["bytes"]


def k3_traffic(w: int, h: int):
    """Recorded ncu DRAM bytes of the global passes, if the sources are unchanged since."""
    if not K3_TRAFFIC["sha256_prefix"] or not k3_digest().startswith(K3_TRAFFIC["sha256_prefix"]) or \
            (w, h) != (16384, 16384):
        return None
    return K3_TRAFFIC["bytes"]


def alu_roofline(px: int, k1_ms: float, hbm_gbs: float, clk: dict | None) -> dict | None:
    """Issue-rate roofline of the fused kernel: its recorded warp instructions per
    launch over the CUDA-event launch time, against SMs x 4 issue slots x the SM clock.
    None once the kernel source differs from the one the count was taken on."""
    import torch
    if not K1_INST["sha256_prefix"] or not k1_digest().startswith(K1_INST["sha256_prefix"]):
        return None
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    mhz = (clk or {}).get("sm_max_mhz") or 2070.0
    peak = sms * ISSUE_PER_SM_CLK * mhz * 1e6 / 1e9            # G warp instructions / s
    inst = K1_INST["warp_inst_per_px"] * px
    achieved = inst / (k1_ms / 1e3) / 1e9
    alu_px_s = peak * 1e9 / K1_INST["warp_inst_per_px"]      # pixel rate if issue-bound
    hbm_px_s = hbm_gbs * 1e9 / K1_BYTES_PER_PX               # pixel rate if HBM-bound
    px_s = px / (k1_ms / 1e3)
    return {"bound": "alu", "achieved": round(achieved, 1), "peak": round(peak, 1), "unit": "Ginst/s",
            "frac": round(achieved / peak, 4), "warp_inst_per_px": round(K1_INST["warp_inst_per_px"], 4),
            "peak_basis": f"{sms} SMs x {ISSUE_PER_SM_CLK} warp instructions/clock x {mhz:.0f} MHz",
            "bound_mpx_s": {"alu": round(alu_px_s / 1e6, 1), "hbm": round(hbm_px_s / 1e6, 1)},
            "frac_of_min_bound": round(px_s / min(alu_px_s, hbm_px_s), 4)}


def config(extra: dict | None = None) -> dict:
    c = {"workload": WORKLOAD, "w": W, "h": H, "objects_per_kind": N_OBJ, "noise_sigma": NOISE,
         "seed": SEED, "low": LOW, "high": HIGH, "path": "integer",
         "l2": "inputs+outputs 512 MiB > 129 MB L2, no flush"}
    if extra:
        c.update(extra)
    return c


# ------------------------------------------------------------------ distributed plumbing
def dist_init(n_gpus: int):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if os.environ.get("CANNY_BENCH_BACKEND", "nccl") == "nccl" else "gloo"
        dist.init_process_group(backend=backend)
    return rank, world


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def job_value(world: int, steps: int, px_per_step: int, ms_max: float) -> float:
    """Whole-job Mpixel/s: every rank runs its own image per step (weak scaling),
    timed by the slowest rank."""
    return world * steps * px_per_step / (ms_max / 1e3) / 1e6


def max_over_ranks(v: float, world: int) -> float:
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------------ clocks during the timed region
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines: list[str] = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.t:
            self.t.join(timeout=2)
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ------------------------------------------------------------------ CPU legs (oracle)
def cpu_info() -> dict:
    """The host the oracle baselines ran on: core count and CPU model."""
    import platform
    import re
    model = None
    try:
        with open("/proc/cpuinfo") as f:
            txt = f.read()
        m = re.search(r"^model name\s*:\s*(.+)$", txt, re.M)
        if m:
            model = m.group(1).strip()
        else:
            impl = re.search(r"^CPU implementer\s*:\s*(\S+)", txt, re.M)
            part = re.search(r"^CPU part\s*:\s*(\S+)", txt, re.M)
            if impl and part:
                known = {("0x41", "0xd4f"): "Arm Neoverse V2", ("0x41", "0xd40"): "Arm Neoverse V1",
                         ("0x41", "0xd0c"): "Arm Neoverse N1"}
                model = known.get((impl.group(1).lower(), part.group(1).lower()),
                                  f"CPU implementer {impl.group(1)} part {part.group(1)}")
    except OSError:
        pass
    return {"nproc": os.cpu_count(), "cpu_model": model, "machine": platform.machine()}


def oracle_median(fn, runs: int = 3) -> float:
    """Median wall time of `runs` single-thread oracle calls."""
    ts = []
    for _ in range(runs):
        t0 = time.perf_counter()
        fn()
        ts.append(time.perf_counter() - t0)
    return statistics.median(ts)


def float_ambiguous(gx, gy, M, lo=0.1, hi=0.3, tol=1e-3):
    """Pixels where one of the oracle's float decisions (a threshold, the sector
    boundary, a suppression neighbour) lies within tol (relative): the only
    pixels, with those connected to them, where the float variant's edge map may
    differ from the oracle's."""
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


def float_error(img: np.ndarray, d_in, d_out, ctx, rows: int | None = None) -> dict:
    """The float variant against the fp32 oracle (run here, single thread): the
    largest relative strength error of the production kernel's strengths
    (canny_magnitude_f32 runs the pipeline's own first pass), and, on a whole
    image, the pixels whose edge bytes differ and the ambiguous pixels. rows:
    compare strengths on rows 0 .. rows - 1 only (the oracle runs on rows 0 ..
    rows + 7, so every compared row has its true neighbours)."""
    import torch

    import oracle
    from paper_1710_07745_gb300 import canny
    h, w = img.shape
    mag = torch.empty((h, w), dtype=torch.float32, device="cuda")
    mx = torch.zeros(1, dtype=torch.float32, device="cuda")
    canny.canny_magnitude_f32(ctx.ctx, canny.image_of(d_in, d_out), mag.data_ptr(), w, mx.data_ptr(),
                              torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    crop = img if rows is None else np.ascontiguousarray(img[:min(h, rows + 8)])
    t0 = time.perf_counter()
    e, M, cls = oracle.canny_f32(crop, want_stages=True)
    dt = time.perf_counter() - t0
    n = crop.shape[0] if rows is None else min(h, rows)
    got = mag[:n].cpu().numpy()
    ref = M[:n]
    rel = float(np.max(np.abs(got.astype(np.float64) - ref) / np.maximum(np.abs(ref), 1.0)))
    out = {"max_rel_strength_error": rel, "strength_rows_compared": int(n), "tolerance": 1e-5,
           "oracle_s": round(dt, 2)}
    if rows is None:
        gx, gy = oracle.sobel_f32(oracle.gauss_f32(crop))
        amb = float_ambiguous(gx, gy, M)
        got_e = d_out.cpu().numpy()
        out.update({"pixels_differing": int((got_e != e).sum()), "pixels_ambiguous": int(amb.sum()),
                    "pixels": int(e.size)})
    return out

def oracle_sample(img: np.ndarray, rows: int) -> tuple[float, str]:
    """Time the oracle on the first `rows` rows of the image; returns (Mpixel/s, description)."""
    import oracle
    sample = np.ascontiguousarray(img[:rows])
    t0 = time.perf_counter()
    oracle.canny_u8(sample, LOW, HIGH)
    dt = time.perf_counter() - t0
    return sample.size / dt / 1e6, f"rows 0..{rows} of the {W}x{H} image ({sample.size / 1e6:.1f} Mpixel), 1 thread"


def oracle_images_parallel(imgs: list) -> tuple:
    """The oracle once per image, one image per thread on every host core (the
    images are independent; the ctypes call releases the GIL)."""
    import concurrent.futures as cf

    import oracle
    cores = os.cpu_count() or 1
    oracle.lib()
    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(max_workers=cores) as ex:
        outs = list(ex.map(lambda im: oracle.canny_u8(im, LOW, HIGH), imgs))
    dt = time.perf_counter() - t0
    px = sum(im.size for im in imgs)
    return {"value": round(px / dt / 1e6, 1), "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"all {len(imgs)} images ({px / 1e6:.1f} Mpixel), one image per thread",
            **cpu_info()}, outs


def run_reference(args, rank: int, world: int) -> None:
    if rank != 0:
        return
    from paper_1710_07745_gb300 import synth
    rows = int(os.environ.get("CANNY_REF_ROWS", "2048"))
    img = np.empty((rows, W), np.uint8)
    full = synth.image(SEED, W, H, N_OBJ, N_OBJ, NOISE)
    img[:] = full[:rows]
    del full
    for _ in range(args.warmup):
        oracle_sample(img, rows)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle_sample(img, rows)
        times.append(time.perf_counter() - t0)
    tot = sum(times)
    value = args.steps * img.size / tot / 1e6
    sample = f"rows 0..{rows} of the {W}x{H} image ({img.size / 1e6:.1f} Mpixel) per step, 1 thread"
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 3), "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(1e3 * tot / args.steps, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": config({"sample_rows": rows}),
            "cpu_baseline": {"value": round(value, 3), "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": round(value, 3), "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ batched vs per-image loop
BATCH_N, BATCH_LO, BATCH_HI, BATCH_SEED = 1024, 64, 2048, 4000


def measure_batched(steps: int, cpu: bool = False) -> dict:
    """1024 images, sides log-uniform in [64, 2048]: one canny_run_batch call (a
    persistent graph-captured launch over all images' units) against a loop of
    canny_run_pitched calls on the same stream, inputs resident; outputs compared."""
    import concurrent.futures as cf
    import ctypes

    import torch

    from paper_1710_07745_gb300 import canny, synth

    ws, hs = synth.batch_sizes(BATCH_N, BATCH_LO, BATCH_HI, BATCH_SEED)
    with cf.ThreadPoolExecutor(max_workers=min(32, os.cpu_count() or 4)) as ex:
        imgs = list(ex.map(lambda i: synth.batch_image(i, int(ws[i]), int(hs[i]), BATCH_SEED), range(BATCH_N)))
    total = int(sum(int(w) * int(h) for w, h in zip(ws, hs)))
    ins = [torch.from_numpy(im).cuda() for im in imgs]
    outs_b = [torch.empty_like(x) for x in ins]
    outs_l = [torch.empty_like(x) for x in ins]
    lib = canny.load()
    sp = torch.cuda.current_stream().cuda_stream
    ctx = canny.Canny(total, 1, low=LOW, high=HIGH)
    arr_b = (canny.canny_image * BATCH_N)(*[canny.image_of(a, b) for a, b in zip(ins, outs_b)])
    arr_l = [canny.image_of(a, b) for a, b in zip(ins, outs_l)]
    tune = canny.canny_autotune_batch(ctx.ctx, list(arr_b), sp,
                                      os.path.join(os.path.expanduser("~"), ".cache", "canny_gb300_tune.jsonl")
                                      if os.access(os.path.expanduser("~"), os.W_OK) else None).as_dict()
    # the loop keeps the single-image default (64-row bands), its faster setting for
    # images this small; the batch's tuned band would shrink its grids
    loop_ctx = canny.Canny(BATCH_HI, BATCH_HI, low=LOW, high=HIGH)

    def run_batch():
        rc = lib.canny_run_batch(ctx.ctx, BATCH_N, arr_b, sp)
        if rc:
            raise canny.CannyError(rc, "canny_run_batch")

    def run_loop():
        for im in arr_l:
            rc = lib.canny_run_pitched(loop_ctx.ctx, ctypes.byref(im), sp)
            if rc:
                raise canny.CannyError(rc, "canny_run_pitched")

    res = {}
    for name, fn in (("batch", run_batch), ("loop", run_loop)):
        for _ in range(2):
            fn()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        res[name] = e0.elapsed_time(e1) / steps
    same = all(torch.equal(a, b) for a, b in zip(outs_b, outs_l))
    ctx.close()
    loop_ctx.close()
    cpu_line, matches = None, None
    if cpu:
        cpu_line, want = oracle_images_parallel(imgs)
        matches = all(np.array_equal(o.cpu().numpy(), wnt) for o, wnt in zip(outs_b, want))
    return {"images": BATCH_N, "sides": [BATCH_LO, BATCH_HI], "pixels": total,
            "batch_ms": round(res["batch"], 4), "loop_ms": round(res["loop"], 4),
            "batch_mpx_s": round(total / res["batch"] / 1e3, 1), "loop_mpx_s": round(total / res["loop"] / 1e3, 1),
            "speedup": round(res["loop"] / res["batch"], 2), "outputs_identical": bool(same),
            "matches_oracle": matches,
            "tuning": {k: tune[k] for k in ("band", "ctas_per_sm", "direct_loads", "chase_budget", "batch_passes",
                                            "from_cache")},
            "cpu_baseline": cpu_line}


# ------------------------------------------------------------------ host link
def host_link_bound(h_in, h_out, d_a, d_b, px: int) -> dict:
    """The host link's own rate, for the end-to-end roofline: plain copies of one
    step's bytes between the pinned buffers and device memory, each direction
    alone and both at once on two streams (best of three timed trials)."""
    import torch
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()

    def timed(fn, reps=5, trials=3):
        # best of a few trials: the link is shared with the host's other work
        for _ in range(2):
            fn()
        torch.cuda.synchronize()
        best = float("inf")
        for _ in range(trials):
            t0 = time.perf_counter()
            for _ in range(reps):
                fn()
            torch.cuda.synchronize()
            best = min(best, (time.perf_counter() - t0) / reps)
        return best

    def h2d():
        with torch.cuda.stream(s1):
            d_a.copy_(h_in, non_blocking=True)

    def d2h():
        with torch.cuda.stream(s2):
            h_out.copy_(d_b, non_blocking=True)

    def both():
        h2d()
        d2h()

    t_h2d, t_d2h, t_both = timed(h2d), timed(d2h), timed(both)
    nbytes = h_in.numel()
    return {"h2d_gbs": round(nbytes / t_h2d / 1e9, 1), "d2h_gbs": round(nbytes / t_d2h / 1e9, 1),
            "both_gbs": round(2 * nbytes / t_both / 1e9, 1),
            "bound_mpx_s": round(px / t_both / 1e6, 1)}


# ------------------------------------------------------------------ the other image sizes
def measure_configs(cpu: bool = False) -> list:
    """Per-image pipeline times on the smaller synthetic workloads: each run timed
    alone with CUDA events (median), stage averages from the library's own events.
    These images fit in the 129 MB L2 except 7680 x 4320 (66 MB in + out: mostly).
    cpu: also the oracle on each image (single thread, median of 3) and, for the
    float variant, its error against the oracle."""
    import torch

    from paper_1710_07745_gb300 import canny, synth

    cases = [("canny_int_512x512", synth.small, canny.CANNY_PATH_INT, 100),
             ("canny_int_4096x4096", synth.medium, canny.CANNY_PATH_INT, 50),
             ("canny_f32_4096x4096", synth.medium, canny.CANNY_PATH_F32, 50),
             ("canny_int_7680x4320", synth.uhd, canny.CANNY_PATH_INT, 50)]
    stream = torch.cuda.current_stream()
    sp = stream.cuda_stream
    out = []
    for name, gen, path, n in cases:
        img = gen()
        h, w = img.shape
        d_in = torch.from_numpy(img).cuda()
        d_out = torch.empty_like(d_in)
        if path == canny.CANNY_PATH_INT:
            ctx = canny.Canny(w, h, low=LOW, high=HIGH)
        else:
            ctx = canny.Canny(w, h, path=path, low=0.1, high=0.3, sigma=1.4, ksize=7)
        for _ in range(10):
            canny.canny_run(ctx.ctx, d_in.data_ptr(), d_out.data_ptr(), sp)
        torch.cuda.synchronize()
        canny.canny_enable_timing(ctx.ctx, True)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n)]
        for e0, e1 in ev:
            e0.record(stream)
            canny.canny_run(ctx.ctx, d_in.data_ptr(), d_out.data_ptr(), sp)
            e1.record(stream)
        torch.cuda.synchronize()
        tm = canny.canny_read_timing(ctx.ctx).as_dict()
        canny.canny_enable_timing(ctx.ctx, False)
        st = ctx.stats()
        ms = statistics.median(e0.elapsed_time(e1) for e0, e1 in ev)
        runs = max(1, tm["runs"])
        entry = {"workload": name, "w": w, "h": h, "runs": n, "median_ms": round(ms, 4),
                 "mpx_s": round(w * h / ms / 1e3, 1),
                 "stencil_ms": round(tm["stencil_ms"] / runs, 4),
                 "local_ms": round(tm["local_ms"] / runs, 4),
                 "global_ms": round(tm["global_ms"] / runs, 4),
                 "hyst_passes": int(st["hyst_passes"]), "pending_tiles": int(st["pending_tiles"]),
                 "tiles_visited": int(st["hyst_tiles_visited"])}
        if cpu:
            import oracle
            if path == canny.CANNY_PATH_INT:
                t = oracle_median(lambda: oracle.canny_u8(img, LOW, HIGH))
            else:
                t = oracle_median(lambda: oracle.canny_f32(img))
                entry["vs_oracle"] = float_error(img, d_in, d_out, ctx)
            entry["cpu_baseline"] = {"value": round(w * h / t / 1e6, 3), "unit": UNIT, "cores": 1, "kind": "oracle",
                                     "sample": "the whole image, median of 3 single-thread runs", **cpu_info()}
        out.append(entry)
        ctx.close()
        del d_in, d_out
    return out


def measure_float_on(d_in, d_out, name: str, n: int, img: np.ndarray | None = None) -> dict:
    """The float32 variant (sigma 1.4, 7 taps, thresholds 0.1 / 0.3 of the largest
    strength) on an image already on the device: n runs timed with CUDA events.
    img: also the production kernel's strength error against the oracle on its
    first 1024 rows."""
    import torch

    from paper_1710_07745_gb300 import canny

    h, w = d_in.shape
    stream = torch.cuda.current_stream()
    sp = stream.cuda_stream
    ctx = canny.Canny(w, h, path=canny.CANNY_PATH_F32, low=0.1, high=0.3, sigma=1.4, ksize=7)
    for _ in range(3):
        canny.canny_run(ctx.ctx, d_in.data_ptr(), d_out.data_ptr(), sp)
    torch.cuda.synchronize()
    canny.canny_enable_timing(ctx.ctx, True)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(n):
        canny.canny_run(ctx.ctx, d_in.data_ptr(), d_out.data_ptr(), sp)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / n
    tm = canny.canny_read_timing(ctx.ctx).as_dict()
    canny.canny_enable_timing(ctx.ctx, False)
    st = ctx.stats()
    runs = max(1, tm["runs"])
    entry = {"workload": name, "w": w, "h": h, "runs": n, "mean_ms": round(ms, 4),
             "mpx_s": round(w * h / ms / 1e3, 1), "stencil_ms": round(tm["stencil_ms"] / runs, 4),
             "global_ms": round(tm["global_ms"] / runs, 4), "hyst_passes": int(st["hyst_passes"]),
             "pending_tiles": int(st["pending_tiles"]), "tiles_visited": int(st["hyst_tiles_visited"])}
    if img is not None:
        entry["vs_oracle"] = float_error(img, d_in, d_out, ctx, rows=1024)
    ctx.close()
    return entry


# ------------------------------------------------------------------ long weak chains
def serpentine(n: int, gap: int = 32) -> np.ndarray:
    """Class map of one weak path through every 32 x 32 tile of an n x n image:
    horizontal runs every `gap` rows joined at alternate ends, strong only at its
    start (the adversarial case for hysteresis)."""
    cls = np.zeros((n, n), np.uint8)
    rows = list(range(gap // 2, n, gap))
    for j, r in enumerate(rows):
        cls[r, :] = 1
        if j + 1 < len(rows):
            c = n - 1 if j % 2 == 0 else 0
            cls[r:rows[j + 1] + 1, c] = 1
    cls[rows[0], 0] = 2
    return cls


def measure_chains(tile_counts=(256, 1024, 4096, 16384), runs: int = 5) -> list:
    """Global hysteresis time and passes against the length of one weak chain
    (a serpentine through every tile), through canny_hysteresis on a class map."""
    import torch

    from paper_1710_07745_gb300 import canny
    out = []
    sp = torch.cuda.current_stream().cuda_stream
    for tiles in tile_counts:
        n = 32 * int(round(tiles ** 0.5))
        cls = serpentine(n)
        d_in = torch.from_numpy(cls).cuda()
        d_out = torch.empty_like(d_in)
        with canny.Canny(n, n) as c:
            img = canny.image_of(d_in, d_out)
            for _ in range(2):
                canny.canny_hysteresis(c.ctx, img, sp)
            torch.cuda.synchronize()
            canny.canny_enable_timing(c.ctx, True)
            for _ in range(runs):
                canny.canny_hysteresis(c.ctx, img, sp)
            torch.cuda.synchronize()
            tm = canny.canny_read_timing(c.ctx).as_dict()
            canny.canny_enable_timing(c.ctx, False)
            st = c.stats()
            reached = int((d_out == 255).sum().item())
        out.append({"tiles": tiles, "chain_pixels": int((cls > 0).sum()), "reached": reached,
                    "global_ms": round(tm["global_ms"] / max(1, tm["runs"]), 4),
                    "hyst_passes": int(st["hyst_passes"]), "tiles_visited": int(st["hyst_tiles_visited"])})
    return out


# ------------------------------------------------------------------ serving
SERVE_POOL, SERVE_LO, SERVE_HI, SERVE_SEED = 256, 128, 4096, 5000


def measure_serving(n_requests: int, loads=(0.1, 0.25, 0.5, 0.9, 1.5), budget_gb: float = 16.0, streams: int = 8,
                    max_trace_s: float = 10.0) -> dict:
    """Continuous-batching server on Poisson arrivals, sides log-uniform in [128, 4096].

    Request i carries image i mod 256 of a seeded pool (the sizes follow the stated
    distribution; the pixels repeat). Capacity is measured first with every request
    arriving at once (median of three runs); the offered loads are fractions of it (above 1: overload, the
    queue grows). Each load's trace has n_requests requests, or fewer when that
    would span more than max_trace_s seconds of arrivals (at least 5000). The
    serial baseline (one canny_run_pitched at a time) runs the second load's trace
    on its first 5000 requests."""
    import concurrent.futures as cf

    import torch

    from paper_1710_07745_gb300 import canny, synth

    ws, hs = synth.log_uniform_sizes(SERVE_SEED, SERVE_POOL, SERVE_LO, SERVE_HI)
    with cf.ThreadPoolExecutor(max_workers=min(32, os.cpu_count() or 4)) as ex:
        pool = list(ex.map(lambda i: synth.batch_image(i, int(ws[i]), int(hs[i]), SERVE_SEED), range(SERVE_POOL)))
    pinned = [torch.from_numpy(im).pin_memory() for im in pool]
    areas = np.array([im.size for im in pool], np.float64)
    mean_area = float(areas.mean())

    def trace(n, rate, seed):
        t = synth.poisson_arrivals(seed, n, rate) if rate else np.zeros(n)
        return [canny.canny_request(int(ws[i % SERVE_POOL]), int(hs[i % SERVE_POOL]),
                                    pinned[i % SERVE_POOL].data_ptr(), int(ws[i % SERVE_POOL]), None, 0,
                                    float(t[i] - t[0]) if rate else 0.0) for i in range(n)]

    def cfg(serial):
        # at most 64 Mpixel a batch on 8 streams: smaller batches on more streams
        # overlap one batch's upload with others' kernels (all-at-once capacity
        # 180 Gpixel/s, against 155 on 6 streams and 140 on 4)
        return canny.canny_serve_config(budget_gb * 2 ** 30, streams, 4096, 64 << 20, serial, LOW, HIGH, 0, 0)

    def summary(rep, offered=None):
        d = rep.as_dict()
        out = {"delivered_mpx_s": round(d["delivered_mpx_s"], 1), "p50_ms": round(d["p50_ms"], 3),
               "p99_ms": round(d["p99_ms"], 3), "max_ms": round(d["max_ms"], 3),
               "mean_batch_images": round(d["mean_batch_images"], 1), "peak_gb": round(d["peak_bytes"] / 2 ** 30, 2)}
        if offered is not None:
            out["offered_mpx_s"] = round(offered, 1)
        return out

    # capacity: median of three all-at-once runs (one run alone varied by up to 15 %)
    caps = sorted(canny.canny_serve(cfg(0), trace(min(n_requests, 20000), 0.0, 1)).delivered_mpx_s for _ in range(3))
    capacity = caps[1]                                 # Mpixel/s
    result = {"requests": n_requests, "sides": [SERVE_LO, SERVE_HI], "budget_gb": budget_gb, "streams": streams,
              "max_batch_mpixel": 64,
              "pool_images": SERVE_POOL, "capacity_mpx_s": round(capacity, 1), "loads": []}
    for k, load in enumerate(loads):
        rate = load * capacity * 1e6 / mean_area        # requests per second
        n = min(n_requests, max(5000, int(max_trace_s * rate)))
        rep = canny.canny_serve(cfg(0), trace(n, rate, 10 + k))
        entry = summary(rep, load * capacity)
        entry["load"] = load
        entry["requests"] = n
        result["loads"].append(entry)
    ls = loads[min(1, len(loads) - 1)]
    rate = ls * capacity * 1e6 / mean_area
    ser = canny.canny_serve(cfg(1), trace(min(n_requests, 5000), rate, 10 + min(1, len(loads) - 1)))
    result["serial"] = dict(summary(ser, ls * capacity), load=ls, requests=min(n_requests, 5000))
    # capacity of the serial loop (one canny_run_pitched per request, all arriving at once)
    ser_cap = canny.canny_serve(cfg(1), trace(min(n_requests, 5000), 0.0, 1)).delivered_mpx_s
    result["serial_capacity_mpx_s"] = round(ser_cap, 1)
    result["capacity_vs_serial"] = round(capacity / ser_cap, 2) if ser_cap > 0 else None
    return result


# ------------------------------------------------------------------ our arm
def run_ours(args, rank: int, world: int) -> None:
    import torch

    from paper_1710_07745_gb300 import canny, synth

    global W, H, N_OBJ, WORKLOAD
    if args.size:
        W, H = (int(v) for v in args.size.lower().split("x"))
        N_OBJ = synth.objects_for_area(W, H)
    if args.size or args.path != "int":
        WORKLOAD = f"canny_{args.path}_{W}x{H}"
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    peaks = measured_peaks()
    img = synth.image(SEED, W, H, N_OBJ, N_OBJ, NOISE)
    d_in = torch.from_numpy(img).cuda()
    d_out = torch.empty_like(d_in)
    stream = torch.cuda.current_stream()
    sp = stream.cuda_stream
    if args.path == "int":
        ctx = canny.Canny(W, H, low=LOW, high=HIGH)
    else:   # float32 variant (profiling runs): sigma 1.4, 7 taps, thresholds 0.1 / 0.3 of the largest strength
        ctx = canny.Canny(W, H, path=canny.CANNY_PATH_F32, low=0.1, high=0.3, sigma=1.4, ksize=7)

    for _ in range(max(3, args.warmup)):
        ctx.run(d_in, d_out, stream)
    torch.cuda.synchronize()
    st = ctx.stats()
    if st["status"] != canny.CANNY_OK:
        raise RuntimeError(f"pipeline status {st['status']}")
    passes = int(st["hyst_passes"])

    canny.canny_enable_timing(ctx.ctx, True)
    clocks = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    if clocks:
        clocks.start()
        time.sleep(0.3)
    barrier(world)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        canny.canny_run(ctx.ctx, d_in.data_ptr(), d_out.data_ptr(), sp)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    ms = e0.elapsed_time(e1)
    clk = clocks.stop() if clocks else None
    tm = canny.canny_read_timing(ctx.ctx).as_dict()
    canny.canny_enable_timing(ctx.ctx, False)
    ms_max = max_over_ranks(ms, world)

    px = W * H
    value = job_value(world, args.steps, px, ms_max)
    k1_ms = tm["stencil_ms"] / max(1, tm["runs"])
    k1_gbs = K1_BYTES_PER_PX * px / (k1_ms / 1e3) / 1e9
    k3_bytes = k3_traffic(W, H) if args.path == "int" else None
    pipe_bytes = PIPE_BYTES_PER_PX * px + (k3_bytes or 0)
    pipe_gbs = pipe_bytes / (ms / args.steps / 1e3) / 1e9
    stages = {"runs": tm["runs"], "reset_ms": round(tm["reset_ms"] / max(1, tm["runs"]), 4),
              "stencil_ms": round(k1_ms, 4),
              "local_ms": round(tm["local_ms"] / max(1, tm["runs"]), 4),
              "global_ms": round(tm["global_ms"] / max(1, tm["runs"]), 4),
              "hyst_passes": passes, "pending_tiles": int(st["pending_tiles"]),
              "tiles_visited": int(st["hyst_tiles_visited"])}
    dominant = max(("reset_ms", "stencil_ms", "local_ms", "global_ms"), key=lambda k: stages[k])

    e2e = None
    if not args.no_e2e:
        # end to end through the C ABI on pinned host buffers: every step uploads its
        # frame, runs the pipeline and downloads the edge map; canny_run_frames overlaps
        # consecutive steps (upload i+1 / pipeline i / download i-1)
        h_in = [torch.from_numpy(img).pin_memory() for _ in range(2)]
        h_out = [torch.empty_like(h_in[0]).pin_memory() for _ in range(2)]
        # (one call streams all e2e_steps frames: the first upload and the last
        # download are not overlapped, so the rate approaches the link bound as
        # n / (n + 1))
        e2e_steps = max(4, min(args.steps, 40))
        ins = [h_in[i % 2].data_ptr() for i in range(e2e_steps)]
        outs = [h_out[i % 2].data_ptr() for i in range(e2e_steps)]
        canny.canny_run_frames(ctx.ctx, ins[:2], W, outs[:2], W, W, H, sp)      # builds the frame graphs
        barrier(world)
        t0 = time.perf_counter()
        canny.canny_run_frames(ctx.ctx, ins, W, outs, W, W, H, sp)
        e2e_s = max_over_ranks(time.perf_counter() - t0, world)
        ref = d_out[:64].cpu().numpy()
        if not all(np.array_equal(o[:64].numpy(), ref) for o in h_out):
            raise RuntimeError("host-buffer run differs from device run")
        # one call per image (canny_run_host: upload, pipeline, download, no overlap)
        for _ in range(2):
            canny.canny_run_host(ctx.ctx, ins[0], W, outs[0], W, W, H, sp)
        single_steps = max(1, min(args.steps, 5))
        t0 = time.perf_counter()
        for i in range(single_steps):
            canny.canny_run_host(ctx.ctx, ins[i % 2], W, outs[i % 2], W, W, H, sp)
        single_s = max_over_ranks(time.perf_counter() - t0, world)
        e2e = {"value": round(world * e2e_steps * px / e2e_s / 1e6, 1), "unit": UNIT,
               "h2d_bytes_per_step": px, "d2h_bytes_per_step": px, "steps": e2e_steps,
               "api": "canny_run_frames (pinned host buffers)",
               "single_call": {"value": round(world * single_steps * px / single_s / 1e6, 1),
                               "api": "canny_run_host", "steps": single_steps},
               "link_bound": host_link_bound(h_in[0], h_out[0], d_in, d_out, px)}

    do_cpu = rank == 0 and not args.no_cpu
    configs = None if args.no_configs else measure_configs(cpu=do_cpu)
    if configs is not None:
        configs.append(measure_float_on(d_in, d_out, f"canny_f32_{W}x{H}", 10, img if do_cpu else None))
    batched = None if args.no_batch else measure_batched(max(3, min(args.steps, 10)), cpu=do_cpu)
    serving = None if args.no_serve else measure_serving(args.serve_requests)
    chains = None if args.no_configs else measure_chains()
    if rank != 0:
        ctx.close()
        return
    cpu = None
    if not args.no_cpu:
        rows = min(H, int(os.environ.get("CANNY_CPU_ROWS", "4096")))
        cpu_v, cpu_sample = oracle_sample(img, rows)
        cpu = {"value": round(cpu_v, 3), "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": cpu_sample, **cpu_info()}
    line = {
        "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_max / args.steps, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "int32" if args.path == "int" else "f32",
        "data": "synthetic", "config": config({"path": "integer" if args.path == "int" else "float32"}),
        "roofline": {"kernel": "stencil stage: k1_fused_kernel (Gauss/Sobel/NMS/thresholds -> 2-bit class masks) "
                               "+ hyst_fill_kernel (tile-local hysteresis -> edge bytes); 2 B/px algorithmic"
                     if args.path == "int" else
                     "k1f_strength_kernel + k1f_nms_kernel (both stencil passes of the float variant)",
                     "bound": "hbm", "achieved": round(k1_gbs, 1), "peak": peaks["hbm_gbs"],
                     "unit": "GB/s", "frac": round(k1_gbs / peaks["hbm_gbs"], 4),
                     "traffic": k1_traffic(W, H) if args.path == "int" else None,
                     "peak_source": peaks["source"],
                     "bytes_per_launch": K1_BYTES_PER_PX * px},
        "alu_roofline": alu_roofline(px, k1_ms, peaks["hbm_gbs"], clk) if args.path == "int" else None,
        "pipeline_roofline": {"achieved": round(pipe_gbs, 1), "unit": "GB/s",
                              "bytes": pipe_bytes, "basis": f"{PIPE_BYTES_PER_PX} B/px (read the image, write the edge "
                              "map) + the global passes' measured DRAM bytes" + ("" if k3_bytes else
                                                                             " (not recorded for this source: 0)"),
                              "frac": round(pipe_gbs / peaks["hbm_gbs"], 4)},
        "stages": stages, "dominant_stage": dominant,
        "configs": configs,
        "batched": batched,
        "serving": serving,
        "hysteresis_chains": chains,
        "cpu_baseline": cpu,
        "e2e": e2e,
        # per step: the control-block reset, the fused stencil, the tile fill and one
        # cooperative launch that runs every global pass
        "gpu_launches": int(args.steps * 4),
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)
    ctx.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--size", default=None, help="WxH instead of 16384x16384 (profiling runs)")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer leg")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle baseline leg")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-vs-loop leg")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving leg")
    ap.add_argument("--no-configs", action="store_true", help="skip the smaller-image leg")
    ap.add_argument("--path", choices=["int", "f32"], default="int",
                    help="f32: time the float32 variant instead (profiling runs)")
    ap.add_argument("--serve-requests", type=int, default=100000)
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.impl == "reference":
        # the oracle runs on rank 0 alone and exchanges nothing: no process group
        run_reference(args, int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")))
        return
    rank, world = dist_init(args.gpus)
    run_ours(args, rank, world)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
