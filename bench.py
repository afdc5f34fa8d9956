"""Benchmark of the sub-1-spp sampling + reconstruction hot path on GB300.

One step = one frame of the plain method at 1920x1080 (8-frame synthetic
sequence, 0.25 spp, 3-level pyramid, 54/29/25 seeded logits, bilinear
reprojection along affine motion of at most 8 px with 5% disoccluded pixels,
tone map tau + sRGB), through the C ABI:
    spp_alloc_sample_map -> spp_render_synthetic -> spp_splat_samples
    -> spp_reconstruct_level (levels 2, 1, 0; level 0 with the temporal term
       over the previous step's output, and the tone map)
Inputs of all 8 frames are resident in HBM before the timed region (value);
the end-to-end figure (e2e) copies each frame's inputs from pinned host memory
and reads the tone-mapped frame back inside the timed region.

Prints ONE JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle
on the host cores instead (the paper ships no code to compare against).
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

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

WORKLOADS = {
    # name: (W, H, frames, budget, levels)
    "1080p": (1920, 1080, 8, 0.25, 3),
    "4k": (3840, 2160, 4, 0.25, 3),
}
METRIC = "Mpix/s per frame of alloc+splat+reconstruct (plain method)"
UNIT = "Mpix/s"

# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of one level-0
# reconstruction launch on the 1920x1080 workload, from one ncu capture of
# that launch; valid only while the kernel's sources are the ones captured,
# which the hash checks.
LEVEL0_TRAFFIC = {
    "workload": "1080p",
    "bytes_per_launch": 546_309_888,  # median of three captured launches
    "sources": ("paper_2602_08642_gb300/csrc/reconstruct_tma.cu",
                "paper_2602_08642_gb300/csrc/recon_common.cuh",
                "paper_2602_08642_gb300/csrc/spp_internal.cuh"),
    "sha256": "77c46e86595ef9af08362c1c849d2c0d56db33ed2a3145daae4acaee3ca1e294",
}


def level0_traffic(workload: str):
    """Captured traffic per level-0 launch, or None if it does not apply to
    this workload or the kernel changed since the capture."""
    import hashlib
    t = LEVEL0_TRAFFIC
    if workload != t["workload"]:
        return None
    h = hashlib.sha256()
    for f in t["sources"]:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return t["bytes_per_launch"] if h.hexdigest() == t["sha256"] else None


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="1080p")
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--cpu-seconds", type=float, default=16.0,
                    help="bounded CPU work for the oracle baseline (four samples)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-learned", action="store_true",
                    help="skip the learned-vs-plain 4K section")
    ap.add_argument("--learned-size", type=int, default=3840,
                    help="width of the learned-vs-plain frames (height = width * 9 / 16)")
    ap.add_argument("--train-steps", type=int, default=300)
    ap.add_argument("--train-crop", type=int, default=256,
                    help="side of the training crops (batches of 8)")
    ap.add_argument("--learned-frames", type=int, default=LEARNED_FRAMES,
                    help="frames of the learned-vs-plain sequence")
    ap.add_argument("--no-oracle-error", action="store_true",
                    help="skip the comparison of the learned frames with the FP64 oracle")
    ap.add_argument("--frames", type=int, default=0,
                    help="distinct input frames resident on the device (default: the workload's)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", str(rank)))
    return rank, world, local


def slowest_rank_ms(ms_local: float, world: int, device="cpu") -> float:
    """The job's timed region ends with its slowest rank: the maximum over
    the ranks of the local milliseconds (every rank gets it)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms_local], device=device, dtype=torch.float64)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, ms: float) -> float:
    """Units (pixels) processed by all ranks together per second, in millions."""
    return units_per_rank * world / (ms / 1e3) / 1e6


def rank_frame(t: int, rank: int) -> int:
    """Frame index of the seeded streams of rank `rank`'s frame t: every rank
    samples and renders its own frames (weak scaling, no shared data)."""
    return t + rank * 1000


# --------------------------------------------------------------------------
# clocks during the timed region
# --------------------------------------------------------------------------
CLOCK_WINDOW_S = 0.5  # the clocks are read over at least this much of the same load

class ClockSampler:
    FIELDS = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines: list[str] = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def mark(self, name: str):
        setattr(self, name, time.time())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        t0 = getattr(self, "t_start", 0.0)
        # the timed region plus the tail of the same steps that follows it
        t1 = max(getattr(self, "t_end", float("inf")), getattr(self, "t_tail_end", 0.0))
        window = [ln for (t, ln) in self.lines if t0 <= t <= t1 + 0.06]
        if not window:  # no sample in the window: the nearest ones after it
            window = [ln for (t, ln) in self.lines if t >= t0][:2]
        for ln in window:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm),
                "window_s": (t1 - t0) if t1 != float("inf") else None}


# --------------------------------------------------------------------------
# inputs
# --------------------------------------------------------------------------
def make_inputs(W, H, L, frames):
    import spp_inputs as inp
    return [inp.frame_inputs(W, H, L, frame=t, temporal=True) for t in range(frames)]


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def level0_algorithmic_bytes(W, H, mask: np.ndarray) -> int:
    """Compulsory bytes of one full-resolution reconstruction launch: 29
    spatial logits everywhere, 25 temporal logits where the pixel is not
    disoccluded, L^0 (12 B), the warped previous output W_t L_{t-1} (12 B),
    L-hat^1 (12 B per coarse pixel), mask (1 B), HDR + sRGB outputs (24 B)."""
    N = W * H
    unmasked = int(N - int(mask.astype(bool).sum()))
    coarse = (W // 2) * (H // 2)
    return N * (29 * 4 + 12 + 12 + 1 + 24) + unmasked * 25 * 4 + coarse * 12


# --------------------------------------------------------------------------
# the oracle on the host cores (cpu_baseline and --impl reference)
# --------------------------------------------------------------------------
def oracle_inputs(W, H, L):
    """One frame of the workload's inputs for the oracle (FP64 logits, a
    previous output), prepared outside the timed calls."""
    import spp_inputs as inp
    x = inp.frame_inputs(W, H, L, frame=1, temporal=True)
    x["logits64"] = [a.astype(np.float64) for a in x["logits"]]
    return x, np.random.default_rng(1).random((3, H, W))


def oracle_frame_seconds(W, H, L, B, x, prev):
    import oracle
    t0 = time.perf_counter()
    oracle.frame(x["d"], x["clean"], x["logits64"], W, H, L, B, prev=prev, mv=x["mv"],
                 mask=x["mask"], frame_index=1)
    return time.perf_counter() - t0


def cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    import platform
    return platform.processor() or platform.machine()


def cpu_sample(W, H, L, B, budget_s, threads=1):
    """Runs the oracle on band crops of the workload's frame (full width,
    H/8 rows, same per-pixel work) on `threads` host threads until budget_s
    of wall time is spent."""
    import oracle
    oracle.set_threads(threads)
    Hs = max(H // 8 // (1 << (L - 1)) * (1 << (L - 1)), 1 << (L - 1))
    x, prev = oracle_inputs(W, Hs, L)
    spent, pix = 0.0, 0
    while spent < budget_s:
        spent += oracle_frame_seconds(W, Hs, L, B, x, prev)
        pix += W * Hs
    n = oracle.get_threads()
    return pix / spent / 1e6, n, (f"oracle frames of {W}x{Hs} (full-width band of the {W}x{H} "
                                  f"workload), {pix // (W * Hs)} runs, {spent:.1f} s, {n} "
                                  f"thread{'s' if n > 1 else ''}")


def cpu_baseline(W, H, L, B, budget_s):
    """The oracle on the host cores: all of them (OpenMP over rows) and one,
    on the workload's frame and on the 4K frame of the same method."""
    import oracle
    oracle.build()
    ncores = os.cpu_count() or 1
    share = budget_s / 4
    v_all, n_all, s_all = cpu_sample(W, H, L, B, share, threads=ncores)
    v_one, _, s_one = cpu_sample(W, H, L, B, share, threads=1)
    W4, H4, _, B4, L4 = WORKLOADS["4k"]
    v4_all, _, s4_all = cpu_sample(W4, H4, L4, B4, share, threads=ncores)
    v4_one, _, s4_one = cpu_sample(W4, H4, L4, B4, share, threads=1)
    oracle.set_threads(0)
    return {"value": v_all, "unit": UNIT, "cores": n_all, "kind": "oracle", "sample": s_all,
            "cpu_model": cpu_model(), "nproc": ncores,
            "single_thread": {"value": v_one, "cores": 1, "sample": s_one},
            "4k": {"all_cores": {"value": v4_all, "cores": n_all, "sample": s4_all},
                   "single_thread": {"value": v4_one, "cores": 1, "sample": s4_one}}}


REFERENCE_SECONDS = 90.0  # about this much CPU time for the timed reference steps
REFERENCE_MIN_ROWS = 32   # a band small enough to make per-call overhead count is not run


def reference_band_rows(W, H, L, steps, seconds_per_pixel, target_s=REFERENCE_SECONDS):
    """Rows of the full-width band one reference step runs: as many as let
    `steps` steps take about target_s, a multiple of 2^(L-1) (one block of the
    coarsest level), between REFERENCE_MIN_ROWS (or H/8 if smaller) and H/8."""
    q = 1 << (L - 1)
    hmax = max(H // 8 // q * q, q)
    hmin = min(max(REFERENCE_MIN_ROWS // q * q, q), hmax)
    rows = int(target_s / max(steps, 1) / (seconds_per_pixel * W))
    return min(max(rows // q * q, hmin), hmax)


def run_reference(args, rank, world):
    W, H, F, B, L = WORKLOADS[args.workload]
    if rank != 0:
        return
    import oracle
    oracle.build()
    oracle.set_threads(0)  # every host core (OpenMP over rows)
    ncores = oracle.get_threads()
    # one calibration frame on the largest band sets the band of the steps
    Hs = max(H // 8 // (1 << (L - 1)) * (1 << (L - 1)), 1 << (L - 1))
    x, prev = oracle_inputs(W, Hs, L)
    per_pixel = oracle_frame_seconds(W, Hs, L, B, x, prev) / (W * Hs)
    rows = reference_band_rows(W, H, L, args.steps, per_pixel)
    if rows != Hs:
        Hs = rows
        x, prev = oracle_inputs(W, Hs, L)
    for _ in range(args.warmup):
        oracle_frame_seconds(W, Hs, L, B, x, prev)
    t = [oracle_frame_seconds(W, Hs, L, B, x, prev) for _ in range(args.steps)]
    total = sum(t)
    value = W * Hs * args.steps / total / 1e6
    sample = (f"each step one oracle frame of a {W}x{Hs} full-width band of the {W}x{H} "
              f"workload (same per-pixel work), FP64, {ncores} threads (OpenMP over rows)")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": workload_config(args.workload),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": ncores, "kind": "oracle",
                         "sample": sample, "cpu_model": cpu_model()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def workload_config(name):
    W, H, F, B, L = WORKLOADS[name]
    return {"workload": f"plain method {W}x{H}, {F}-frame sequence, {B} spp, {L}-level pyramid, "
                        f"54/29/25 seeded logits, bilinear reprojection (|mv| <= 8 px, 5% "
                        f"disoccluded), tone map tau + sRGB",
            "W": W, "H": H, "frames": F, "spp": B, "levels": L,
            "l2": "inputs larger than L2 (about 0.8 GB read per frame vs 129 MB L2)"}


# --------------------------------------------------------------------------
# our arm
# --------------------------------------------------------------------------
def run_ours(args, rank, world, local):
    import torch
    import torch.distributed as dist

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import paper_2602_08642_gb300 as spp
    from paper_2602_08642_gb300 import _binding as Bnd

    W, H, F, B, L = WORKLOADS[args.workload]
    if args.frames > 0:
        F = args.frames
    N = W * H
    dev = torch.device("cuda", local)
    host_inputs = make_inputs(W, H, L, F)
    stream = torch.cuda.current_stream()

    def to_dev(a):
        return torch.from_numpy(np.ascontiguousarray(a)).to(dev)

    frames = []
    for x in host_inputs:
        frames.append(dict(d=to_dev(x["d"]), clean=to_dev(x["clean"]),
                           logits=[to_dev(a) for a in x["logits"]], mv=to_dev(x["mv"]),
                           mask=to_dev(x["mask"])))
    fr = spp.Frame(W, H, L, max_budget=B, device=dev)
    tm = spp.make_tonemap()
    hats = [None] + [torch.empty((3, H >> l, W >> l), device=dev) for l in range(1, L)]
    warped = torch.empty((3, H, W), device=dev)
    state = {"prev": None, "parity": 0}
    ev_l0 = []
    # W_t L_{t-1} needs only the previous output and the motion: it runs on a
    # side stream, overlapping the sampling and the coarse levels, and level 0
    # waits for it
    side = torch.cuda.Stream(device=dev)
    ev_prev = torch.cuda.Event()
    ev_warp = torch.cuda.Event()

    def step(k, timed_l0=False, inp=None):
        t = k % F
        x = inp if inp is not None else frames[t]
        prev = state["prev"]
        if prev is not None:  # the first frame of the run has no previous output
            ev_prev.record(stream)
            side.wait_event(ev_prev)
            Bnd.check(spp.spp_warp_previous(prev, x["mv"], W, H, warped, stream=side), "warp")
            ev_warp.record(side)
        params = spp.make_params(B, frame=rank_frame(t, rank))
        fr.alloc(x["d"], params)
        fr.render(x["clean"], 0xC0FFEE + rank, t)
        fr.splat()
        for l in range(L - 1, 0, -1):
            C = 25 if l == L - 1 else 29
            Bnd.check(spp.spp_reconstruct_level(
                fr.layers[l], x["logits"][l], C, hats[l + 1] if l + 1 < L else None, None, None,
                W >> l, H >> l, None, hats[l], None, status=fr.status), "level")
        out = fr.hdr[state["parity"]]
        if prev is not None:
            stream.wait_event(ev_warp)
        if timed_l0:
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
        Bnd.check(spp.spp_reconstruct_level(fr.layers[0], x["logits"][0], 54, hats[1],
                                            warped if prev is not None else None,
                                            x["mask"] if prev is not None else None, W, H, tm, out,
                                            fr.ldr, status=fr.status), "level 0")
        if timed_l0:
            e1.record(stream)
            ev_l0.append((e0, e1))
        state["prev"] = out
        state["parity"] ^= 1
        return out

    fr.clear_status()
    for k in range(max(args.warmup, 3)):
        step(k)
    torch.cuda.synchronize()
    fr.check_status()

    clocks = ClockSampler(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    launches0 = spp.spp_launch_count()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    clocks.mark("t_start")
    t0.record(stream)
    for k in range(args.steps):
        step(args.warmup + k, timed_l0=True)
    t1.record(stream)
    torch.cuda.synchronize()
    clocks.mark("t_end")
    launches = spp.spp_launch_count() - launches0
    # a timed region shorter than the sampler's period holds no clock sample
    # of its own: the same steps keep running, untimed, until CLOCK_WINDOW_S
    # have passed since it began, and the clocks are read over both
    k = args.warmup + args.steps
    while time.time() - clocks.t_start < CLOCK_WINDOW_S:
        for _ in range(16):
            step(k)
            k += 1
        torch.cuda.synchronize()
    clocks.mark("t_tail_end")
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    ms = t0.elapsed_time(t1)
    fr.check_status()
    ms_max = slowest_rank_ms(ms, world, dev)
    value = whole_job_rate(N * args.steps, world, ms_max)

    l0_ms = [a.elapsed_time(b) for a, b in ev_l0]
    l0_avg = sum(l0_ms) / len(l0_ms)
    masks = [x["mask"] for x in host_inputs]
    l0_bytes = sum(level0_algorithmic_bytes(W, H, masks[(args.warmup + k) % F])
                   for k in range(args.steps)) / args.steps
    peaks, peak_kind = measured_peaks()
    achieved = l0_bytes / (l0_avg / 1e3) / 1e9
    roofline = {"bound": "hbm", "kernel": "recon_tma_kernel<54,UP,TEMP,TONE,3> (level 0)",
                "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / peaks["hbm_gbs"], "peak_kind": peak_kind,
                "traffic": level0_traffic(args.workload),
                "algorithmic_bytes_per_launch": l0_bytes,
                "avg_launch_ms": l0_avg,
                "share_of_step": l0_avg * args.steps / ms}

    # end to end: host inputs -> device -> frame -> tone-mapped frame on host
    e2e = run_e2e(args, spp, Bnd, fr, host_inputs, step, dev, stream, W, H, L, F, world, dist)

    learned = None
    if not args.no_learned:
        learned = run_learned(args, spp, Bnd, dev, rank)

    cpu = None
    if rank == 0 and not args.no_cpu_baseline and world == 1:
        cpu = cpu_baseline(W, H, L, B, args.cpu_seconds)
    if learned is not None:
        crops = learned.pop("_oracle_crops")
        if rank == 0 and not args.no_oracle_error:
            learned["error_vs_fp64_oracle"] = oracle_crop_errors(crops)
        del crops

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": workload_config(args.workload),
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk,
            "gpu_launches": launches,
            "samples_per_frame": int(fr.sample_count()),
            "learned_vs_plain": learned,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


LEARNED_FRAMES = 16     # the 4K sequence of the learned-vs-plain comparison
ORACLE_CROP = 256       # side of the region of each frame compared with the FP64 oracle
ORACLE_MARGIN = 48      # context around it: the network's receptive field (about 25 px)
                        # plus the reconstruction's footprint over the levels (about 8 px)


def make_scene_frames(W, H, F, seed=3):
    """Clean image and G-buffer of frames 0..F-1 of one drifting procedural
    scene, generated on host threads (numpy releases the interpreter lock)."""
    from concurrent.futures import ThreadPoolExecutor

    import spp_inputs as inp
    with ThreadPoolExecutor(max(1, min(F, os.cpu_count() or 1))) as ex:
        return list(ex.map(lambda t: inp.scene(W, H, seed=seed, frame=t), range(F)))


def crop_window(W, H):
    """Origin (x0, y0) of the compared window (side ORACLE_CROP + 2 margins)
    at the centre of the frame, on a multiple of 4 so that its pyramid
    levels line up with the frame's."""
    side = ORACLE_CROP + 2 * ORACLE_MARGIN
    return (W - side) // 2 // 4 * 4, (H - side) // 2 // 4 * 4, side


def run_learned(args, spp, Bnd, dev, rank):
    """Learned (BF16 tensor-core network + FP32 reconstruction) against the
    plain method (uniform density, fixed kernels) on the same frames of a
    16-frame 4K sequence, at 0.125 / 0.25 / 0.5 spp: per-frame time and
    PSNR in tone-mapped sRGB against the clean image and against the 64-spp
    mean of the renderer stand-in.  The network is first trained on the GPU
    by the library's own kernels: batches of 8 two-frame 256 x 256 crops at
    0.25 spp, the loss against the 64-spp reference.  The crops for the
    error against the FP64 oracle are kept (evaluated after all timing)."""
    import torch

    import spp_inputs as inp
    from paper_2602_08642_gb300 import learned as Lm

    W = args.learned_size
    H = W * 9 // 16 // 4 * 4
    F = args.learned_frames
    crop = args.train_crop
    # training: batch 8 of crop x crop two-frame samples, 0.25 spp, 64-spp target
    seeds = [100 + i + 1000 * rank for i in range(32)]
    train = [Lm.FrameData(inp.training_pair(crop, seed=sd), seed=sd) for sd in seeds]
    for x in train:  # the references are pre-rendered, as the paper's are
        x.reference("spp64")
        x.reference("spp64", prev=True)
    theta0 = torch.from_numpy(inp.unet_params(Lm.layer_table(), seed=5,
                                              head_bias=inp.fixed_head_bias()))
    tr = Lm.Trainer(theta0, 8, crop, 0.25, lr=1e-3, reference="spp64")
    rng = np.random.default_rng(rank)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    losses = []
    for k in range(args.train_steps):
        idx = rng.choice(len(train), 8, replace=False)
        losses.append(tr.step([train[i] for i in idx], seed=1000 + 17 * k))
    torch.cuda.synchronize()
    train_ms = (time.perf_counter() - t0) * 1e3 / max(args.train_steps, 1)
    theta = tr.net.theta
    del tr, train

    # the sequence: F frames of one scene drifting (1.5, -0.75) px per frame
    scenes = make_scene_frames(W, H, F)
    frames = []
    for t, (clean, gb) in enumerate(scenes):
        c = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)  # noqa: E731
        frames.append(dict(clean=c(clean), albedo=c(gb["albedo"]), normal=c(gb["normal"]),
                           depth=c(gb["depth"]), mv=c(inp.scene_motion(W, H, t))))
    fixed = [torch.from_numpy(a).to(dev) for a in inp.fixed_logits(W, H, 3, True)]
    tm = spp.make_tonemap()
    refs, refs64 = [], []
    for t, x in enumerate(frames):
        r = torch.empty((3, H, W), device=dev)
        Bnd.check(Bnd.spp_tonemap_image(x["clean"], W, H, tm, r), "tonemap")
        refs.append(r)
        hdr64 = Lm.render_reference(x["clean"], seed=0x64000000 + t, frame=t)
        r64 = torch.empty((3, H, W), device=dev)
        Bnd.check(Bnd.spp_tonemap_image(hdr64, W, H, tm, r64), "tonemap")
        refs64.append(r64)
        del hdr64
    Lm._REF_FRAMES.clear()
    net = Lm.Predictor(theta, 1, W, H)
    ones = torch.ones((H, W), device=dev)
    mask = torch.zeros((H, W), dtype=torch.uint8, device=dev)
    warped = torch.empty((3, H, W), device=dev)
    prev_ldr = torch.empty((3, H, W), device=dev)
    hats = [None] + [torch.empty((3, H >> l, W >> l), device=dev) for l in range(1, 3)]
    # per frame: MSE against the clean image and against the 64-spp mean
    # (each value in a 16-byte slot)
    mse = torch.zeros(F * 2 * 2, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()
    flops = Lm.flops_per_frame(W, H)
    peaks, peak_kind = measured_peaks()
    x0, y0, side = crop_window(W, H)
    out = {"workload": f"{W}x{H} sequence of {F} frames of one drifting procedural scene, "
                       f"3-level pyramid, temporal term with true motion, tone map tau + sRGB; "
                       f"learned = feature assembly + BF16 tensor-core U-Net + density softmax "
                       f"+ the plain path; plain = uniform density and fixed kernels (kd = "
                       f"-r^2/2, ku = kt = 0); each form runs the sequence once untimed, then "
                       f"once timed frame by frame (CUDA events around each frame)",
           "training": {"steps": args.train_steps, "crop": crop, "batch": 8, "spp": 0.25,
                        "reference": f"{Lm.REF_SPP}-spp mean of the renderer stand-in",
                        "ms_per_step": train_ms, "loss_first20": float(np.mean(losses[:20])),
                        "loss_last20": float(np.mean(losses[-20:]))},
           "network": {"gflop_per_frame": flops / 1e9}, "budgets": {}}
    net_ms = []
    captured = []
    for budget in (0.125, 0.25, 0.5):
        fr = spp.Frame(W, H, 3, max_budget=budget, device=dev)
        res = {}
        for form in ("plain", "learned"):
            state = {"prev": None, "parity": 0}

            def frame(k, record=None):
                x = frames[k]
                prev = state["prev"]
                if prev is not None:
                    Bnd.check(Bnd.spp_warp_previous(prev, x["mv"], W, H, warped), "warp")
                if form == "learned":
                    if prev is not None:
                        Bnd.check(Bnd.spp_tonemap_image(warped, W, H, tm, prev_ldr), "tonemap")
                    net.features(0, x["albedo"], x["normal"], x["depth"], x["mv"],
                                 prev_ldr if prev is not None else None)
                    if record is not None:
                        e0 = torch.cuda.Event(enable_timing=True)
                        e1 = torch.cuda.Event(enable_timing=True)
                        e0.record(stream)
                    net.forward()
                    if record is not None:
                        e1.record(stream)
                        record.append((e0, e1))
                    d = net.density[0]
                    lg = net.frame_logits(0, prev is not None)
                else:
                    d = ones
                    lg = [fixed[0] if prev is not None else fixed[0][:29], fixed[1], fixed[2]]
                fr.alloc(d, spp.make_params(budget, frame=k))
                fr.render(x["clean"], 0xC0FFEE, k)
                fr.splat()
                for l in (2, 1):
                    Bnd.check(Bnd.spp_reconstruct_level(
                        fr.layers[l], lg[l], lg[l].shape[0], hats[l + 1] if l < 2 else None, None,
                        None, W >> l, H >> l, None, hats[l], None, status=fr.status), "level")
                o = fr.hdr[state["parity"]]
                Bnd.check(Bnd.spp_reconstruct_level(
                    fr.layers[0], lg[0], lg[0].shape[0], hats[1],
                    warped if prev is not None else None, mask if prev is not None else None,
                    W, H, tm, o, fr.ldr, status=fr.status), "level 0")
                state["prev"] = o
                state["parity"] ^= 1
                return prev is not None, lg, o

            def cut(t, l=0):
                a, b = y0 >> l, (y0 + side) >> l
                return t[..., a:b, (x0 >> l):((x0 + side) >> l)].detach().cpu().numpy().copy()

            # pass 1, untimed: warms up and keeps the compared crops (the
            # timed pass recomputes the same values: every step is seeded)
            keep = form == "learned" and budget == 0.25
            for k in range(F):
                temporal, lg, o = frame(k)
                if keep:
                    captured.append(dict(
                        k=k, temporal=temporal,
                        prev_ldr=cut(prev_ldr) if temporal else None,
                        warped=cut(warped) if temporal else None,
                        logits=[cut(lg[l], l) for l in range(3)],
                        z=cut(net.heads[0][0, 54]),
                        noisy=[cut(fr.layers[l], l) for l in range(3)],
                        hdr=cut(o), ldr=cut(fr.ldr)))
            # pass 2, timed frame by frame
            state.update(prev=None, parity=0)
            rec = [] if form == "learned" else None
            evs = []
            torch.cuda.synchronize()
            for k in range(F):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                frame(k, rec)
                e1.record(stream)
                evs.append((e0, e1))
                Bnd.check(Bnd.spp_mse(fr.ldr, refs[k], 3 * W * H, mse[4 * k:4 * k + 1]), "mse")
                Bnd.check(Bnd.spp_mse(fr.ldr, refs64[k], 3 * W * H, mse[4 * k + 2:4 * k + 3]),
                          "mse")
            torch.cuda.synchronize()
            fr.check_status()
            m = mse.view(F, 4)[:, [0, 2]].cpu().numpy()
            p = -10.0 * np.log10(np.maximum(m, 1e-30))
            ms = [a.elapsed_time(b) for a, b in evs]
            res[form + "_ms"] = float(np.mean(ms[1:]))
            res[form + "_psnr_db"] = float(np.mean(p[1:, 0]))
            res[form + "_psnr_vs_64spp_db"] = float(np.mean(p[1:, 1]))
            res[form + "_per_frame"] = {"ms": ms, "psnr_db": p[:, 0].tolist(),
                                        "psnr_vs_64spp_db": p[:, 1].tolist()}
            if rec:
                net_ms += [a.elapsed_time(b) for a, b in rec]
        res["learned_gain_db"] = res["learned_psnr_db"] - res["plain_psnr_db"]
        res["note"] = ("means over frames 1..15 (frame 0 has no previous output); per-frame "
                       "arrays over frames 0..15")
        out["budgets"][str(budget)] = res
        del fr
    avg = float(np.mean(net_ms))
    tflops = flops / (avg / 1e3) / 1e12
    out["network"].update({"ms": avg, "tflops": tflops,
                           "bf16_peak_tflops": peaks.get("bf16_tflops_sustained",
                                                         peaks["bf16_tflops"]),
                           "frac_of_bf16_peak": tflops / peaks.get("bf16_tflops_sustained",
                                                                   peaks["bf16_tflops"]),
                           "peak_kind": peak_kind + " (sustained, the network runs inside a "
                                                    "longer frame)"})
    del net
    out["estimator_ablation"] = run_estimator_ablation(args, spp, rank)
    out["two_stage"] = run_two_stage(args, spp, Bnd, dev, rank, frames, refs, W, H, F, peaks,
                                     peak_kind)
    # kept for the comparison with the FP64 oracle after every timed section
    out["_oracle_crops"] = dict(theta=theta.detach().cpu().numpy().astype(np.float64),
                                crops=captured, scenes=scenes, W=W, H=H, x0=x0, y0=y0,
                                side=side)
    return out


def oracle_crop_errors(data):
    """Error of the learned BF16 frames against the FP64 oracle on a fixed
    crop of every frame of the 0.25-spp sequence (measurement only: nothing
    of it feeds the GPU path).  For each frame the oracle runs the exact FP64
    network (oracle/unet.py) on the window's features (from the frame's
    G-buffer and motion, and the previous tone-mapped output of the GPU
    sequence, the recurrent input of the frame) and reconstructs the window
    (the oracle's gather pyramid and tone map) from the FP64 logits over the
    frame's noisy pyramid and warped previous output as the GPU rendered
    them.  The inner ORACLE_CROP x ORACLE_CROP region is compared: logits
    and density logit (errors relative to the RMS of the oracle's values,
    as the parity tests measure BF16 networks), the HDR output (per-element
    relative) and the sRGB output (absolute).  A control reconstructs the
    window from the GPU's own logits, which must agree with the GPU's HDR to
    the reconstruction's 1e-5."""
    import oracle
    import oracle.unet as U
    theta, side, x0, y0 = data["theta"], data["side"], data["x0"], data["y0"]
    M, C = ORACLE_MARGIN, ORACLE_CROP
    rows = []
    for c in data["crops"]:
        clean, gb = data["scenes"][c["k"]]
        win = lambda a: np.asarray(a)[..., y0:y0 + side, x0:x0 + side]  # noqa: E731
        import spp_inputs as inp
        mv = win(inp.scene_motion(data["W"], data["H"], c["k"]))
        prev = c["prev_ldr"] if c["temporal"] else np.zeros((3, side, side))
        x12 = U.features(win(gb["albedo"]), win(gb["normal"]), win(gb["depth"]), mv, prev)
        fe = U.forward(theta, x12, round_bf16_acts=False)
        lg_ref = [fe["logits"][0] if c["temporal"] else fe["logits"][0][:29],
                  fe["logits"][1], fe["logits"][2]]

        def rec(lgs):
            hats = [None] * 3
            for l in (2, 1, 0):
                hats[l] = oracle.reconstruct_level(
                    c["noisy"][l], lgs[l], coarse=hats[l + 1] if l < 2 else None,
                    warped=c["warped"] if (l == 0 and c["temporal"]) else None,
                    mask=np.zeros((side, side), np.uint8) if (l == 0 and c["temporal"]) else None)
            return hats[0]

        hdr_ref = rec(lg_ref)
        hdr_ctl = rec([a.astype(np.float64) for a in c["logits"]])
        ldr_ref = oracle.tonemap(hdr_ref)
        inner = lambda a, l=0: a[..., (M >> l):((M + C) >> l), (M >> l):((M + C) >> l)]  # noqa

        def rel_rms(g, r):
            sc = np.sqrt(np.mean(r * r))
            return float(np.sqrt(np.mean((g - r) ** 2)) / sc), float(np.abs(g - r).max() / sc)

        row = {"frame": c["k"]}
        for l in range(3):
            row[f"logits_l{l}"] = rel_rms(inner(c["logits"][l], l), inner(lg_ref[l], l))
        row["z"] = rel_rms(inner(c["z"]), inner(fe["z"]))
        gh, rh = inner(c["hdr"]), inner(hdr_ref)
        er = np.abs(gh - rh) / np.maximum(np.abs(rh), 1e-30)
        row["hdr"] = (float(np.sqrt(np.mean(er ** 2))), float(er.max()))
        el = np.abs(inner(c["ldr"]) - inner(ldr_ref))
        row["ldr_abs"] = (float(np.sqrt(np.mean(el ** 2))), float(el.max()))
        ec = np.abs(inner(hdr_ctl) - gh) / np.maximum(np.abs(inner(hdr_ctl)), 1e-30)
        row["control_hdr_max_rel"] = float(ec.max())
        rows.append(row)

    def agg(key):
        return {"rms_rel_mean": float(np.mean([r[key][0] for r in rows])),
                "max_rel_max": float(np.max([r[key][1] for r in rows]))}
    return {
        "what": f"inner {C}x{C} of a {side}x{side} window at ({x0}, {y0}) of each of the "
                f"{len(rows)} frames at 0.25 spp; oracle: exact FP64 network and FP64 "
                f"reconstruction on the frame's noisy pyramid as rendered",
        "logits_l0": agg("logits_l0"), "logits_l1": agg("logits_l1"),
        "logits_l2": agg("logits_l2"), "density_logit": agg("z"),
        "hdr_per_element": agg("hdr"),
        "ldr_abs": {"rms_mean": float(np.mean([r["ldr_abs"][0] for r in rows])),
                    "max": float(np.max([r["ldr_abs"][1] for r in rows]))},
        "control_recon_from_gpu_logits_max_rel": float(np.max([r["control_hdr_max_rel"]
                                                               for r in rows])),
        "per_frame_hdr_rms_rel": [r["hdr"][0] for r in rows],
        "per_frame_logits_l0_rms_rel": [r["logits_l0"][0] for r in rows],
    }


def run_estimator_ablation(args, spp, rank):
    """The gradient estimators of the discretisation (Sec. 4.3 and the
    ablation of Sec. 7): the joint predictor trained from the same start
    with the relaxed ramp, the straight-through estimator, the
    Gumbel-softmax relaxation and the DASR surrogate of Sec. 4.1
    (deterministic rounding); held-out PSNR at 0.25 spp on 128 x 128
    two-frame samples (each model with its own test-time rule)."""
    import torch

    import spp_inputs as inp
    from paper_2602_08642_gb300 import learned as Lm

    size, budget = 128, 0.25
    steps = max(args.train_steps // 2, 1)
    train = [Lm.FrameData(inp.training_pair(size, seed=100 + i + 1000 * rank)) for i in range(32)]
    held = [Lm.FrameData(inp.training_pair(size, seed=5000 + i)) for i in range(8)]
    fixed = [torch.from_numpy(a).cuda() for a in inp.fixed_logits(size, size, 3, True)]
    res = {"steps": steps, "crop": size, "batch": 8, "spp": budget,
           "plain_psnr_db": float(np.mean(Lm.evaluate(held, budget, None, fixed)))}
    for est in ("relaxed", "straight_through", "gumbel", "dasr"):
        theta0 = torch.from_numpy(inp.unet_params(Lm.layer_table(), seed=5,
                                                  head_bias=inp.fixed_head_bias()))
        tr = Lm.Trainer(theta0, 8, size, budget, lr=1e-3, estimator=est)
        rng = np.random.default_rng(rank)
        losses = []
        for k in range(steps):
            idx = rng.choice(len(train), 8, replace=False)
            losses.append(tr.step([train[i] for i in idx], seed=1000 + 17 * k))
        cov = []
        res[est] = {"psnr_db": float(np.mean(Lm.evaluate(held, budget, tr.net.theta, None,
                                                         estimator=est, coverage=cov))),
                    "loss_first20": float(np.mean(losses[:20])),
                    "loss_last20": float(np.mean(losses[-20:])),
                    "test_spp": float(np.mean([c[0] for c in cov])),
                    "test_pixels_without_sample": float(np.mean([c[1] for c in cov]))}
        del tr
    return res


def run_two_stage(args, spp, Bnd, dev, rank, frames, refs, W, H, F, peaks, peak_kind):
    """The two-stage pipeline (sampler network, rendering, denoiser network
    with learned demodulation and shared latents), trained on the GPU like
    the joint predictor, on the same frames: per-frame time (every step from
    the sampler's feature assembly to the tone-mapped output) and PSNR."""
    import torch

    import spp_inputs as inp
    from paper_2602_08642_gb300 import learned as Lm
    from paper_2602_08642_gb300 import two_stage as T2

    train = [Lm.FrameData(inp.training_pair(128, seed=100 + i + 1000 * rank)) for i in range(32)]
    fb = inp.fixed_head_bias()
    ts = torch.from_numpy(inp.unet_params(T2.layer_table(Bnd.SPP_NET_SAMPLER), seed=3))
    td = torch.from_numpy(inp.unet_params(
        T2.layer_table(Bnd.SPP_NET_DENOISER), seed=4,
        head_bias={"h0": np.concatenate([fb["h0"][:54], np.zeros(10, np.float32)]),
                   "h1": fb["h1"], "h2": fb["h2"]}))
    tr = T2.TwoStageTrainer(ts, td, 8, 128, 0.25, lr=1e-3)
    rng = np.random.default_rng(rank)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    losses = []
    for k in range(args.train_steps):
        idx = rng.choice(len(train), 8, replace=False)
        losses.append(tr.step([train[i] for i in idx], seed=1000 + 17 * k))
    torch.cuda.synchronize()
    train_ms = (time.perf_counter() - t0) * 1e3 / max(args.train_steps, 1)
    theta_s, theta_d = tr.p.sampler.theta, tr.p.denoiser.theta
    del tr, train

    stream = torch.cuda.current_stream()
    flops = T2.flops_per_frame(W, H)
    out = {"pipeline": "sampler features -> sampler U-Net (BF16 tcgen05) -> density softmax -> "
                       "sample map -> renderer stand-in -> splat -> denoiser features -> "
                       "denoiser U-Net -> demodulation + pyramid -> gather pyramid with the "
                       "temporal term -> remodulation + tone map; latents warped to the next "
                       "frame",
           "training": {"steps": args.train_steps, "crop": 128, "batch": 8, "spp": 0.25,
                        "ms_per_step": train_ms, "loss_first20": float(np.mean(losses[:20])),
                        "loss_last20": float(np.mean(losses[-20:]))},
           "networks": {"gflop_per_frame": flops / 1e9}, "budgets": {}}
    p = None
    for budget in (0.125, 0.25, 0.5):
        p = T2.TwoStage(theta_s, theta_d, 1, W, H, budget)
        x_of = lambda k: frames[k % F]  # noqa: E731
        p.begin_sequence()
        psnr = []
        for k in range(F):  # one coherent pass: PSNR of frames 1..F-1
            x = x_of(k)
            p.frame([x], [x["mv"]], [x["clean"]], 0, k)
            if k > 0:
                p.ref[0].copy_(refs[k])
                psnr.append(p.psnr(0))
        steps = 12
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for k in range(F, F + steps):
            x = x_of(k)
            p.frame([x], [x["mv"]], [x["clean"]], 0, k)
        e1.record(stream)
        torch.cuda.synchronize()
        for fr in p.frames:
            fr.check_status()
        out["budgets"][str(budget)] = {"ms": e0.elapsed_time(e1) / steps,
                                       "psnr_db": float(np.mean(psnr))}
        if budget != 0.5:
            del p
    # variants of Sec. 7 at 0.25 spp with the same trained networks: the
    # low-resolution density map (2 x 2 blocks) and systematic rounding
    variants = {}
    for name, kw in (("lowres_density_2x2", dict(density_factor=2)),
                     ("systematic_rounding", dict(rounding="systematic"))):
        q = T2.TwoStage(theta_s, theta_d, 1, W, H, 0.25, **kw)
        q.begin_sequence()
        ps, totals = [], []
        for k in range(F):
            x = frames[k % F]
            q.frame([x], [x["mv"]], [x["clean"]], 0, k)
            totals.append(int(q.frames[0].total.item()))
            if k > 0:
                q.ref[0].copy_(refs[k])
                ps.append(q.psnr(0))
        variants[name] = {"psnr_db": float(np.mean(ps)), "samples_per_frame": totals}
        del q
    out["variants_at_0.25spp"] = variants
    # the two networks alone, on the last frame's inputs
    reps = 10
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        p.sampler.forward_prepared()
        p.denoiser.forward_prepared()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    tflops = flops / (ms / 1e3) / 1e12
    peak = peaks.get("bf16_tflops_sustained", peaks["bf16_tflops"])
    out["networks"].update({"ms": ms, "tflops": tflops, "bf16_peak_tflops": peak,
                            "frac_of_bf16_peak": tflops / peak, "peak_kind": peak_kind})
    del p
    return out


def run_e2e(args, spp, Bnd, fr, host_inputs, step, dev, stream, W, H, L, F, world, dist):
    import torch
    pinned = []
    for x in host_inputs:
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()  # noqa: E731
        pinned.append(dict(d=pin(x["d"]), clean=pin(x["clean"]),
                           logits=[pin(a) for a in x["logits"]], mv=pin(x["mv"]),
                           mask=pin(x["mask"])))

    def make_staging():
        return dict(d=torch.empty_like(pinned[0]["d"], device=dev),
                    clean=torch.empty_like(pinned[0]["clean"], device=dev),
                    logits=[torch.empty_like(a, device=dev) for a in pinned[0]["logits"]],
                    mv=torch.empty_like(pinned[0]["mv"], device=dev),
                    mask=torch.empty_like(pinned[0]["mask"], device=dev))

    # two staging sets: the copy stream fills one with frame k + 1's inputs
    # while the frame stream computes frame k from the other (the host link,
    # about 210 GB/s, is the bound); the result goes back on its own stream
    staging = [make_staging(), make_staging()]
    copy_stream = torch.cuda.Stream(device=dev)
    d2h_stream = torch.cuda.Stream(device=dev)
    ev_copied = [torch.cuda.Event(), torch.cuda.Event()]
    ev_used = [torch.cuda.Event(), torch.cuda.Event()]
    ev_done = torch.cuda.Event()
    ev_read = torch.cuda.Event()
    out_host = torch.empty((3, H, W), dtype=torch.float32).pin_memory()
    h2d = sum(t.numel() * t.element_size() for t in
              [pinned[0]["d"], pinned[0]["clean"], pinned[0]["mv"], pinned[0]["mask"],
               *pinned[0]["logits"]])
    d2h = out_host.numel() * out_host.element_size()

    def issue_copy(k):
        x, buf = pinned[k % F], staging[k % 2]
        copy_stream.wait_event(ev_used[k % 2])  # the frame that read this set is done
        with torch.cuda.stream(copy_stream):
            buf["d"].copy_(x["d"], non_blocking=True)
            buf["clean"].copy_(x["clean"], non_blocking=True)
            for a, b in zip(buf["logits"], x["logits"]):
                a.copy_(b, non_blocking=True)
            buf["mv"].copy_(x["mv"], non_blocking=True)
            buf["mask"].copy_(x["mask"], non_blocking=True)
        ev_copied[k % 2].record(copy_stream)

    def e2e_step(k, last):
        stream.wait_event(ev_copied[k % 2])
        stream.wait_event(ev_read)  # the previous result has left fr.ldr
        step(k, inp=staging[k % 2])
        ev_used[k % 2].record(stream)
        ev_done.record(stream)
        d2h_stream.wait_event(ev_done)
        with torch.cuda.stream(d2h_stream):
            out_host.copy_(fr.ldr, non_blocking=True)
        ev_read.record(d2h_stream)
        if not last:
            issue_copy(k + 1)

    issue_copy(0)
    for k in range(2):
        e2e_step(k, last=k == 1)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    copy_stream.wait_event(t0)
    issue_copy(2)
    for k in range(args.e2e_steps):
        e2e_step(2 + k, last=k == args.e2e_steps - 1)
    stream.wait_event(ev_read)  # the last result is on the host
    t1.record(stream)
    torch.cuda.synchronize()
    ms = slowest_rank_ms(t0.elapsed_time(t1), world, dev)
    return {"value": whole_job_rate(W * H * args.e2e_steps, world, ms), "unit": UNIT,
            "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
            "ms_per_step": ms / args.e2e_steps, "steps": args.e2e_steps}


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    run_ours(args, rank, world, local)


if __name__ == "__main__":
    main()
