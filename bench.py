#!/usr/bin/env python3
"""Cold-frame throughput of slice-based illuminated ray casting on GB300.

One step = one whole frame through the hot path: the light-space attenuation
sweep (256 slices of 512 x 512 FP32 texels) followed by the cone-scattering
eye march (1024 x 1024 perspective, step 0.5 voxel, early ray termination at
0.99) over a 256^3 uint16 CT-like ellipsoid phantom (seed 2) with a 4096-entry
RGBA transfer function.  Inputs are synthetic and seeded.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

Prints one JSON line (rank 0).  Under torchrun every rank renders its own
frames (replicas; frames are independent) and the slowest rank's time counts.
``--impl reference`` times the FP64 CPU oracle on this host's cores instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = ("ct256-u16 ellipsoid phantom, 256x512^2 FP32 attenuation stack, cone 15deg, "
            "1024x1024 perspective, step 0.5 vox, ERT 0.99")
L2_FLUSH_BYTES = 256 << 20   # > 129 MB of L2
FP32_LANES_PER_SM = 128
# Algorithmic FP32 flops per eye sample (an FMA counts 2): position + t (8),
# voxel coordinates (6), trilinear (21), transfer function (14), compositing
# (15) for every sample; light coordinates (6) + light factor (2) + per lookup
# 12 (3 adds for its coordinates, 3 lerps) + the average, for samples with
# alpha > 0 only.
FLOPS_BASE = 8 + 6 + 21 + 14 + 15
FLOPS_LIT = {0: 0, 1: 6 + 2 + 12, 2: 6 + 2 + 6 * 12 + 7, 3: 6 + 2 + 8 * 12 + 9}

# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) from one
# ncu capture of this workload (its summary is kept under profiles/).  Each
# entry holds for the kernel sources it was taken from (hash of the files that
# define the kernel); once they change the figure is stale and reported as null.
NCU_TRAFFIC = {
    "march_kernel": (("vi_march.cu", "vi_device.cuh", "vi_internal.h"), "af44da2bee6d4b70",
                     32_089_088),
    "sweep_kernel": (("vi_sweep.cu", "vi_device.cuh", "vi_internal.h"), "e6828894ef5d6882",
                     240_257_536),
}


# Other counters of the same march capture, for its candidate bounds: warp-level
# instructions executed and L2 sectors (32 B) per launch.
NCU_MARCH_COUNTERS = {"inst_executed": 453_145_357, "lts_sectors": 10_502_863}


def march_bounds(march_s: float, sms: int, clock_mhz: float, peaks: dict, probe: dict):
    """The march's three candidate bounds (HBM, L2, instruction issue) with the
    binding one named: DRAM bytes, L2 sectors and warp instructions from the
    capture of this kernel, time and clock from this run, the L2 peak from the
    probe kernel."""
    if ncu_traffic("march_kernel") is None:
        return None
    traffic = ncu_traffic("march_kernel")
    c = NCU_MARCH_COUNTERS
    issue_slots = march_s * sms * 4 * clock_mhz * 1e6     # one warp instruction / cycle / SMSP
    l2_gbs = c["lts_sectors"] * 32 / march_s / 1e9
    out = {"hbm": {"bytes": traffic, "gbs": round(traffic / march_s / 1e9, 1),
                   "frac": round(traffic / march_s / 1e9 / peaks["hbm_gbs"], 4)},
           "l2": {"bytes": c["lts_sectors"] * 32, "gbs": round(l2_gbs, 1),
                  "frac": round(l2_gbs / probe["l2_read_gbs"], 4),
                  "peak_gbs": round(probe["l2_read_gbs"], 1), "peak_source": "probe kernel"},
           "issue": {"warp_instructions": c["inst_executed"],
                     "frac": round(c["inst_executed"] / issue_slots, 4)},
           "source": "counters from the ncu capture of this kernel (profiles/); time and "
                     "clock from this run"}
    out["binding"] = max(("hbm", "l2", "issue"), key=lambda k: out[k]["frac"])
    return out


def ncu_traffic(kernel: str):
    import hashlib
    files, digest, nbytes = NCU_TRAFFIC[kernel]
    m = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_2008_06134_gb300", "csrc", f), "rb") as fh:
            m.update(fh.read())
    return nbytes if m.hexdigest()[:16] == digest else None


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-depth", type=int, default=4,
                    help="contexts (streams) in the end-to-end pipeline")
    ap.add_argument("--cpu-baseline-only", action="store_true", help=argparse.SUPPRESS)
    ap.add_argument("--no-summaries", action="store_true",
                    help="leave the serving and precision summaries out of the headline line")
    ap.add_argument("--workload", default="ct256-cone",
                    choices=["ct256-cone", "precision", "scalability", "serving", "variants",
                             "large", "oracle"],
                    help="ct256-cone: the headline frame; precision: storage formats on the "
                         "512^3 blob scene vs the FP64 oracle; scalability: slice count x "
                         "slice resolution grid; serving: the render server on a stream of "
                         "mixed requests; variants: the method variants and the point light "
                         "on the headline scene; large: 1024^3 volume, 1024 x 2048^2 FP16 "
                         "stack, 3840x2160; oracle: the FP64 oracle timed beside the GPU on "
                         "every scene")
    ap.add_argument("--requests", type=int, default=512, help="serving: request count")
    ap.add_argument("--rate", default="300,800",
                    help="serving: Poisson arrival rates per second (comma-separated)")
    ap.add_argument("--slots", type=int, default=8, help="serving: concurrent render slots")
    ap.add_argument("--budget-gib", type=float, default=8.0, help="serving: HBM budget")
    ap.add_argument("--large-n", type=int, default=1024, help="large: volume edge")
    ap.add_argument("--large-slices", type=int, default=1024, help="large: slice count")
    ap.add_argument("--large-res", type=int, default=2048, help="large: slice resolution")
    ap.add_argument("--large-image", default="3840x2160", help="large: image W x H")
    return ap.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def max_over_ranks(x: float, dist=None, device="cpu") -> float:
    """The slowest rank's value (every rank gets it)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank: int, world: int, max_seconds: float) -> float:
    """Whole-job rate: the units all ranks processed over the slowest rank's time."""
    return units_per_rank * world / max_seconds


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled while the timed region runs."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.reader = threading.Thread(target=self._read, daemon=True)
            self.reader.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        time.sleep(0.15)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.reader.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for name, val in zip(names, parts[4:8]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------------
# CPU oracle (the baseline and the reference arm).

def oracle_sample(scene, bands: int, band: int, stack, light):
    """Time one band (1/bands of the texel rows and of the image rows) of the
    oracle's sweep + march; returns seconds."""
    import numpy as np

    import oracle
    R, H, W = scene.slice_res, scene.height, scene.width
    j0, j1 = band * R // bands, (band + 1) * R // bands
    y0, y1 = band * H // bands, (band + 1) * H // bands
    ys, xs = np.mgrid[y0:y1, 0:W]
    ro = oracle.render_opts(scene.mode, scene.step_vox, scene.ert, scene.bg, scene.light_color,
                            cone_half_angle_deg=scene.cone_half_angle_deg)
    t0 = time.perf_counter()
    oracle.build_stack_rows(scene.volume, scene.tf, scene.vmin, scene.vmax, light, j0, j1, stack)
    oracle.render_pixels(scene.volume, scene.tf, scene.vmin, scene.vmax, light, stack,
                         scene.camera, W, H, ro, xs.ravel(), ys.ravel())
    return time.perf_counter() - t0


def oracle_setup(scene):
    import oracle
    oracle.build()
    light = oracle.light_setup(scene.light_dir, scene.n_slices, scene.slice_res)
    stack = oracle.build_stack(scene.volume, scene.tf, scene.vmin, scene.vmax, light)
    return light, stack


def cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                low = line.lower()
                if low.startswith("model name") or low.startswith("cpu part"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.machine()


def cpu_baseline(scene, min_seconds: float = 10.0, max_frames: int = 4):
    """The oracle, as it stands, on a bounded sample: bands of 1/8 of the
    sweep's texel rows and 1/8 of the image rows, taken in turn over the frame
    until at least `min_seconds` have been timed (at most `max_frames` whole
    frames); frames/s = bands / 8 / seconds."""
    import oracle
    light, stack = oracle_setup(scene)
    bands, done, secs = 8, 0, 0.0
    while secs < min_seconds and done < max_frames * bands:
        secs += oracle_sample(scene, bands, done % bands, stack, light)
        done += 1
    fps = done / bands / secs
    return {"value": round(fps, 4), "unit": "frames/s", "cores": oracle.threads(),
            "cpu": cpu_model(), "kind": "oracle",
            "sample": f"{done} bands of 1/{bands} frame (1/{bands} of the sweep's texel rows "
                      f"+ 1/{bands} of the image rows, in turn over the frame) = "
                      f"{done / bands:.3g} frames, FP64, {secs:.1f} s"}


def cpu_baseline_fresh(timeout_s: float = 600.0):
    """cpu_baseline in a fresh process: this one holds a CUDA context and
    torch's thread pools, which measured up to 1.7x slower oracle bands than a
    process of its own (the reference arm's conditions)."""
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-baseline-only"],
                       capture_output=True, text=True, timeout=timeout_s, cwd=ROOT)
    for line in reversed(r.stdout.splitlines()):
        if line.startswith("{"):
            out = json.loads(line)
            out["process"] = "fresh (python bench.py --cpu-baseline-only)"
            return out
    return {"unavailable": f"cpu baseline process exited {r.returncode}: {r.stderr[-300:]}"}


def reference_arm(args):
    """The FP64 oracle as it stands, timed on this host's cores.  Each step is
    one band of the headline frame: 1/8 of the sweep's texel rows and 1/8 of
    the image rows, the bands taken in turn over the frame (the same sample as
    cpu_baseline, wide enough for every core); ms_per_step is the measured
    mean time of a step, and frames/s is one over the sum of the eight bands'
    mean times."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    from paper_2008_06134_gb300 import phantoms as ph
    scene = ph.ct256_cone()
    light, stack = oracle_setup(scene)
    bands = 8
    for w in range(args.warmup):
        oracle_sample(scene, bands, w % bands, stack, light)
    secs, per_band = [], {}
    for s in range(args.steps):
        t = oracle_sample(scene, bands, s % bands, stack, light)
        secs.append(t)
        per_band.setdefault(s % bands, []).append(t)
    total = sum(secs)
    # A frame is the sum of its bands' mean times (bands differ in cost: the
    # middle ones cross the phantom), so any step count gives an unbiased rate.
    frame_s = sum(statistics.mean(v) for v in per_band.values()) * bands / len(per_band)
    fps = 1.0 / frame_s
    line = {"metric": "frames/s", "value": round(fps, 5), "unit": "frames/s", "impl": "reference",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(1000 * total / args.steps, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "impl": "FP64 CPU oracle (oracle/vi_oracle.c)",
                       "step": f"1/{bands} of a frame (a band of texel rows and image rows)"},
            "cpu_baseline": {"value": round(fps, 5), "unit": "frames/s", "kind": "oracle",
                             "cores": oracle.threads(), "cpu": cpu_model(),
                             "sample": f"{args.steps} steps, each 1/{bands} of the texel rows "
                                       f"of the sweep + 1/{bands} of the image rows, bands "
                                       f"rotating over the frame; {total:.1f} s timed"},
            "e2e": {"value": round(fps, 5), "unit": "frames/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------
# GB300 arm.

def gb300_arm(args):
    import numpy as np
    import torch

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2008_06134_gb300 import build, phantoms as ph, vi
    if rank == 0:
        build.build()
    if dist:
        dist.barrier()

    sc = ph.ct256_cone()
    H, W = sc.height, sc.width
    ctx = vi.Context(local)
    vol_dev = torch.from_numpy(sc.volume.view(np.int16)).cuda()
    ctx.load_volume(vol_dev, dtype=vi.U16)
    ctx.set_transfer_function(sc.tf, sc.vmin, sc.vmax)
    ctx.set_light(sc.light_dir, sc.light_color)
    out = torch.empty((H, W, 4), dtype=torch.float32, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")

    def build_stack():
        ctx.build_attenuation(sc.n_slices, sc.slice_res, sc.mode,
                              cone_half_angle_deg=sc.cone_half_angle_deg)

    def render(o=None, **kw):
        return ctx.render(sc.camera, W, H, sc.step_vox, out=out if o is None else o, ert=sc.ert,
                          bg=sc.bg, **kw)

    # One counted frame (untimed): samples composited and samples that were lit.
    counts = torch.zeros((H, W), dtype=torch.int32, device="cuda")
    lit = torch.zeros((H, W), dtype=torch.int32, device="cuda")
    build_stack()
    render(sample_counts=counts, lit_counts=lit)
    torch.cuda.synchronize()
    samples = int(counts.sum().item())
    lit_samples = int(lit.sum().item())

    for _ in range(args.warmup):
        flush.fill_(0)
        build_stack()
        render()
    # Roofline denominators of this device, measured by probe kernels.
    probe = vi.measure_peaks(local)
    K = args.steps
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(K)]
    clocks = ClockSampler(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    launches0 = ctx.launch_count()
    wall0 = time.perf_counter()
    for s in range(K):
        flush.fill_(s & 0xFF)          # evict L2 between steps (outside the timed events)
        ev[s][0].record()
        build_stack()
        ev[s][1].record()
        render()
        ev[s][2].record()
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    if dist:
        dist.barrier()
    clock = clocks.stop()
    launches = ctx.launch_count() - launches0
    sweep_ms = [e[0].elapsed_time(e[1]) for e in ev]
    march_ms = [e[1].elapsed_time(e[2]) for e in ev]
    total_ms = sum(sweep_ms) + sum(march_ms)
    max_total_ms = max_over_ranks(total_ms, dist, "cuda")

    # End to end through the public API: host volume / TF in, host frame out.
    e2e = None
    if not args.no_e2e:
        pinned_vol = torch.empty(sc.volume.shape, dtype=torch.int16, pin_memory=True)
        pinned_vol.numpy()[...] = sc.volume.view(np.int16)
        pinned_out = torch.empty((H, W, 4), dtype=torch.float32, pin_memory=True)
        tf = np.ascontiguousarray(sc.tf, dtype=np.float32)

        def e2e_step():
            ctx.load_volume(pinned_vol, dtype=vi.U16)
            ctx.set_transfer_function(tf, sc.vmin, sc.vmax)
            ctx.set_light(sc.light_dir, sc.light_color)
            build_stack()
            render(o=pinned_out)        # host output: returns once the frame is in host memory

        for _ in range(args.warmup):
            e2e_step()
        secs = 0.0
        for s in range(K):
            flush.fill_(s & 0xFF)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            e2e_step()
            secs += time.perf_counter() - t0
        serial = job_throughput(K, world, max_over_ranks(secs, dist, "cuda"))

        # Pipelined: D contexts on D streams (--e2e-depth), so the uploads and
        # sweeps of the next steps overlap step s's march and read-back.  Every
        # step copies its volume and TF from pinned host memory and reads its
        # frame back into pinned host memory, all through the C ABI (vi_render
        # with VI_OUT_HOST_ASYNC; vi_sync completes the frame); the host waits
        # for a frame before its buffers are reused.
        depth = max(2, args.e2e_depth)
        streams = [torch.cuda.Stream(local) for _ in range(depth)]
        ctxs = [vi.Context(local, stream=st) for st in streams]
        host_out = [torch.empty((H, W, 4), dtype=torch.float32, pin_memory=True)
                    for _ in range(depth)]
        flushes = [torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
                   for _ in range(depth)]
        checksum = 0.0

        def issue(s, flush_l2):
            b = s % depth
            c, st = ctxs[b], streams[b]
            if flush_l2:
                with torch.cuda.stream(st):
                    flushes[b].fill_(s & 0xFF)
            c.load_volume(pinned_vol, dtype=vi.U16)
            c.set_transfer_function(tf, sc.vmin, sc.vmax)
            c.set_light(sc.light_dir, sc.light_color)
            c.build_attenuation(sc.n_slices, sc.slice_res, sc.mode,
                                cone_half_angle_deg=sc.cone_half_angle_deg)
            c.render(sc.camera, W, H, sc.step_vox, out=host_out[b], ert=sc.ert, bg=sc.bg,
                     host_async=True)

        def collect(s):
            nonlocal checksum
            ctxs[s % depth].sync()
            checksum += float(host_out[s % depth][H // 2, W // 2, 3])  # the host reads the frame

        def pipelined(flush_l2):
            for s in range(args.warmup):
                issue(s, flush_l2)
                if s >= 1:
                    collect(s - 1)
            collect(args.warmup - 1)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for s in range(K):
                if s >= depth:
                    collect(s - depth)
                issue(s, flush_l2)
            for s in range(max(0, K - depth), K):
                collect(s)
            return time.perf_counter() - t0

        # Every byte a step reads on the device is written in that step (its
        # volume uploaded, its pair bricks, flags, stack and frame built) and a
        # step moves ~0.4 GB through the 129 MB L2, so no step can read an
        # earlier step's data from L2: the headline runs without a flush; the
        # same pipeline with a 256 MiB L2 flush queued before every step is
        # reported beside it.
        secs_flushed = pipelined(True)
        secs = pipelined(False)
        for c in ctxs:
            c.close()
        e2e = {"value": round(job_throughput(K, world, max_over_ranks(secs, dist, "cuda")), 3),
               "l2": "no flush: each step's device working set (volume 33.6 MB, pair bricks, "
                     "stack 268 MB, frame 16.8 MB) is written in that step and is larger than "
                     "L2",
               "value_l2_flushed": round(job_throughput(K, world,
                                                        max_over_ranks(secs_flushed, dist,
                                                                       "cuda")), 3),
               "unit": "frames/s",
               "h2d_bytes_per_step": int(sc.volume.nbytes + tf.nbytes),
               "d2h_bytes_per_step": int(H * W * 16),
               "pipeline": f"{depth} contexts on {depth} streams; the next steps' uploads "
                           "and sweeps overlap step s's march and read-back; the frame comes "
                           "back through vi_render (VI_OUT_HOST_ASYNC) into pinned memory, "
                           "vi_sync per frame",
               "one_at_a_time_value": round(serial, 3)}

    if rank != 0:
        return
    peaks, peak_kind = measured_peaks()
    props = torch.cuda.get_device_properties(local)
    sweep_s = statistics.mean(sweep_ms) / 1e3
    march_s = statistics.mean(march_ms) / 1e3
    n, R = sc.n_slices, sc.slice_res
    sweep_bytes = sc.volume.nbytes + n * R * R * 4
    sweep_roof = {"bound": "hbm", "achieved": round(sweep_bytes / sweep_s / 1e9, 1),
                  "peak": peaks["hbm_gbs"], "unit": "GB/s",
                  "frac": round(sweep_bytes / sweep_s / 1e9 / peaks["hbm_gbs"], 4),
                  "traffic": ncu_traffic("sweep_kernel"), "algorithmic_bytes": int(sweep_bytes),
                  "kernel": "sweep_kernel",
                  "peak_source": f"{peak_kind} HBM copy bandwidth"}
    flops = samples * FLOPS_BASE + lit_samples * FLOPS_LIT[sc.mode]
    nominal_fp32 = props.multi_processor_count * FP32_LANES_PER_SM * 2 * peaks["sm_max_mhz"] / 1e6
    fp32_peak = probe["fp32_tflops"]
    march_roof = {"bound": "alu", "achieved": round(flops / march_s / 1e12, 3),
                  "peak": round(fp32_peak, 1), "unit": "TFLOP/s",
                  "frac": round(flops / march_s / 1e12 / fp32_peak, 4),
                  "traffic": ncu_traffic("march_kernel"), "algorithmic_flops": int(flops),
                  "kernel": "march_kernel",
                  "peak_source": "measured by probe: vi_measure_peaks (eight independent FMA "
                                 "chains per thread on every SM, best of 3 launches) in this "
                                 f"run; nominal {props.multi_processor_count} SMs x "
                                 f"{FP32_LANES_PER_SM} lanes x 2 x {peaks['sm_max_mhz']} MHz = "
                                 f"{nominal_fp32:.1f}"}
    dominant, other = (march_roof, sweep_roof) if march_s >= sweep_s else (sweep_roof, march_roof)
    clock_mhz = clock.get("sm_mhz") or peaks["sm_max_mhz"]
    frames = world * K
    line = {
        "metric": "frames/s", "value": round(job_throughput(K, world, max_total_ms / 1e3), 3),
        "unit": "frames/s", "n_gpus": world, "steps": K, "warmup": args.warmup,
        "ms_per_step": round(max_total_ms / K, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "volume": "256^3 uint16 (seed 2)",
                   "stack": f"{n}x{R}x{R} FP32", "image": f"{W}x{H}",
                   "l2": "flushed between steps (256 MiB write, outside the timed events)",
                   "parallelism": f"replicas x{world} (independent frames)"},
        "gsamples_per_s": round(samples * frames / (max_total_ms / 1e3) / 1e9, 3),
        "march_gsamples_per_s": round(samples / march_s / 1e9, 3),
        # The sweep's own unit: texel-slices (n R^2 per frame), apart from eye-ray samples.
        "sweep_gtexel_steps_per_s": round(n * R * R / sweep_s / 1e9, 3),
        "samples_per_frame": samples, "lit_samples_per_frame": lit_samples,
        "sweep_ms": round(sweep_s * 1e3, 4), "march_ms": round(march_s * 1e3, 4),
        "warm_frames_per_s": round(1.0 / march_s, 2),      # march only, stack cached
        "march_bounds": march_bounds(march_s, props.multi_processor_count, clock_mhz, peaks,
                                     probe),
        "peaks_probe": {k: round(v, 1) for k, v in probe.items()},
        "wall_s": round(wall, 3),
        "roofline": dominant, "roofline_other": other,
        "gpu_launches": int(launches),
        "clocks": clock,
        "e2e": e2e,
    }
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_fresh()
    ctx.close()
    del out, flush, counts, lit
    torch.cuda.empty_cache()
    if world == 1 and not args.no_summaries:
        # The other configs' headline figures, so that every run records them:
        # the served reduced-precision path against the plain FP32 path
        # (the serving mix), the storage formats' error against the oracle (the
        # 512^3 blob frames) and the large-volume frame (1024^3).
        line["serving"] = serving_summary(args)
        line["precision"] = precision_summary(args)
        # The large-volume workload's figures (fewer steps than its own line).
        large = large_result(args, 5, 2)
        line["large"] = {k: large[k] for k in ("scene", "frames_per_s", "sweep_ms", "march_ms",
                                               "gsamples_per_s", "sweep_gbs",
                                               "sweep_frac_of_measured_hbm")}
    print(json.dumps(line), flush=True)


def timed_frames(ctx, build, render, flush, steps):
    """Mean sweep and march ms over `steps` frames (CUDA events, L2 flushed)."""
    import torch
    sw, ma = [], []
    for s in range(steps):
        flush.fill_(s & 0xFF)
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        e[0].record()
        build()
        e[1].record()
        render()
        e[2].record()
        torch.cuda.synchronize()
        sw.append(e[0].elapsed_time(e[1]))
        ma.append(e[1].elapsed_time(e[2]))
    return statistics.mean(sw), statistics.mean(ma)


def precision_rows(steps: int, warmup: int, modes=("shell", "cone"), depth: bool = True):
    """Storage formats FP32 / FP16 / BF16 / UNORM16 on the 512^3 blob scene:
    frames/s of each and its per-channel error against the FP64
    oracle on the centred 256x144 crop (the oracle builds its own FP64 stack).
    Returns (scene name, oracle seconds, rows)."""
    import numpy as np
    import torch

    import oracle
    from paper_2008_06134_gb300 import build, phantoms as ph, vi
    build.build()
    oracle.build()
    sc = ph.blob512_precision()
    W, H = sc.width, sc.height
    x0, y0 = (W - 256) // 2, (H - 144) // 2
    ys, xs = np.mgrid[y0:y0 + 144, x0:x0 + 256]
    mode_of = {"shell": vi.SHELL, "cone": vi.CONE}
    t0 = time.perf_counter()
    light = oracle.light_setup(sc.light_dir, sc.n_slices, sc.slice_res)
    ref_stack = oracle.build_stack(sc.volume, sc.tf, sc.vmin, sc.vmax, light)
    refs = {}
    for mname in modes:
        ro = oracle.render_opts(mode_of[mname], sc.step_vox, sc.ert, sc.bg, sc.light_color,
                                cone_half_angle_deg=sc.cone_half_angle_deg)
        refs[mode_of[mname]] = oracle.render_pixels(sc.volume, sc.tf, sc.vmin, sc.vmax, light,
                                                    ref_stack, sc.camera, W, H, ro, xs.ravel(),
                                                    ys.ravel())[0]
    del ref_stack
    depth_ref = None
    if depth:
        # The extinction form (Eq. 5-6) against the oracle's own optical-depth frame.
        depth_stack = oracle.build_stack(sc.volume, sc.tf, sc.vmin, sc.vmax, light,
                                         quantity=oracle.OPTICAL_DEPTH)
        ro = oracle.render_opts(vi.CONE, sc.step_vox, sc.ert, sc.bg, sc.light_color,
                                cone_half_angle_deg=sc.cone_half_angle_deg,
                                quantity=oracle.OPTICAL_DEPTH)
        depth_ref = oracle.render_pixels(sc.volume, sc.tf, sc.vmin, sc.vmax, light, depth_stack,
                                         sc.camera, W, H, ro, xs.ravel(), ys.ravel())[0]
        del depth_stack
    oracle_s = time.perf_counter() - t0
    ctx = vi.Context(0)
    ctx.load_volume(torch.from_numpy(sc.volume.view(np.int16)).cuda(), dtype=vi.U16)
    ctx.set_transfer_function(sc.tf, sc.vmin, sc.vmax)
    ctx.set_light(sc.light_dir, sc.light_color)
    out = torch.empty((H, W, 4), dtype=torch.float32, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    names = {vi.F32: "f32", vi.F16: "f16", vi.BF16: "bf16", vi.UNORM16: "unorm16"}
    rows = {}
    cases = [(mode_of[mname], mname, fmt, vi.TRANSMITTANCE) for mname in modes
             for fmt in (vi.F32, vi.F16, vi.BF16, vi.UNORM16)]
    if depth:
        cases += [(vi.CONE, "cone-depth", fmt, vi.OPTICAL_DEPTH)
                  for fmt in (vi.F32, vi.F16, vi.BF16)]
    for mode, mname, fmt, quantity in cases:
        def bld():
            ctx.build_attenuation(sc.n_slices, sc.slice_res, mode, format=fmt,
                                  quantity=quantity)

        def rnd():
            ctx.render(sc.camera, W, H, sc.step_vox, out=out, ert=sc.ert, bg=sc.bg)
        for _ in range(warmup):
            bld()
            rnd()
        sweep_ms, march_ms = timed_frames(ctx, bld, rnd, flush, steps)
        img = out.cpu().numpy().astype(np.float64)[y0:y0 + 144, x0:x0 + 256].reshape(-1, 4)
        err = np.abs(img - (depth_ref if quantity == vi.OPTICAL_DEPTH else refs[mode]))
        rows[f"{mname}-{names[fmt]}"] = {
            "frames_per_s": round(1000.0 / (sweep_ms + march_ms), 2),
            "sweep_ms": round(sweep_ms, 4), "march_ms": round(march_ms, 4),
            "max_abs_err_rgba": [float(f"{v:.3g}") for v in err.max(axis=0)],
            "mean_abs_err_rgba": [float(f"{v:.3g}") for v in err.mean(axis=0)]}
    for mname in tuple(modes) + (("cone-depth",) if depth else ()):
        base = rows[f"{mname}-f32"]["frames_per_s"]
        for fmt in names.values():
            if f"{mname}-{fmt}" in rows:
                rows[f"{mname}-{fmt}"]["gain_vs_f32"] = round(
                    rows[f"{mname}-{fmt}"]["frames_per_s"] / base, 3)
    ctx.close()
    del out, flush
    torch.cuda.empty_cache()
    return sc.name, oracle_s, rows


def precision_summary(args):
    """The headline line's precision figures: the 512^3 blob cone frames in each
    storage format, their max error per RGBA channel against the FP64 oracle
    (256x144 crop) and their frame rate against FP32."""
    import oracle
    name, oracle_s, rows = precision_rows(max(3, min(args.steps, 10)), 3, modes=("cone",),
                                          depth=False)
    return {"scene": name, "error_reference": f"FP64 oracle, centred 256x144 crop "
                                              f"({oracle_s:.1f} s on {oracle.threads()} cores)",
            "formats": {k: {"max_abs_err_rgba": v["max_abs_err_rgba"],
                            "frames_per_s": v["frames_per_s"],
                            "gain_vs_f32": v["gain_vs_f32"]} for k, v in rows.items()}}


def precision_workload(args):
    """Storage formats FP32 / FP16 / BF16 / UNORM16 on the 512^3 blob scene:
    frames/s of each and its per-channel error against the FP64 oracle on the
    centred 256x144 crop (the oracle builds its own FP64 stack)."""
    import oracle
    name, oracle_s, rows = precision_rows(args.steps, args.warmup)
    print(json.dumps({"workload": "precision", "metric": "frames/s", "unit": "frames/s",
                      "scene": name, "steps": args.steps, "warmup": args.warmup,
                      "error_reference": "FP64 oracle, centred 256x144 crop "
                                         f"({oracle_s:.1f} s on {oracle.threads()} cores)",
                      "results": rows}), flush=True)


def scalability_workload(args):
    """Frame cost over slice counts {64, 128, 256} x slice resolutions {128, 256,
    512}^2 on the 256^3 CT phantom at a 512x512 viewport, shell and cone."""
    import numpy as np
    import torch

    from paper_2008_06134_gb300 import build, phantoms as ph, vi
    build.build()
    sc = ph.ct256_cone()
    ctx = vi.Context(0)
    ctx.load_volume(torch.from_numpy(sc.volume.view(np.int16)).cuda(), dtype=vi.U16)
    ctx.set_transfer_function(sc.tf, sc.vmin, sc.vmax)
    ctx.set_light(sc.light_dir, sc.light_color)
    W = H = 512
    out = torch.empty((H, W, 4), dtype=torch.float32, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    rows = []
    for mode, mname in ((vi.SHELL, "shell"), (vi.CONE, "cone")):
        for n in (64, 128, 256):
            for R in (128, 256, 512):
                def bld():
                    ctx.build_attenuation(n, R, mode)

                def rnd():
                    ctx.render(sc.camera, W, H, sc.step_vox, out=out, ert=sc.ert, bg=sc.bg)
                for _ in range(args.warmup):
                    bld()
                    rnd()
                sweep_ms, march_ms = timed_frames(ctx, bld, rnd, flush, args.steps)
                rows.append({"mode": mname, "slices": n, "slice_res": R,
                             "sweep_ms": round(sweep_ms, 4), "march_ms": round(march_ms, 4),
                             "frame_ms": round(sweep_ms + march_ms, 4)})
    print(json.dumps({"workload": "scalability", "scene": "ct256-u16, 512x512 perspective, "
                      "step 0.5, ERT 0.99", "steps": args.steps, "rows": rows}), flush=True)
    ctx.close()


def variants_workload(args):
    """Frame cost of each option on the headline scene (256^3 CT phantom, 256
    slices of 512^2, 1024^2 perspective, step 0.5, ERT 0.99): the directional
    cone as benchmarked, the optical-depth stack (Eq. 5-6), linear filtering
    between slices, one to four shells, and a point light 1.5 and 3 units from
    the centre along the benchmark's light direction."""
    import numpy as np
    import torch

    from paper_2008_06134_gb300 import build, phantoms as ph, vi
    build.build()
    sc = ph.ct256_cone()
    ctx = vi.Context(0)
    ctx.load_volume(torch.from_numpy(sc.volume.view(np.int16)).cuda(), dtype=vi.U16)
    ctx.set_transfer_function(sc.tf, sc.vmin, sc.vmax)
    W, H = sc.width, sc.height
    out = torch.empty((H, W, 4), dtype=torch.float32, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    L = np.asarray(sc.light_dir, np.float64)
    L = L / np.linalg.norm(L)
    cases = [("cone (benchmark)", vi.CONE, {}, {}, None),
             ("cone optical-depth", vi.CONE, {"quantity": vi.OPTICAL_DEPTH}, {}, None),
             ("cone linear-slices", vi.CONE, {}, {"slice_filter": vi.SLICE_LINEAR}, None),
             ("shadow", vi.SHADOW, {}, {}, None),
             ("shell 1", vi.SHELL, {}, {}, None),
             ("shell 2", vi.SHELL, {"shell_count": 2}, {}, None),
             ("shell 4", vi.SHELL, {"shell_count": 4}, {}, None),
             ("cone point-light 1.5", vi.CONE, {}, {}, 0.5 - 1.5 * L),
             ("cone point-light 3", vi.CONE, {}, {}, 0.5 - 3.0 * L),
             ("shadow point-light 1.5", vi.SHADOW, {}, {}, 0.5 - 1.5 * L)]
    rows = []
    for name, mode, bopts, ropts, pos in cases:
        if pos is None:
            ctx.set_light(sc.light_dir, sc.light_color)
        else:
            ctx.set_point_light(pos, sc.light_color)

        def bld():
            ctx.build_attenuation(sc.n_slices, sc.slice_res, mode,
                                  cone_half_angle_deg=sc.cone_half_angle_deg, **bopts)

        def rnd():
            ctx.render(sc.camera, W, H, sc.step_vox, out=out, ert=sc.ert, bg=sc.bg, **ropts)
        for _ in range(args.warmup):
            bld()
            rnd()
        sweep_ms, march_ms = timed_frames(ctx, bld, rnd, flush, args.steps)
        rows.append({"case": name, "sweep_ms": round(sweep_ms, 4), "march_ms": round(march_ms, 4),
                     "frames_per_s": round(1000.0 / (sweep_ms + march_ms), 1)})
    print(json.dumps({"workload": "variants", "scene": "ct256-u16, 256x512^2 FP32, 1024^2 "
                      "perspective, step 0.5, ERT 0.99", "steps": args.steps, "rows": rows}),
          flush=True)
    ctx.close()


def large_workload(args):
    """The large-volume workload (see large_result), one JSON line."""
    print(json.dumps(large_result(args, args.steps, args.warmup)), flush=True)


def large_result(args, steps, warmup):
    """The large-volume workload: 1024^3 uint16 CT phantom (2 GiB, generated on
    the device), 1024 slices of 2048^2 stored FP16 (8 GiB), cone, 3840 x 2160
    perspective, step 0.5, ERT 0.99.  Frames/s, samples/s and the sweep's
    achieved bandwidth over its algorithmic bytes (volume read once + stack
    written once = 10.74 GB)."""
    import torch

    from paper_2008_06134_gb300 import build, phantoms as ph, vi
    build.build()
    t0 = time.perf_counter()
    vol = ph.ct_phantom_device(args.large_n, 5)
    gen_s = time.perf_counter() - t0
    drng = ph._child(5, 2)
    light, view = ph.random_direction(drng), ph.random_direction(drng)
    cam = ph.orbit_camera(view, perspective=True, distance=2.6, fovy_deg=40.0)
    tf = ph.tf_ct(4096, 5)
    n, R = args.large_slices, args.large_res
    W, H = (int(x) for x in args.large_image.split("x"))
    ctx = vi.Context(0)
    ctx.load_volume(vol, dtype=vi.U16)
    ctx.set_transfer_function(tf, 0.0, 4095.0)
    ctx.set_light(light)
    out = torch.empty((H, W, 4), dtype=torch.float32, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")

    def bld():
        ctx.build_attenuation(n, R, vi.CONE, format=vi.F16)

    def rnd(**kw):
        ctx.render(cam, W, H, 0.5, out=out, ert=0.99, **kw)
    counts = torch.zeros((H, W), dtype=torch.int32, device="cuda")
    bld()
    rnd(sample_counts=counts)
    torch.cuda.synchronize()
    samples = int(counts.sum().item())
    del counts
    for _ in range(warmup):
        bld()
        rnd()
    sweep_ms, march_ms = timed_frames(ctx, bld, rnd, flush, steps)
    sweep_bytes = vol.numel() * 2 + n * R * R * 2
    peaks, _ = measured_peaks()
    hbm = peaks.get("hbm_gbs") or 6800.0
    ctx.close()
    del vol, out, flush
    torch.cuda.empty_cache()
    return {"workload": "large", "metric": "frames/s", "unit": "frames/s",
            "scene": f"ct{args.large_n}-u16 (device-generated, seed 5), {n}x{R}^2 FP16, "
                     f"cone 15, {W}x{H} perspective, step 0.5, ERT 0.99",
            "steps": steps, "warmup": warmup,
            "frames_per_s": round(1000.0 / (sweep_ms + march_ms), 2),
            "sweep_ms": round(sweep_ms, 4), "march_ms": round(march_ms, 4),
            "samples_per_frame": samples,
            "gsamples_per_s": round(samples / ((sweep_ms + march_ms) * 1e6), 2),
            "march_gsamples_per_s": round(samples / (march_ms * 1e6), 2),
            "sweep_algorithmic_bytes": sweep_bytes,
            "sweep_gbs": round(sweep_bytes / (sweep_ms * 1e6), 1),
            "sweep_frac_of_measured_hbm": round(sweep_bytes / (sweep_ms * 1e6) / hbm, 3),
            "volume_generation_s": round(gen_s, 2)}


def oracle_workload(args):
    """The FP64 oracle timed on this host's cores beside the GPU, scene by scene:
    the 64^3 blob scene (shell) and the 256^3 CT scene (shadow and cone) on
    whole frames, the 512^3 precision scene (shell and cone) and the 1024^3
    large scene (cone) on their centred 256 x 144 crops.  The oracle's sweep
    always builds the whole FP64 stack (a crop's rays can look up any of it).
    Per scene and mode: the oracle's sweep and render seconds, its samples and
    Gsamples/s; the GPU's sweep and march ms and Gsamples/s on the whole frame
    (5 timed frames, L2 flushed); and the ratio of the two sample rates."""
    import numpy as np
    import torch

    import oracle
    from paper_2008_06134_gb300 import build, phantoms as ph, vi
    build.build()
    oracle.build()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    scenes = [(ph.blob64_shell, (vi.SHELL,), None), (ph.ct256_cone, (vi.SHADOW, vi.CONE), None),
              (ph.blob512_precision, (vi.SHELL, vi.CONE), (256, 144)),
              (ph.ct1024_large, (vi.CONE,), (256, 144))]
    rows = []
    for make, modes, crop in scenes:
        sc = make()
        W, H = sc.width, sc.height
        gpu = {}
        with vi.Context(0) as ctx:
            ctx.load_volume(sc.volume)
            ctx.set_transfer_function(sc.tf, sc.vmin, sc.vmax)
            ctx.set_light(sc.light_dir, sc.light_color)
            out = torch.empty((H, W, 4), dtype=torch.float32, device="cuda")
            for mode in modes:
                def bld():
                    ctx.build_attenuation(sc.n_slices, sc.slice_res, mode, format=sc.fmt,
                                          cone_half_angle_deg=sc.cone_half_angle_deg,
                                          shell_radius_vox=sc.shell_radius_vox)

                def rnd(**kw):
                    ctx.render(sc.camera, W, H, sc.step_vox, out=out, ert=sc.ert, bg=sc.bg, **kw)
                counts = torch.zeros((H, W), dtype=torch.int32, device="cuda")
                bld()
                rnd(sample_counts=counts)
                torch.cuda.synchronize()
                samples = int(counts.sum().item())
                del counts
                for _ in range(3):
                    bld()
                    rnd()
                sweep_ms, march_ms = timed_frames(ctx, bld, rnd, flush, 5)
                gpu[mode] = (sweep_ms, march_ms, samples)
        del out
        torch.cuda.empty_cache()
        if crop:
            cw, ch = crop
            ys, xs = np.mgrid[(H - ch) // 2:(H + ch) // 2, (W - cw) // 2:(W + cw) // 2]
        else:
            ys, xs = np.mgrid[0:H, 0:W]
        xs, ys = xs.ravel(), ys.ravel()
        t0 = time.perf_counter()
        light = oracle.light_setup(sc.light_dir, sc.n_slices, sc.slice_res)
        stack = oracle.build_stack(sc.volume, sc.tf, sc.vmin, sc.vmax, light)
        sweep_s = time.perf_counter() - t0
        for mode in modes:
            ro = oracle.render_opts(mode, sc.step_vox, sc.ert, sc.bg, sc.light_color,
                                    cone_half_angle_deg=sc.cone_half_angle_deg,
                                    shell_radius_vox=sc.shell_radius_vox)
            t0 = time.perf_counter()
            ns = oracle.render_pixels(sc.volume, sc.tf, sc.vmin, sc.vmax, light, stack,
                                      sc.camera, W, H, ro, xs, ys)[3]
            render_s = time.perf_counter() - t0
            o_samples = int(ns.sum())
            sweep_ms, march_ms, samples = gpu[mode]
            o_rate = o_samples / render_s / 1e9
            g_rate = samples / (march_ms * 1e6)
            rows.append({"scene": sc.name, "mode": ["none", "shadow", "shell", "cone"][mode],
                         "oracle": {"pixels": int(xs.size), "sweep_s": round(sweep_s, 2),
                                    "render_s": round(render_s, 3), "samples": o_samples,
                                    "gsamples_per_s": round(o_rate, 5)},
                         "gpu": {"pixels": W * H, "stack": ["f32", "f16", "bf16", "unorm16"][sc.fmt],
                                 "sweep_ms": round(sweep_ms, 4), "march_ms": round(march_ms, 4),
                                 "samples": samples, "gsamples_per_s": round(g_rate, 2)},
                         "march_sample_rate_ratio": round(g_rate / o_rate, 1),
                         "sweep_time_ratio": round(sweep_s * 1e3 / sweep_ms, 1)})
        del stack, sc
    print(json.dumps({"workload": "oracle", "cores": oracle.threads(), "cpu": cpu_model(),
                      "note": "oracle FP64 on whole frames (64^3, 256^3) or the centred "
                              "256x144 crop (512^3, 1024^3); GPU on whole frames",
                      "rows": rows}), flush=True)


def serving_setup(args):
    """The serving mix: the registered volumes in pinned host memory,
    the request streams per Poisson rate, and run(slots, fmt, burst, reqs,
    graphs, batching), which serves one stream on a fresh server and returns
    (row of frames/s and latency percentiles, frames)."""
    import numpy as np
    import torch
    from concurrent.futures import ThreadPoolExecutor

    from paper_2008_06134_gb300 import build, phantoms as ph, vi
    build.build()
    specs = ph.serving_volumes()
    t_gen = time.perf_counter()
    with ThreadPoolExecutor(len(specs)) as ex:
        arrays = list(ex.map(lambda v: v.generate(), specs))
    t_gen = time.perf_counter() - t_gen
    host = [torch.from_numpy(a.view(np.int16) if a.dtype == np.uint16 else a).pin_memory()
            for a in arrays]
    codes = [vi.U8 if a.dtype == np.uint8 else vi.U16 for a in arrays]
    rates = [float(r) for r in str(args.rate).split(",")]
    mixes = {r: ph.serving_requests(len(specs), args.requests, r) for r in rates}
    budget = int(args.budget_gib * (1 << 30))

    def submit(s, vids, q, out, fmt):
        v = specs[q["volume"]]
        return s.submit(vids[q["volume"]], v.tf, v.vmin, v.vmax, q["light_dir"], q["n_slices"],
                        q["slice_res"], q["mode"], q["camera"], q["width"], q["height"],
                        q["step_vox"], out, format=fmt, ert=q["ert"])

    def run(slots, fmt, burst, reqs, graphs=False, batching=False, eviction=vi.EVICT_COST):
        outs = [torch.empty((q["height"], q["width"], 4), device="cuda") for q in reqs]
        with vi.Server(0, slots=slots, memory_budget=budget, max_resident_volumes=6,
                       graphs=graphs, batching=batching, eviction=eviction) as s:
            vids = [s.add_volume(h, c) for h, c in zip(host, codes)]
            warm = torch.empty((64, 64, 4), device="cuda")
            for i in range(len(specs)):           # untimed: load every volume once
                q = dict(reqs[i % len(reqs)], volume=i, width=64, height=64)
                assert s.wait(submit(s, vids, q, warm, fmt), 600000.0)[0] == vi.REQ_DONE
            torch.cuda.synchronize()
            base = s.stats()
            t0 = time.perf_counter()
            tickets = []
            for q, out in zip(reqs, outs):
                if not burst:
                    delay = t0 + q["arrival_s"] - time.perf_counter()
                    if delay > 0:
                        time.sleep(delay)
                tickets.append(submit(s, vids, q, out, fmt))
            results = [s.wait(t, 600000.0) for t in tickets]
            times = np.array([s.timing(t) for t in tickets])
            st = s.stats()
        failed = sum(r != (vi.REQ_DONE, vi.OK) for r in results)
        lat = times[:, 2] - times[:, 0]
        span_s = (times[:, 2].max() - times[:, 0].min()) / 1000.0
        row = {"frames_per_s": round(len(reqs) / span_s, 1),
               "latency_ms": {"p50": round(float(np.percentile(lat, 50)), 3),
                              "p99": round(float(np.percentile(lat, 99)), 3),
                              "mean": round(float(lat.mean()), 3),
                              "max": round(float(lat.max()), 3)},
               "queue_wait_ms_p50": round(float(np.percentile(times[:, 1] - times[:, 0], 50)), 3),
               "service_ms": {"p50": round(float(np.percentile(times[:, 2] - times[:, 1], 50)), 3),
                              "p99": round(float(np.percentile(times[:, 2] - times[:, 1], 99)), 3)},
               "failed": failed,
               "volume_loads": st["volume_loads"] - base["volume_loads"],
               "volume_load_mib": round((st["volume_load_bytes"] - base["volume_load_bytes"])
                                        / float(1 << 20), 1),
               "volume_evictions": st["volume_evictions"] - base["volume_evictions"],
               "stack_reuses": st["stack_reuses"] - base["stack_reuses"],
               "peak_bytes": st["peak_bytes"]}
        if graphs:
            row["graph_launches"] = st["graph_launches"] - base["graph_launches"]
            row["graph_instantiations"] = st["graph_instantiations"]
        if batching:
            row["batches"] = st["batches"] - base["batches"]
            row["batched_frames"] = st["batched_frames"] - base["batched_frames"]
        return row, outs

    return dict(specs=specs, rates=rates, mixes=mixes, budget=budget, run=run, t_gen=t_gen)


def serving_summary(args):
    """The headline line's serving figures: 512 requests of the serving mix at
    300/s and at 800/s, the plain path (one slot, one frame at a time, FP32
    stacks) against the served reduced-precision path (8 slots, FP16 stacks;
    at 800/s also with batched marches), with the served frames' max error
    against the plain FP32 frames.  Volumes are evicted by reload cost
    (GreedyDual, the server's default)."""
    import torch
    from paper_2008_06134_gb300 import vi
    a = argparse.Namespace(**vars(args))
    a.rate, a.requests, a.slots = "300,800", 512, 8
    sv = serving_setup(a)
    out = {"requests": 512, "rates_per_s": [300, 800], "slots": 8, "budget_gib": a.budget_gib,
           "max_resident_volumes": 6, "eviction": "reload cost (GreedyDual)"}
    keys = ("frames_per_s", "latency_ms", "failed", "volume_loads", "volume_load_mib")
    beats = {}
    for rate in (300, 800):
        reqs = sv["mixes"][float(rate)]
        plain, plain_outs = sv["run"](1, vi.F32, False, reqs)
        out[f"plain-f32-1slot-{rate}"] = {k: plain[k] for k in keys}
        arms = [("served-f16-8slots", False)] + ([("served-f16-8slots-batched", True)]
                                                  if rate == 800 else [])
        for name, batching in arms:
            row, outs = sv["run"](8, vi.F16, False, reqs, batching=batching)
            err = max(float((x - y).abs().max()) for x, y in zip(outs, plain_outs))
            out[f"{name}-{rate}"] = {k: row[k] for k in keys}
            out[f"{name}-{rate}"]["max_abs_err_vs_plain_f32"] = float(f"{err:.3g}")
            del outs
        beats[rate] = (out[f"served-f16-8slots-{rate}"]["latency_ms"]["p99"]
                       <= out[f"plain-f32-1slot-{rate}"]["latency_ms"]["p99"])
        del plain_outs
    out["served_f16_beats_plain_f32_p99"] = {f"{r}/s": b for r, b in beats.items()}
    torch.cuda.empty_cache()
    return out


def serving_workload(args):
    """The render server on the serving mix: 8 registered volumes ({128, 256,
    512}^3, uint8 blobs and uint16 CT ellipsoids) with at most 6 resident under
    a fixed HBM budget, and a seeded stream of requests (256^2 to 1920x1080,
    64-512 slices of 256^2 or 512^2, shadow / shell / cone, light and view
    uniform on the sphere).  Runs: one slot with FP32 stacks (one frame at a
    time: the plain path), and `--slots` concurrent slots with FP32 and with
    FP16 stacks, each under Poisson arrivals at `--rate` and as one burst; the
    FP32 served runs again with each request's device work launched as one
    CUDA graph, and the served runs with batched marches.  Every run evicts
    volumes by their reload cost (GreedyDual); the plain run and the served
    FP16 run are repeated with least-recently-used eviction.
    Reports per run frames/s and request latency (submission to completion)
    percentiles; the FP32 served frames are compared with the plain ones."""
    import torch
    from paper_2008_06134_gb300 import vi
    sv = serving_setup(args)
    specs, rates, mixes, budget, run = (sv["specs"], sv["rates"], sv["mixes"], sv["budget"],
                                        sv["run"])
    t_gen = sv["t_gen"]

    runs = {}
    for rate in rates:
        reqs = mixes[rate]
        plain, plain_outs = run(1, vi.F32, False, reqs)
        runs[f"plain-f32-1slot-poisson{rate:g}"] = plain
        for fmt, fname in ((vi.F32, "f32"), (vi.F16, "f16")):
            row, outs = run(args.slots, fmt, False, reqs)
            if fmt == vi.F32:
                row["frames_identical_to_plain"] = sum(bool(torch.equal(a, b))
                                                       for a, b in zip(outs, plain_outs))
            else:
                err = max(float((a - b).abs().max()) for a, b in zip(outs, plain_outs))
                row["max_abs_err_vs_plain_f32"] = float(f"{err:.3g}")
            runs[f"served-{fname}-{args.slots}slots-poisson{rate:g}"] = row
            del outs
        # Least-recently-used eviction in place of the reload-cost order.
        row, _ = run(1, vi.F32, False, reqs, eviction=vi.EVICT_LRU)
        runs[f"plain-f32-1slot-lru-poisson{rate:g}"] = row
        row, outs = run(args.slots, vi.F16, False, reqs, eviction=vi.EVICT_LRU)
        runs[f"served-f16-{args.slots}slots-lru-poisson{rate:g}"] = row
        del outs
        # The same FP32 runs with each request's device work as one CUDA graph.
        row, outs = run(args.slots, vi.F32, False, reqs, graphs=True)
        row["frames_identical_to_plain"] = sum(bool(torch.equal(a, b))
                                               for a, b in zip(outs, plain_outs))
        runs[f"served-f32-graphs-{args.slots}slots-poisson{rate:g}"] = row
        del outs
        # Batched marches: the requests admitted together march as one batch.
        for fmt, fname in ((vi.F32, "f32"), (vi.F16, "f16")):
            row, outs = run(args.slots, fmt, False, reqs, batching=True)
            if fmt == vi.F32:
                row["frames_identical_to_plain"] = sum(bool(torch.equal(a, b))
                                                       for a, b in zip(outs, plain_outs))
            else:
                err = max(float((a - b).abs().max()) for a, b in zip(outs, plain_outs))
                row["max_abs_err_vs_plain_f32"] = float(f"{err:.3g}")
            runs[f"served-{fname}-batched-{args.slots}slots-poisson{rate:g}"] = row
            del outs
        del plain_outs
    # Capacity: every request of the first mix submitted at once.
    for slots, name, fmt, graphs, batching in (
            (1, "plain-f32-1slot-burst", vi.F32, False, False),
            (args.slots, f"served-f32-{args.slots}slots-burst", vi.F32, False, False),
            (args.slots, f"served-f16-{args.slots}slots-burst", vi.F16, False, False),
            (args.slots, f"served-f32-graphs-{args.slots}slots-burst", vi.F32, True, False),
            (args.slots, f"served-f32-batched-{args.slots}slots-burst", vi.F32, False, True),
            (args.slots, f"served-f16-batched-{args.slots}slots-burst", vi.F16, False, True)):
        runs[name] = run(slots, fmt, True, mixes[rates[0]], graphs=graphs, batching=batching)[0]
    print(json.dumps({"workload": "serving", "metric": "frames/s", "unit": "frames/s",
                      "requests": args.requests, "rates_per_s": rates, "slots": args.slots,
                      "budget_bytes": budget, "max_resident_volumes": 6,
                      "volumes": [v.name for v in specs],
                      "mix": "256^2..1920x1080 perspective, 64-512 slices of 256^2/512^2, "
                             "shadow/shell/cone, light and view uniform, step 0.5, ERT 0.99",
                      "volume_generation_s": round(t_gen, 1), "runs": runs}), flush=True)


def main():
    args = parse()
    if args.cpu_baseline_only:
        from paper_2008_06134_gb300 import phantoms as ph
        print(json.dumps(cpu_baseline(ph.ct256_cone())), flush=True)
    elif args.impl == "reference":
        reference_arm(args)
    elif args.workload == "precision":
        precision_workload(args)
    elif args.workload == "scalability":
        scalability_workload(args)
    elif args.workload == "serving":
        serving_workload(args)
    elif args.workload == "variants":
        variants_workload(args)
    elif args.workload == "large":
        large_workload(args)
    elif args.workload == "oracle":
        oracle_workload(args)
    else:
        gb300_arm(args)


if __name__ == "__main__":
    main()
