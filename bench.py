"""Benchmark of the GB300 depth stage: depth frames/s on the 1280x720, D=128,
7x7-census, 8-path workload (one rectified pair per step, plain path).

    python bench.py [--gpus N --steps K --warmup W] [--impl reference]

Prints ONE JSON line (rank 0).  ``value`` is device-timed whole-job
throughput with the inputs resident in HBM; ``e2e`` is the same metric
through the host-buffer C-ABI call (pinned host -> device copies, compute,
depth copied back and read on the host, every step), with 2-4 frames in
flight on as many handles and streams as a camera stream runs it (the figure
for each number of frames in flight, one included, is in the same object); ``roofline`` reports the dominant kernel's
achieved integer-op rate (algorithmic ops / its CUDA-event duration) against
the derived INT32 peak; ``cpu_baseline`` is the CPU oracle timed on a bounded
sample on this host.  ``--impl reference`` times that oracle alone, on the
same workload and metric (the paper's own SimSense implementation is not
public code, so the oracle is the reference arm).

Under torchrun each rank runs an independent replica on its own GPU (pairs
are independent; no data-path collective); the value divides all ranks'
frames by the slowest rank's time.
"""
from __future__ import annotations

import argparse
import dataclasses
import datetime
import json
import os
import shutil
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2201_11924_gb300 import configs, replicas, scenes  # noqa: E402

METRIC = "depth_frames_per_s"
UNIT = "frames/s"
N_SM_NOMINAL = 152
INT32_LANES_PER_SM = 128          # INT32 results per clock per SM
SM_MAX_MHZ = 2070.0


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            return json.load(fh), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "sm_max_mhz": SM_MAX_MHZ}, "fallback"


# Measured issue rates of this GPU (probes/op_rates.cu, results per clock per
# SM): a 32-bit integer add and a 32-bit minimum.
MEASURED_ADD_PER_CLK_SM = 124
MEASURED_MIN_PER_CLK_SM = 64


def roofline_object(wl, stage_ms, n_prof, n_sm, peaks, peak_src):
    """The bench line's roofline for the dominant kernel: its algorithmic
    integer ops over its live duration (stage_ms summed over n_prof steps)
    against the derived INT32 peak, with the measured add and minimum rates
    and, where an ncu capture of the current source exists, its DRAM bytes
    against the HBM peak."""
    ops = algorithmic_ops(wl)
    dom = max(stage_ms, key=stage_ms.get)
    launch_s = stage_ms[dom] / 1e3 / max(1, n_prof)
    sm_max = float(peaks.get("sm_max_mhz", SM_MAX_MHZ))
    int_peak = n_sm * INT32_LANES_PER_SM * sm_max * 1e6 / 1e12        # T ops/s
    achieved = ops[dom] / launch_s / 1e12
    add_peak = n_sm * MEASURED_ADD_PER_CLK_SM * sm_max * 1e6 / 1e12
    min_peak = n_sm * MEASURED_MIN_PER_CLK_SM * sm_max * 1e6 / 1e12
    roofline = {"bound": "alu", "kernel": dom, "achieved": achieved, "peak": int_peak,
                "unit": "Tops/s", "frac": achieved / int_peak, "traffic": measured_traffic(wl, dom),
                "traffic_unit": "bytes per launch (ncu dram read + write)",
                "peak_source": f"derived: {n_sm} SMs x {INT32_LANES_PER_SM} INT32 lanes x {sm_max:.0f} MHz",
                "peak_measured": {"add_tops": add_peak, "min_tops": min_peak,
                                  "frac_of_add": achieved / add_peak,
                                  "source": "probes/op_rates.cu: 124 adds and 64 minima per clock per SM"},
                "stage_ms_per_step": {k: v / max(1, n_prof) for k, v in stage_ms.items()},
                "hbm_algorithmic_bytes_per_frame": algorithmic_bytes(wl),
                "hbm_peak_gbs": float(peaks.get("hbm_gbs", 6800.0)), "hbm_peak_source": peak_src}
    total, per = dram_bytes_per_frame(wl)
    roofline["dram_bytes_per_frame"] = total
    roofline["dram_bytes_per_kernel"] = per
    if total is not None:
        # the whole frame's measured traffic at the copy peak: the shortest
        # time these bytes allow, against the measured time of the stages
        frame_s = sum(stage_ms.values()) / 1e3 / max(1, n_prof)
        roofline["dram_gbs_per_frame_time"] = total / frame_s / 1e9
        roofline["dram_bound_frames_per_s"] = roofline["hbm_peak_gbs"] * 1e9 / total
    if roofline["traffic"] is not None:
        # the same launch against the HBM roof: its measured DRAM bytes over
        # its live duration (how close its actual traffic runs to the copy peak)
        roofline["traffic_gbs"] = roofline["traffic"] / launch_s / 1e9
        roofline["traffic_frac_of_hbm_peak"] = roofline["traffic_gbs"] / roofline["hbm_peak_gbs"]
    return roofline


def algorithmic_ops(wl):
    """Scalar integer ops per launch of each kernel (no SIMD credit).

    Per cell (x, y, d): the Hamming cost once (XOR, POPC on 64-bit codes:
    5 ops; on 32-bit codes: 2; the cost kernel), 7 ops per path for the
    recurrence (min of the neighbours, +P1, min with L'(d), -m', min with P2,
    +C, the min-reduction over d; the path kernel), then in the selection
    kernel the sum over the paths (1 per path) and 6 for WTA, uniqueness and
    the right-view argmin.  The census costs 2 ops per bit per view and
    pixel.  The sum over the stages is the per-cell count cost + 8 P + 6 +
    4 nbits / D."""
    cells = wl.W * wl.H * wl.D
    cost = 5 if wl.nbits > 32 else 2
    bw, bh = getattr(wl, "block", (1, 1))
    if bw * bh > 1:
        cost += bw * bh + 1          # SGBM: the block sum and the rounded division
    k = getattr(wl, "median", 0)
    # sensor noise: per pixel and view one Philox4x64-10 block (10 rounds of
    # two 64-bit products and four xor/adds: ~80 integer ops) and ~20 ops of
    # Box-Muller, rejection test and the affine model
    noise = 2 * wl.W * wl.H * 100 if getattr(wl, "noise", False) else 0
    return {
        "census": wl.W * wl.H * 4 * wl.nbits + noise,
        "cost": cells * cost,
        "paths": cells * 7 * wl.paths,
        "select": cells * (wl.paths + 6) + wl.W * wl.H * k * k * (k * k // 2 + 1) * (2 if k else 0),
    }


# DRAM bytes (read, write) of one launch of each kernel, from one one-pass
# ncu capture of the dram__bytes counters over the four kernels of a frame,
# with the SHA-1 of each kernel's source at the time: a kernel whose source
# has changed since reports null.
# Per-kernel DRAM bytes of one launch (read, write) from a one-pass ncu
# capture of the default workload, keyed on the SHA-1 of the kernel's sources
# (its .cu file and the device headers it includes, concatenated in this
# order) at the time of the capture: a kernel whose sources changed since
# reports None.
KERNEL_SOURCES = {
    "census": ("paper_2201_11924_gb300/csrc/census.cu",),
    "cost": ("paper_2201_11924_gb300/csrc/cost.cu",),
    "paths": ("paper_2201_11924_gb300/csrc/sgm_paths.cu", "paper_2201_11924_gb300/csrc/sgm_walk.cuh",
              "paper_2201_11924_gb300/csrc/simd.cuh"),
    "select": ("paper_2201_11924_gb300/csrc/sgm_select.cu", "paper_2201_11924_gb300/csrc/sgm_row.cuh"),
}
MEASURED_DRAM = {
    "1280x720_D128_census7x7_8path": {
        "census": (1855232, 0, "56aba98b2aec52d52bdbada4a33bc0c40c7d6642"),
        "cost": (14918656, 31478016, "75f1f95ce775e3e03b6fdf09f3b42f7ba1b88054"),
        "paths": (565320960, 885341440, "7608e5e1ed7f8a9871ce0a9dd0d139216a1b1cad"),
        "select": (943805184, 2999552, "36b7eada1e28f2e124cfcf2d77d9af6a325dff36"),
    },
}


def kernel_source_sha(kernel):
    """SHA-1 of the kernel's sources, concatenated (None if one is missing)."""
    import hashlib
    h = hashlib.sha1()
    try:
        for src in KERNEL_SOURCES[kernel]:
            with open(os.path.join(ROOT, src), "rb") as fh:
                h.update(fh.read())
    except OSError:
        return None
    return h.hexdigest()


def measured_traffic(wl, kernel):
    """(read + write) DRAM bytes of one launch of `kernel`, or None."""
    ent = MEASURED_DRAM.get(wl.name, {}).get(kernel)
    if not ent:
        return None
    rd, wr, sha = ent
    if kernel_source_sha(kernel) != sha:
        return None
    return rd + wr


def dram_bytes_per_frame(wl):
    """Measured DRAM bytes of all four kernels of a frame (None unless every
    kernel's capture matches its current source)."""
    per = {k: measured_traffic(wl, k) for k in ("census", "cost", "paths", "select")}
    if any(v is None for v in per.values()):
        return None, per
    return sum(per.values()), per


def stage_roofline_frac(wl, ms_per_frame, n_sm, peaks):
    """The whole stage against its roofline: the slower of the algorithmic
    HBM bytes at the measured copy peak and the algorithmic integer ops at the
    derived INT32 peak, over the measured time per frame."""
    sm_max = float(peaks.get("sm_max_mhz", SM_MAX_MHZ))
    int_peak = n_sm * INT32_LANES_PER_SM * sm_max * 1e6                  # ops/s
    bw = float(peaks.get("hbm_gbs", 6800.0)) * 1e9                        # bytes/s
    t_ops = sum(algorithmic_ops(wl).values()) / int_peak
    t_bytes = algorithmic_bytes(wl) / bw
    t_roof = max(t_ops, t_bytes)
    return {"frac": t_roof / (ms_per_frame / 1e3), "roofline_frames_per_s": 1.0 / t_roof,
            "bound": "alu" if t_ops >= t_bytes else "hbm", "t_ops_us": t_ops * 1e6, "t_bytes_us": t_bytes * 1e6}


def batch_roofline_frac(wls, ms_per_batch, n_sm, peaks):
    """A batch of pairs against the sum of its pairs' rooflines."""
    t = 0.0
    for w in wls:
        r = stage_roofline_frac(w, 1.0, n_sm, peaks)          # t_roof = frac * 1 ms
        t += r["frac"] * 1e-3
    return {"frac": t / (ms_per_batch / 1e3), "roofline_ms_per_batch": t * 1e3}


def algorithmic_bytes(wl):
    """HBM bytes per frame the method must move: both views in (2 B/px),
    depth out (4 B/px) and one spilled partial-sum volume between the forward
    and backward path sweeps (uint16 for 8 paths, 2 B written + 2 B read per
    cell; uint8 for 4 paths)."""
    spill = 4 if wl.paths == 8 else 2
    return 6 * wl.W * wl.H + spill * wl.W * wl.H * wl.D


class ClockSampler:
    """nvidia-smi clock/throttle samples while the timed region runs."""
    FIELDS = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, bus_id=None):
        self.proc = None
        self.path = None
        exe = shutil.which("nvidia-smi")
        if not exe:
            return
        fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
        os.close(fd)
        cmd = [exe, f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "100"]
        if bus_id:
            cmd += ["-i", bus_id]
        self.fh = open(self.path, "w")
        self.proc = subprocess.Popen(cmd, stdout=self.fh, stderr=subprocess.DEVNULL)
        t0 = time.time()
        while time.time() - t0 < 5.0:           # wait for the first sample
            if os.path.getsize(self.path) > 0:
                break
            time.sleep(0.05)

    def stop(self, t0, t1):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        rows = []
        with open(self.path) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                    rows.append((ts, float(parts[1]), float(parts[2]), parts[5:9]))
                except ValueError:
                    continue
        os.unlink(self.path)
        inside = [r for r in rows if t0 - 0.05 <= r[0] <= t1 + 0.05] or rows[-3:]
        if not inside:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in inside for i, v in enumerate(r[3]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[1] for r in inside), "sm_max_mhz": max(r[2] for r in inside),
                "reasons": reasons, "samples": len(inside)}


def _bus_id(torch, dev):
    try:
        p = torch.cuda.get_device_properties(dev)
        return f"{p.pci_domain_id:08X}:{p.pci_bus_id:02X}:{p.pci_device_id:02X}.0"
    except Exception:
        return None


def cpu_oracle_rate(wl, pair, budget_s=10.0, strip_rows=90):
    """Oracle cells/s on full-width horizontal strips of the pair (each strip
    is a complete W x strip_rows problem: same per-cell work as the frame)."""
    import oracle
    cells = 0
    t0 = time.perf_counter()
    n = 0
    H = wl.H
    while True:
        y0 = (n * strip_rows) % max(1, H - strip_rows + 1)
        l = pair["left"][y0:y0 + strip_rows]
        r = pair["right"][y0:y0 + strip_rows]
        if wl.noise:
            l = oracle.noise(l, **oracle.D415_NOISE, seed=wl.seed, view=0)[0]
            r = oracle.noise(r, **oracle.D415_NOISE, seed=wl.seed, view=1)[0]
        oracle.compute(l, r, wl.D, wl.win_w, wl.win_h, wl.P1, wl.P2, wl.paths, wl.uniq,
                       wl.lr_max_diff, wl.subpixel, wl.f, wl.baseline, census_cs=wl.census_cs,
                       block=wl.block, median=wl.median)
        cells += wl.W * l.shape[0] * wl.D
        n += 1
        el = time.perf_counter() - t0
        if el >= budget_s:
            break
    return cells / el, n, el


def workload_config(wl):
    """The keys both arms report for a workload."""
    return {"workload": wl.name, "W": wl.W, "H": wl.H, "D": wl.D, "paths": wl.paths,
            "census": f"{wl.win_w}x{wl.win_h}" + (" centre-symmetric" if wl.census_cs else ""),
            "block": f"{wl.block[0]}x{wl.block[1]}", "median": wl.median,
            "sensor_noise": "D415 (Sec. VI-C / VII)" if wl.noise else None,
            "P1": wl.P1, "P2": wl.P2, "uniq": wl.uniq,
            "lr_max_diff": wl.lr_max_diff, "subpixel": wl.subpixel, "seed": wl.seed}


def run_reference(args, wl):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    pair = scenes.make_pair(wl)
    strip = args.ref_strip_rows
    import oracle
    oracle.build()

    def step(i):
        y0 = (i * strip) % max(1, wl.H - strip + 1)
        l, r = pair["left"][y0:y0 + strip], pair["right"][y0:y0 + strip]
        if wl.noise:
            l = oracle.noise(l, **oracle.D415_NOISE, seed=wl.seed, frame=i, view=0)[0]
            r = oracle.noise(r, **oracle.D415_NOISE, seed=wl.seed, frame=i, view=1)[0]
        oracle.compute(l, r, wl.D, wl.win_w, wl.win_h,
                       wl.P1, wl.P2, wl.paths, wl.uniq, wl.lr_max_diff, wl.subpixel, wl.f, wl.baseline,
                       census_cs=wl.census_cs, block=wl.block, median=wl.median)

    for i in range(args.warmup):
        step(i)
    t0 = time.perf_counter()
    for i in range(args.steps):
        step(i)
    el = time.perf_counter() - t0
    cells = args.steps * wl.W * strip * wl.D
    value = cells / el / wl.cells
    sample = f"{wl.W}x{strip} full-width strip of the {wl.W}x{wl.H} pair per step, per-cell rate extrapolated to frames"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic",
        "config": {**workload_config(wl), "path": "CPU oracle, one thread, full-width strips"},
        "cells_per_s": cells / el,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


PAPER_TABLE2_SGM_FPS = {64: 414.51, 96: 326.79, 128: 281.26, 256: 147.13}   # RTX 4090, Table 2
PAPER_TABLE2_SGBM_FPS = {64: 342.24, 96: 268.98, 128: 232.49, 256: 128.56}


def _table2_cameras(W, H):
    """Synthetic raw cameras of a D415-like IR pair (small distortion and
    misalignment, rectified intrinsics f = 0.9 W) and the RGB camera at twice
    the resolution the depth is registered to."""
    f = 0.9 * W
    c = ((W - 1) / 2, (H - 1) / 2)

    def rot(a, b, g):
        ca, sa, cb, sb, cg, sg = np.cos(a), np.sin(a), np.cos(b), np.sin(b), np.cos(g), np.sin(g)
        return (np.array([[cg, -sg, 0], [sg, cg, 0], [0, 0, 1]]) @ np.array([[cb, 0, sb], [0, 1, 0], [-sb, 0, cb]])
                @ np.array([[1, 0, 0], [0, ca, -sa], [0, sa, ca]]))

    def cam(k1, k2, p1, p2, R):
        return [f * 1.002, f, c[0] + 1.5, c[1] - 1.0, k1, k2, p1, p2, 0.0, *rot(*R).ravel(), f, f, c[0], c[1]]

    left = cam(0.08, -0.02, 4e-4, -3e-4, (0.004, -0.003, 0.002))
    right = cam(0.07, -0.015, -2e-4, 5e-4, (-0.003, 0.002, -0.001))
    reg = (f, f, c[0], c[1], 2 * f, 2 * f, 2 * c[0] + 0.5, 2 * c[1] + 0.5, rot(0.001, 0.002, 0.0),
           (0.015, 0.0, 0.0), 2 * W, 2 * H)
    return left, right, reg


def run_table2(args):
    """The workload of the paper's Table 2 (Sec. VI-D): a 960 x 540 pair
    rectified, census (centre-symmetric 7 x 7), four-path SGM, uniqueness,
    sub-pixel, left-right check, 3 x 3 median, depth registered to a
    1920 x 1080 RGB camera; frames/s for D = 64, 96, 128, 256, with the
    per-pixel cost (SGM) and with a 3 x 3 SGBM block cost, like the two
    SimSense columns of the table."""
    import torch
    from paper_2201_11924_gb300 import simsense
    dev = torch.device("cuda", 0)
    by_d = {}
    ms = {}
    for D, block in [(d, b) for d in (64, 96, 128, 256) for b in ((1, 1), (3, 3))]:
        wl = dataclasses.replace(configs.HD_720, name=f"table2_960x540_D{D}", W=960, H=540, D=D, paths=4,
                                 census_cs=True, median=3, block=block, seed=7000 + D)
        pair = scenes.make_pair(wl)
        L = torch.from_numpy(pair["left"]).to(dev)
        R = torch.from_numpy(pair["right"]).to(dev)
        depth = torch.empty((wl.H, wl.W), dtype=torch.float32, device=dev)
        left, right, reg_args = _table2_cameras(wl.W, wl.H)
        reg = simsense.registration_t(*reg_args)
        with simsense.SimSense.from_workload(wl) as m:
            m.set_rectify(left, right)
            for _ in range(args.warmup):
                m.compute(L, R, depth)
                simsense.register_depth(depth, reg)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(args.steps):
                m.compute(L, R, depth)
                simsense.register_depth(depth, reg)
            e1.record()
            torch.cuda.synchronize()
            ms[(D, block)] = e0.elapsed_time(e1) / args.steps
            by_d[(D, block)] = 1e3 / ms[(D, block)]
    sgm = {d: by_d[(d, (1, 1))] for d in (64, 96, 128, 256)}
    sgbm = {d: by_d[(d, (3, 3))] for d in (64, 96, 128, 256)}
    value = sgm[128]
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms[(128, (1, 1))], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": value / PAPER_TABLE2_SGM_FPS[128], "dtype": "int32", "data": "synthetic",
        "config": {"workload": "table2_960x540_D128_csct7x7_sgm4_median3_rectify_register1920x1080",
                   "note": "Table 2 of the paper: RTX 4090 frames/s 281.26 at D = 128 (context, other hardware)",
                   "l2": "no flush: inputs and volumes stay resident between steps (~66 MB of path bytes per frame)"},
        "by_disparity": {str(d): {"sgm_frames_per_s": sgm[d], "paper_rtx4090_sgm_fps": PAPER_TABLE2_SGM_FPS[d],
                                  "sgbm3x3_frames_per_s": sgbm[d], "paper_rtx4090_sgbm_fps": PAPER_TABLE2_SGBM_FPS[d],
                                  "sgm_cells_per_s": sgm[d] * 960 * 540 * d} for d in sgm},
        # per frame of the reported (SGM, D = 128) run: rectify, census, cost,
        # paths, select, median, register (+ one memset)
        "gpu_launches": 7 * args.steps,
    }
    print(json.dumps(line), flush=True)
    return 0


def _sim_scene(seed, W, H):
    """A random analytic scene for the simulated sensor: a back wall, tilted
    rectangles and spheres with random materials (Sec. VI-A)."""
    rng = np.random.default_rng(seed)

    def rect(c, u, v, **m):
        return (1, 0, c, u, v, 0.0, m["albedo"], m["metallic"], m["roughness"], m["transmission"])

    def sph(c, r, **m):
        return (0, 0, c, (0, 0, 0), (0, 0, 0), r, m["albedo"], m["metallic"], m["roughness"], m["transmission"])

    def mat():
        return dict(albedo=rng.uniform(0.2, 1.0), metallic=rng.uniform(0, 0.6), roughness=rng.uniform(0.2, 0.9),
                    transmission=rng.uniform(0, 0.3))
    prims = [rect((0.0, 0.0, 2.0), (2.5, 0.0, 0.0), (0.0, 1.5, 0.0), albedo=0.7, metallic=0.0, roughness=0.8,
                  transmission=0.0)]
    for _ in range(6):
        a, b = rng.uniform(-0.5, 0.5, 2)
        prims.append(rect((rng.uniform(-0.7, 0.7), rng.uniform(-0.4, 0.4), rng.uniform(0.5, 1.8)),
                          (rng.uniform(0.1, 0.4) * np.cos(a), 0.0, rng.uniform(0.1, 0.4) * np.sin(a)),
                          (0.0, rng.uniform(0.1, 0.3) * np.cos(b), rng.uniform(0.1, 0.3) * np.sin(b)), **mat()))
    for _ in range(8):
        prims.append(sph((rng.uniform(-0.7, 0.7), rng.uniform(-0.4, 0.4), rng.uniform(0.4, 1.8)),
                         rng.uniform(0.03, 0.15), **mat()))
    return prims


def run_sim(args):
    """The whole simulated active-stereo sensor on the device: IR rendering of
    an analytic scene with the projector pattern (Sec. VI-A/B), sensor noise
    (Sec. VI-C) and the depth stage (Sec. VI-D); 1280 x 720, D = 128."""
    import torch
    from paper_2201_11924_gb300 import simsense
    wl = dataclasses.replace(configs.HD_720, noise=True)
    W, H = wl.W, wl.H
    f = wl.f
    dev = torch.device("cuda", 0)
    pat = torch.from_numpy(((np.random.default_rng(11).random((H, W)) < 0.15) * 230 + 20).astype(np.uint8)).to(dev)
    prims = _sim_scene(12, W, H)
    ra = dict(W=W, H=H, f=f, cx=(W - 1) / 2, cy=(H - 1) / 2, baseline=wl.baseline, proj=(0.02, 0.0, 0.0), pf=f,
              pcx=(W - 1) / 2, pcy=(H - 1) / 2, power=1.2, ambient=0.04, gain=350.0)
    depth = torch.empty((H, W), dtype=torch.float32, device=dev)
    with simsense.SimSense.from_workload(wl) as m:
        for _ in range(args.warmup):
            l, r = simsense.render_ir(prims, pat, **ra)
            m.compute(l, r, depth)
        torch.cuda.synchronize()
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record()
        for _ in range(args.steps):
            l, r = simsense.render_ir(prims, pat, **ra)
        e1.record()
        for _ in range(args.steps):
            m.compute(l, r, depth)
        e2.record()
        torch.cuda.synchronize()
    render_ms = e0.elapsed_time(e1) / args.steps
    depth_ms = e1.elapsed_time(e2) / args.steps
    value = 1e3 / (render_ms + depth_ms)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": render_ms + depth_ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "int32", "data": "synthetic",
        "config": {"workload": "sim_1280x720_render15prims_noiseD415_D128_census7x7_8path",
                   "l2": "no flush: each step renders and matches a full frame"},
        "render_ms": render_ms, "depth_with_noise_ms": depth_ms,
        # render, noise, census, cost, paths, select per frame
        "gpu_launches": 6 * args.steps,
    }
    print(json.dumps(line), flush=True)
    return 0


def batchmix_measure(steps, warmup, tune_reps=2):
    """The 64-pair batch of uneven sizes ({640x360 D64, 848x480 D96,
    1280x720 D128, 1280x720 D256}, 7x7 census, 8 paths): frames/s of one
    CUDA-graph launch per batch (autotuned per class) against the same pairs
    as 64 sequential plain calls (one handle per size, one call per pair)."""
    import torch
    from paper_2201_11924_gb300 import simsense
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    wls = configs.batch_workloads()
    pairs = [scenes.make_pair(w) for w in wls]
    L = [torch.from_numpy(p["left"]).to(dev) for p in pairs]
    R = [torch.from_numpy(p["right"]).to(dev) for p in pairs]
    Z = [torch.empty((w.H, w.W), dtype=torch.float32, device=dev) for w in wls]
    cells = sum(w.cells for w in wls)
    stream = torch.cuda.current_stream(dev)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    # plain: one handle per size class, 64 calls in sequence
    handles = {}
    for w in wls:
        key = (w.W, w.H, w.D)
        if key not in handles:
            handles[key] = simsense.SimSense.from_workload(w)

    def plain_round():
        for i, w in enumerate(wls):
            handles[(w.W, w.H, w.D)].compute(L[i], R[i], Z[i])
    for _ in range(warmup):
        plain_round()
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(steps):
        plain_round()
    ev1.record(stream)
    torch.cuda.synchronize()
    plain_ms = ev0.elapsed_time(ev1) / steps
    plain_depth = [z.clone() for z in Z]
    for h in handles.values():
        h.close()

    with simsense.SimSenseBatch(wls) as b:
        t0 = time.perf_counter()
        tuning = b.tune(L, R, Z, reps=tune_reps)
        tune_s = time.perf_counter() - t0
        for _ in range(warmup):
            b.compute(L, R, Z)
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(steps):
            b.compute(L, R, Z)
        ev1.record(stream)
        torch.cuda.synchronize()
        batch_ms = ev0.elapsed_time(ev1) / steps
        status = b.device_status()
        same = all(torch.equal(a, z) for a, z in zip(plain_depth, Z))
        schedule = b.get_schedule()
        classes = [dict(b.class_info(c)[0], pairs=b.class_info(c)[1], **tuning[c]) for c in range(b.num_classes())]
        # the other form of the batch, for comparison: per-class launches if
        # the tuner chose the fused launch, else the fused default
        other = dict(schedule, fused=0) if schedule["fused"] else dict(fused=1, prefetch=16, keep_paths=1, lag=1,
                                                                        order=1)
        b.set_schedule(**other)
        for _ in range(warmup):
            b.compute(L, R, Z)
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(steps):
            b.compute(L, R, Z)
        ev1.record(stream)
        torch.cuda.synchronize()
        other_ms = ev0.elapsed_time(ev1) / steps
        same = same and all(torch.equal(a, z) for a, z in zip(plain_depth, Z))
    return {
        "workload": "batch64_mixed_640x360D64_848x480D96_1280x720D128_1280x720D256_census7x7_8path",
        "pairs": len(wls), "cells_per_batch": cells, "steps": steps, "warmup": warmup,
        "value": len(wls) / (batch_ms / 1e3), "unit": UNIT, "ms_per_batch": batch_ms,
        "cells_per_s": cells / (batch_ms / 1e3),
        "plain_value": len(wls) / (plain_ms / 1e3), "plain_ms_per_batch": plain_ms,
        "speedup_vs_plain": plain_ms / batch_ms, "depth_equals_plain": same,
        "schedule": schedule, "other_form": {"schedule": other, "value": len(wls) / (other_ms / 1e3),
                                              "ms_per_batch": other_ms},
        "classes": classes, "tune_s": tune_s, "device_status": status, "graph": True,
        # census and cost per class, then one persistent launch for the paths
        # and selection of every pair (fused), or those two per class
        "gpu_launches_per_batch": 2 * len(classes) + (1 if schedule["fused"] else 2 * len(classes)),
    }


def run_batch(args, wl):
    """--batch-pairs pairs of one workload per batch call, tuned first."""
    import torch
    torch.cuda.set_device(0)
    n_sm = torch.cuda.get_device_properties(0).multi_processor_count
    peaks, _ = _peaks()
    r = batched_measure(wl, args.batch_pairs, args.steps, args.warmup, n_sm, peaks)
    line = {
        "metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": r["ms_per_batch"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {**workload_config(wl), "pairs_per_batch": args.batch_pairs, "graph": True},
        "schedule": r["schedule"], "stage_roofline": r["stage_roofline"], "device_status": r["device_status"],
        "gpu_launches": (3 if r["schedule"]["fused"] else 4) * args.steps,
    }
    print(json.dumps(line), flush=True)
    return 0


def run_batchmix(args):
    r = batchmix_measure(args.steps, args.warmup)
    line = {
        "metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": r["ms_per_batch"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": r["workload"], "pairs": r["pairs"], "cells_per_batch": r["cells_per_batch"],
                   "graph": True, "l2": "no flush: every batch streams ~60 GB of path volumes through HBM"},
        "cells_per_s": r["cells_per_s"], "plain_value": r["plain_value"],
        "plain_ms_per_batch": r["plain_ms_per_batch"], "speedup_vs_plain": r["speedup_vs_plain"],
        "schedule": r["schedule"], "other_form": r["other_form"], "depth_equals_plain": r["depth_equals_plain"],
        "classes": r["classes"], "device_status": r["device_status"],
        "gpu_launches": r["gpu_launches_per_batch"] * args.steps,
    }
    print(json.dumps(line), flush=True)
    return 0


SERVE_WORKLOAD = "serve_1024cams_poisson_50pct848x480D96_40pct1280x720D128_10pct1920x1080D256"


def serve_measure(rate, seconds, sustain, sustain_seconds, slots):
    """Request loop over 1024 cameras (sizes 50% 848x480 D96, 40% 1280x720
    D128, 10% 1920x1080 D256; 7x7 census, 8 paths, uniqueness 15, L/R 1,
    sub-pixel), Poisson arrivals: the continuous-batching server against the
    same trace served one request at a time (the plain per-request path), at
    the offered rate and at a rate below the GPU's capacity.  Latency =
    arrival to depth ready, including the frame upload."""
    import torch
    from paper_2201_11924_gb300 import serve
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    cams = [configs.serve_camera(c) for c in range(1024)]
    frames = {}
    for w in cams:
        key = (w.W, w.H, w.D)
        frames.setdefault(key, [])
        if len(frames[key]) < 2:
            p = scenes.make_pair(w)
            frames[key].append((p["left"], p["right"]))
    srv = serve.DepthServer(cams, frames, slots_per_class=slots, device=dev)
    mean_cells = sum(w.cells for w in cams) / len(cams)
    out = {}
    for tag, r, secs in (("offered", rate, seconds), ("sustainable", sustain, sustain_seconds)):
        for name, seq in (("plain_sequential", True), ("continuous", False)):
            srv.run(serve.poisson_trace(len(cams), 500.0, 0.2, seed=1), sequential=seq)   # warm-up
            trace = serve.poisson_trace(len(cams), r, secs, seed=5999)
            t0 = time.perf_counter()
            done = srv.run(trace, time_limit=secs + 2.0, sequential=seq)
            wall = time.perf_counter() - t0
            st = serve.latency_stats(done, wall, cams)
            st.update({"rate_per_s": r, "offered": len(trace), "offered_per_s": len(trace) / secs,
                       "offered_cells_per_s": len(trace) * mean_cells / secs,
                       "backlog_at_stop": srv.backlog, "wall_s": wall, **srv.stats})
            out[f"{tag}_{name}"] = st
    res = {"workload": SERVE_WORKLOAD, "cameras": len(cams), "rate_per_s": rate, "seconds": seconds,
           "sustainable_rate_per_s": sustain, "sustainable_seconds": sustain_seconds,
           "slots": srv.slot_counts(), "hbm": srv.hbm_summary(), "upload": True, **out}
    srv.close()
    c = out["offered_continuous"]
    res.update({"value": c["served_per_s"], "unit": UNIT, "p50_ms": c["p50_ms"], "p99_ms": c["p99_ms"],
                "served_cells_per_s": c["served_cells_per_s"],
                "speedup_vs_sequential_offered": (c["served_per_s"] / out["offered_plain_sequential"]["served_per_s"]
                                                  if out["offered_plain_sequential"]["served_per_s"] else None),
                "sustainable_p50_ms": out["sustainable_continuous"]["p50_ms"],
                "sustainable_p99_ms": out["sustainable_continuous"]["p99_ms"]})
    return res


def run_serve(args):
    r = serve_measure(args.serve_rate, args.serve_seconds, args.serve_sustain, 3.0, args.serve_slots)
    c = r["offered_continuous"]
    line = {
        "metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": 1, "steps": c["served"],
        "warmup": 1, "ms_per_step": 1e3 / c["served_per_s"] if c["served_per_s"] else None,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic",
        "config": {"workload": SERVE_WORKLOAD, "rate_per_s": args.serve_rate, "seconds": args.serve_seconds,
                   "slots": r["slots"], "upload": True},
        "p50_ms": r["p50_ms"], "p99_ms": r["p99_ms"], "served_cells_per_s": r["served_cells_per_s"],
        "sustainable_p50_ms": r["sustainable_p50_ms"], "sustainable_p99_ms": r["sustainable_p99_ms"],
        "serve": r,
    }
    print(json.dumps(line), flush=True)
    return 0


def batched_measure(wl, nb, batches, warmup, n_sm, peaks, n_pairs=2):
    """Device-timed frames/s of nb pairs of one workload per batch call
    (simsense_batch_*, tuned by the native autotuner first), with the
    whole-stage roofline fraction."""
    import torch
    from paper_2201_11924_gb300 import simsense
    dev = torch.device("cuda", torch.cuda.current_device())
    pairs = [scenes.make_pair(wl, seed=wl.seed + u) for u in range(n_pairs)]
    L = [torch.from_numpy(pairs[i % n_pairs]["left"]).to(dev) for i in range(nb)]
    R = [torch.from_numpy(pairs[i % n_pairs]["right"]).to(dev) for i in range(nb)]
    Z = [torch.empty((wl.H, wl.W), dtype=torch.float32, device=dev) for _ in range(nb)]
    stream = torch.cuda.current_stream(dev)
    with simsense.SimSenseBatch([wl] * nb) as b:
        b.tune(L, R, Z, reps=1)
        schedule = b.get_schedule()
        for _ in range(warmup):
            b.compute(L, R, Z)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(batches):
            b.compute(L, R, Z)
        e1.record(stream)
        torch.cuda.synchronize()
        status = b.device_status()
    ms = e0.elapsed_time(e1) / batches
    return {"pairs_per_batch": nb, "batches": batches, "value": nb * 1e3 / ms, "unit": UNIT,
            "ms_per_batch": ms, "schedule": schedule, "device_status": status,
            "stage_roofline": stage_roofline_frac(wl, ms / nb, n_sm, peaks)}


def plain_measure(wl, steps, warmup, n_sm, peaks, peak_src, n_pairs=2):
    """Device-timed frames/s of the plain call on one workload (inputs
    resident in HBM, a few distinct seeded pairs cycled), with its roofline."""
    import torch
    from paper_2201_11924_gb300 import simsense
    dev = torch.device("cuda", torch.cuda.current_device())
    pairs = [scenes.make_pair(wl, seed=wl.seed + u) for u in range(n_pairs)]
    lefts = [torch.from_numpy(p["left"]).to(dev) for p in pairs]
    rights = [torch.from_numpy(p["right"]).to(dev) for p in pairs]
    depth = torch.empty((wl.H, wl.W), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    with simsense.SimSense.from_workload(wl) as m:
        for i in range(warmup):
            m.compute(lefts[i % n_pairs], rights[i % n_pairs], depth)
        torch.cuda.synchronize()
        st = m.device_status()
        if st != 0:
            raise SystemExit(f"bench: device status {st} after the warm-up steps of {wl.name}")
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for i in range(steps):
            m.compute(lefts[i % n_pairs], rights[i % n_pairs], depth)
        e1.record(stream)
        torch.cuda.synchronize()
        m.set_option(simsense.OPT_PROFILE, 1)           # stage times from a separate pass
        for i in range(min(steps, 200)):
            m.compute(lefts[i % n_pairs], rights[i % n_pairs], depth)
        torch.cuda.synchronize()
        stage_ms, n_prof = m.profile_read()
        m.set_option(simsense.OPT_PROFILE, 0)
        status = m.device_status()
    ms = e0.elapsed_time(e1) / steps
    roof = roofline_object(wl, stage_ms, n_prof, n_sm, peaks, peak_src)
    return {"config": workload_config(wl), "steps": steps, "warmup": warmup, "value": 1e3 / ms, "unit": UNIT,
            "ms_per_step": ms, "cells_per_s": wl.cells * 1e3 / ms,
            "stage_frac_of_roofline": stage_roofline_frac(wl, ms, n_sm, peaks),
            "roofline": roof, "device_status": status, "gpu_launches": 4 * steps}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="simsense", choices=["simsense", "reference"])
    ap.add_argument("--workload", default=configs.HD_720.name, choices=sorted(configs.ALL))
    ap.add_argument("--cpu-budget-s", type=float, default=10.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ref-strip-rows", type=int, default=90)
    ap.add_argument("--mode", default="plain", choices=["plain", "batch", "batchmix", "serve", "table2", "sim"],
                    help="plain: the default contract line; batch: --batch-pairs pairs of --workload per "
                         "batch call (tuned); batchmix: the 64-pair mixed batch; "
                         "table2: the paper's Table 2 workload (960x540, rectified, registered to 1920x1080); "
                         "sim: the whole simulated sensor on the device (render, noise, depth); "
                         "serve: the continuous-batching request loop")
    ap.add_argument("--serve-rate", type=float, default=4000.0, help="Poisson arrivals per second")
    ap.add_argument("--serve-seconds", type=float, default=8.0, help="trace length")
    ap.add_argument("--serve-slots", type=int, default=4, help="compute slots per size class")
    ap.add_argument("--serve-sustain", type=float, default=1200.0,
                    help="second, below-capacity arrival rate for the latency figures")
    ap.add_argument("--noise", action="store_true", help="IR sensor noise (D415 values) before the census")
    ap.add_argument("--census-cs", action="store_true", help="variant: centre-symmetric census")
    ap.add_argument("--block", default="1x1", help="variant: SGBM block, e.g. 3x3 (1x1 = per-pixel cost)")
    ap.add_argument("--median", type=int, default=0, choices=[0, 3, 5], help="variant: k x k median filter")
    ap.add_argument("--no-extras", action="store_true",
                    help="plain line only: skip the small and large workloads, the 64-pair batch and serving")
    ap.add_argument("--batch-pairs", type=int, default=8,
                    help="pairs per batch for the batched sub-measurement of the plain workload")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    wl = configs.ALL[args.workload]
    if args.census_cs or args.block != "1x1" or args.median or args.noise:
        # a variant of the stage Sec. VI-D names (and the sensor noise of
        # Sec. VI-C before it), on the same workload
        bw, bh = (int(v) for v in args.block.split("x"))
        wl = dataclasses.replace(wl, census_cs=bool(args.census_cs), block=(bw, bh), median=args.median,
                                 noise=bool(args.noise),
                                 name=wl.name + ("_noise" if args.noise else "") +
                                 ("_csct" if args.census_cs else "") +
                                 (f"_sgbm{bw}x{bh}" if bw * bh > 1 else "") +
                                 (f"_median{args.median}" if args.median else ""))

    if args.impl == "reference":
        return run_reference(args, wl)
    if args.mode == "batchmix":
        return run_batchmix(args)
    if args.mode == "batch":
        return run_batch(args, wl)
    if args.mode == "table2":
        return run_table2(args)
    if args.mode == "sim":
        return run_sim(args)
    if args.mode == "serve":
        return run_serve(args)

    import torch
    from paper_2201_11924_gb300 import simsense

    # one replica per GPU: no data-path collective, only the timing barrier
    # and the maximum of the ranks' elapsed times
    rep = replicas.from_env()
    world, rank = rep.world, rep.rank
    dev = torch.device("cuda", rep.local)
    torch.cuda.set_device(dev)

    # a few distinct seeded pairs per rank, resident in HBM: rank r owns pairs
    # r, r + N, r + 2N, ... of the job (weak scaling, nothing shared)
    n_pairs = 4
    pairs = [scenes.make_pair(wl, seed=wl.seed + u) for u in replicas.shard(world * n_pairs, rank, world)]
    lefts = [torch.from_numpy(p["left"]).to(dev) for p in pairs]
    rights = [torch.from_numpy(p["right"]).to(dev) for p in pairs]
    depth = torch.empty((wl.H, wl.W), dtype=torch.float32, device=dev)
    m = simsense.SimSense.from_workload(wl)
    stream = torch.cuda.current_stream(dev)

    for i in range(args.warmup):
        m.compute(lefts[i % n_pairs], rights[i % n_pairs], depth)
    torch.cuda.synchronize()
    # a bounded device wait that gave up makes every later frame slow and
    # wrong: stop before the timed region instead of timing it
    st = m.device_status()
    if st != 0:
        raise SystemExit(f"bench: device status {st} after the warm-up steps (a bounded wait gave up)")

    sampler = ClockSampler(_bus_id(torch, dev))
    rep.barrier()
    torch.cuda.synchronize()
    t_wall0 = time.time()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for i in range(args.steps):
        m.compute(lefts[i % n_pairs], rights[i % n_pairs], depth)
    ev1.record(stream)
    torch.cuda.synchronize()
    rep.barrier()
    t_wall1 = time.time()
    clocks = sampler.stop(t_wall0, t_wall1)
    el_ms = ev0.elapsed_time(ev1)
    el_ms = rep.max_over_ranks(el_ms, dev)
    # the stage times for the roofline, from a separate pass with the stage
    # events on (they sit between the kernels, so the timed region runs
    # without them)
    m.set_option(simsense.OPT_PROFILE, 1)
    for i in range(min(args.steps, 200)):
        m.compute(lefts[i % n_pairs], rights[i % n_pairs], depth)
    torch.cuda.synchronize()
    stage_ms, n_prof = m.profile_read()
    m.set_option(simsense.OPT_PROFILE, 0)
    value = world * args.steps / (el_ms / 1e3)

    # end to end through the host-buffer call, as a camera stream runs it: k
    # frames in flight (k handles, each on its own stream); every frame
    # uploads its own pinned inputs, computes and downloads its depth, and its
    # result is read on the host before its handle takes the frame k later
    hl = [torch.from_numpy(p["left"]).pin_memory() for p in pairs]
    hr = [torch.from_numpy(p["right"]).pin_memory() for p in pairs]
    e2e_steps = max(4, min(args.steps, 500))

    def e2e_run(kf):
        hd = [torch.empty((wl.H, wl.W), dtype=torch.float32).pin_memory() for _ in range(kf)]
        extra = [simsense.SimSense.from_workload(wl) for _ in range(kf - 1)]
        hs = [m] + extra
        ss = [stream] + [torch.cuda.Stream(device=dev) for _ in range(kf - 1)]
        for i in range(max(args.warmup, kf)):
            hs[i % kf].compute_host(hl[i % n_pairs], hr[i % n_pairs], hd[i % kf], stream=ss[i % kf])
        torch.cuda.synchronize()
        rep.barrier()
        t0 = time.perf_counter()
        for i in range(e2e_steps):
            k = i % kf
            if i >= kf:                          # frame i - kf on this handle: done, read
                ss[k].synchronize()
                _ = float(hd[k][0, 0])
            hs[k].compute_host(hl[i % n_pairs], hr[i % n_pairs], hd[k], stream=ss[k])
        for k in range(kf):
            ss[k].synchronize()
            _ = float(hd[k][0, 0])
        el = time.perf_counter() - t0
        for h in extra:
            h.close()
        return rep.max_over_ranks(el, dev)

    by_k = {kf: world * e2e_steps / e2e_run(kf) for kf in (1, 2, 3, 4, 6, 8)}
    best_k = max((2, 3, 4, 6, 8), key=lambda kf: by_k[kf])
    e2e = {"value": by_k[best_k], "unit": UNIT,
           "h2d_bytes_per_step": 2 * wl.W * wl.H, "d2h_bytes_per_step": 4 * wl.W * wl.H,
           "steps": e2e_steps, "frames_in_flight": best_k,
           "by_frames_in_flight": {str(k): v for k, v in by_k.items()},
           "one_in_flight_value": by_k[1]}

    # the batched form on the same workload: batch_pairs pairs per CUDA-graph launch
    batched = None
    variant = wl.census_cs or wl.block != (1, 1) or wl.median or wl.noise
    if args.batch_pairs > 1 and not variant:      # the batched form runs the plain stage
        nb = args.batch_pairs
        bwl = [wl] * nb
        bl = [lefts[i % n_pairs] for i in range(nb)]
        br = [rights[i % n_pairs] for i in range(nb)]
        bd = [torch.empty((wl.H, wl.W), dtype=torch.float32, device=dev) for _ in range(nb)]
        with simsense.SimSenseBatch(bwl) as bt:
            bt.tune(bl, br, bd, reps=1)            # the native autotuner picks the form and schedule
            schedule = bt.get_schedule()
            for _ in range(args.warmup):
                bt.compute(bl, br, bd)
            torch.cuda.synchronize()
            bsteps = max(3, args.steps // nb)
            rep.barrier()
            b0 = torch.cuda.Event(enable_timing=True)
            b1 = torch.cuda.Event(enable_timing=True)
            b0.record(stream)
            for _ in range(bsteps):
                bt.compute(bl, br, bd)
            b1.record(stream)
            torch.cuda.synchronize()
            b_ms = b0.elapsed_time(b1)
            status = bt.device_status()
        b_ms = rep.max_over_ranks(b_ms, dev)
        batched = {"value": world * nb * bsteps / (b_ms / 1e3), "unit": UNIT, "pairs_per_batch": nb,
                   "batches": bsteps, "ms_per_batch": b_ms / bsteps, "graph": True, "schedule": schedule,
                   "device_status": status}

    if rank != 0:
        m.close()
        rep.close()
        return 0
    m.close()

    # roofline of the dominant kernel, from the live stage events
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    peaks, peak_src = _peaks()
    roofline = roofline_object(wl, stage_ms, n_prof, n_sm, peaks, peak_src)
    if batched is not None:
        batched["stage_roofline"] = stage_roofline_frac(wl, 1e3 / (batched["value"] / world), n_sm, peaks)

    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        rate, n, el = cpu_oracle_rate(wl, pairs[0], budget_s=args.cpu_budget_s)
        cpu = {"value": rate / wl.cells, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"{n} full-width {wl.W}x90 strips of one pair ({el:.1f} s), per-cell rate extrapolated"}

    # the other configurations of the stage, at N = 1 on this GPU: the small
    # and the large single pair, the 64-pair uneven batch against 64 plain
    # calls, and the serving loop at the offered and a sustainable rate
    extras = {}
    if world == 1 and not args.no_extras and not variant:
        extras["workloads"] = {
            configs.SMALL_320.name: plain_measure(configs.SMALL_320, 2000, 20, n_sm, peaks, peak_src),
            configs.FHD_1080.name: plain_measure(configs.FHD_1080, 60, 5, n_sm, peaks, peak_src),
        }
        # the same workloads as batches of pairs (the throughput form)
        extras["workloads"][configs.SMALL_320.name]["batched"] = batched_measure(
            configs.SMALL_320, 64, 20, 3, n_sm, peaks)
        extras["workloads"][configs.FHD_1080.name]["batched"] = batched_measure(
            configs.FHD_1080, 8, 6, 2, n_sm, peaks)
        extras["batched_cfg3"] = batchmix_measure(steps=3, warmup=2)
        extras["batched_cfg3"]["stage_roofline"] = batch_roofline_frac(
            configs.batch_workloads(), extras["batched_cfg3"]["ms_per_batch"], n_sm, peaks)
        extras["serve_cfg5"] = serve_measure(args.serve_rate, 2.0, args.serve_sustain, 2.0, args.serve_slots)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": el_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {**workload_config(wl), "pairs_cycled": n_pairs,
                   "l2": "no flush: every step streams its own ~1 GB path volume through HBM, "
                         "far above the 129 MB L2", "path": "plain (one pair per call)"},
        "cells_per_s": value * wl.cells,
        "e2e": e2e,
        # census, cost, paths, select; plus the noise, block-cost and median kernels of a variant
        "gpu_launches": (4 + int(wl.noise) + int(wl.block != (1, 1)) + int(wl.median > 0)) * args.steps,
        "batched": batched,
        "roofline": roofline,
        "stage_roofline": stage_roofline_frac(wl, el_ms / args.steps, n_sm, peaks),
        "cpu_baseline": cpu,
        "clocks": clocks,
        "gpu": torch.cuda.get_device_name(dev),
        "host_cores": os.cpu_count(),
        **extras,
    }
    print(json.dumps(line), flush=True)
    rep.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
