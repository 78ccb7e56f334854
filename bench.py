#!/usr/bin/env python
"""Frame-step benchmark of the hybrid WP/FFT ocean synthesis on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload realistic|batched|mixed_large|serving|sweep|...]
                    [--synth sat|gather|fp16] [--plain]

One step = one whole frame of the hot path (background spectrum update and
inverse FFT, advection/expiry/compaction, injection, wake emission, binning,
synthesis with blend) on the workload's resident scene.  The default
workload is the largest single-GPU scene, mixed_large (2048^2 FFT over 4 km,
8 patches of 1024^2 texels, 2M particles each, 32 buckets), stepped in
batched mode (one synthesis launch over all patches, frames replayed as
captured CUDA graphs; a one-patch scene launches eagerly, chained by
programmatic dependent launch) with the summed-area synthesis.  Beside it on
the same line: the same scene in plain mode (one synthesis launch per
patch, eager launches), the tensor-core gather, and the metric's "batched vs
plain" on the 32-patch batched workload (--compare-frames frames in each
mode).  The metric is particle-pixel (bump-texel) evaluations per second,
the eval count being the exact integer count of (bump, texel-centre) pairs
inside the kernel supports (checked bit-exact against the FP64 oracle by the
tests); p50/p99 frame-step latency is reported beside it, and the same
evals over the synthesis stage alone.

Timing: W untimed warm-up steps, then K steps timed with CUDA events on the
scene's stream, L2 flushed (256 MiB write, then a 256 MiB read that evicts the
written lines) between timed steps, barrier +
synchronize around the timed region, max over ranks.  N > 1 (torchrun) runs
one independent scene per rank (weak scaling, no collective on the data
path).  ``--impl reference`` times the FP64 CPU oracle on the host cores.
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

from paper_2511_02852_gb300 import workloads as wl  # noqa: E402

METRIC = "particle-pixel evals/s + frame-step p50/p99 ms, batched vs plain, at \u22641e-4\u00b7Hs"
UNIT = "evals/s"
# tensor work of one operand stage of the tile gather: 6 MMAs of M = N = 128, K = 16
FLOPS_PER_STAGE = 6 * 2 * 128 * 128 * 16
# issue-rate peak of one GB300 in thread instructions: 152 SMs x 4 schedulers x
# 32 lanes x 2.070 GHz
ALU_PEAK_TOPS = 152 * 4 * 32 * 2.070e9 / 1e12
# algorithmic operations of the summed-area synthesis per (texel, bucket): for
# each of the 9 S_ij components one add in each prefix pass and one
# int-to-float conversion (27), and the contraction of h, Dx and Dy with the
# texel's u, u', v, v' factors (21 multiply-adds); the per-bump corner events
# are not counted (a lower bound on the work)
SAT_OPS_PER_TEXEL_BUCKET = 48
# and per candidate bump of a (tile, bucket): its 9 corner weights (A p_i q_j)
# and 4 corner adds of each (corners outside the tile are dropped, so this is
# an upper bound on that part; the whole count stays algorithmic, independent
# of how the kernel aggregates or orders the adds)
SAT_OPS_PER_CANDIDATE = 45


def tensor_peak():
    """Dense FP16 tensor peak: the measured bf16 GEMM rate (same nominal rate)."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        v = float(json.load(open(path))["bf16_tflops"])
        return v, "measured: bf16 cuBLAS GEMM burst (FP16 dense has the same nominal rate)"
    except Exception:
        return 1900.0, "fallback: 1.9 PFLOP/s bf16 burst (FP16 dense has the same nominal rate)"
# algorithmic bytes of the background FFT per grid point: h0 read (8), the
# two complex planes written by the row pass and read by the column pass
# (16 + 16), h, Dx, Dy written (12)
FFT_BYTES_PER_POINT = 52


def workload_config(name, rank=0):
    cfg = wl.ALL[name]()
    cfg["spectrum"]["seed"] = int(cfg["spectrum"]["seed"]) + 1000 * rank
    return cfg


def reduce_over_ranks(total_s, total_evals, world, device):
    """Whole-job figures of a weak-scaled run: the slowest rank's timed
    seconds and the evals of all ranks (one process per GPU, each with its
    own scene replica; no exchange on the data path)."""
    if world <= 1:
        return total_s, float(total_evals)
    import torch
    import torch.distributed as dist
    t = torch.tensor([total_s], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    e = torch.tensor([float(total_evals)], dtype=torch.float64, device=device)
    dist.all_reduce(e, op=dist.ReduceOp.SUM)
    return float(t.item()), float(e.item())


def describe(cfg):
    s = cfg["spectrum"]
    ps = cfg["patches"]
    p = ps[0]
    nbs = sorted({int(q["n_buckets"]) if int(q["n_buckets"]) > 0 else int(s["n_buckets"]) for q in ps})
    sides = sorted({(int(q["width"]), int(q["height"])) for q in ps})
    shape = (f"{sides[0][0]}x{sides[0][1]}" if len(sides) == 1 else
             f"{min(a * b for a, b in sides)}..{max(a * b for a, b in sides)} texels each")
    return {
        "workload": (f"{cfg['name']}: {'JONSWAP' if s['spectrum'] == 0 else 'Phillips'} "
                     f"U10={s['wind_speed']} m/s, {s['fft_n']}^2 FFT over {s['fft_L']} m, "
                     f"{len(ps)} patch(es) {shape} at {p['cell']} m, "
                     f"{nbs[0] if len(nbs) == 1 else f'{nbs[0]}-{nbs[-1]}'} buckets x {s['n_theta']} directions, "
                     f"{sum(int(q['prefill']) for q in ps)} prefilled particles in all, "
                     f"wake={'on' if any(q['emitter'] for q in ps) else 'off'}"),
        "patches": len(cfg["patches"]),
        "fft_n": s["fft_n"],
        "patch_texels": sum(q["width"] * q["height"] for q in cfg["patches"]),
        "buckets": s["n_buckets"],
        "dt": cfg["dt"],
        "l2": "flushed between timed steps (256 MiB write, then a 256 MiB read that evicts it)",
    }


# ---- clocks --------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu_id), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
            return
        # the timed region starts only once the sampler is delivering
        t0 = time.time()
        while not self.lines and time.time() - t0 < 5.0 and self.proc.poll() is None:
            time.sleep(0.01)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---- CPU oracle ------------------------------------------------------------------
def first_patch(cfg):
    """The scene with its first patch only: patch 0 evolves exactly as in the
    whole scene (its particles depend on its own description, index and the
    seed), so the oracle's sample needs no other patch."""
    import copy
    c = copy.deepcopy(cfg)
    c["patches"] = c["patches"][:1]
    return c


def oracle_strip_rate(cfg, target_s=10.0, frames=1, state=None, rows=None):
    """Time the FP64 oracle's synthesis on a strip of rows of patch 0 (a
    bounded sample of the frame; `rows` given: that many, else as many as
    fit target_s).  Returns (evals/s, evals, seconds, rows, threads)."""
    import numpy as np
    from oracle.scene import OracleScene
    from oracle.synth import synth_maps
    orc = state
    if orc is None:
        orc = OracleScene(first_patch(cfg))
        for _ in range(frames):
            orc.step(cfg["dt"])
    ps = orc.patches[0]
    bm = ps.bumps()

    def run(rows, y0=0):
        b = dict(bm)
        b["Y"] = bm["Y"] - y0 * 65536
        t0 = time.perf_counter()
        _, _, _, ev = synth_maps(ps.T.W, rows, b, orc.lam)
        return ev, time.perf_counter() - t0

    if rows is None:
        ev, dt = run(8)
        per_row = max(dt / 8, 1e-6)
        rows = int(min(ps.T.H, max(8, target_s / per_row)))
    y0 = max(0, (ps.T.H - rows) // 2)
    ev, dt = run(rows, y0)
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return ev / dt, ev, dt, rows, threads


def oracle_rate_one_core(workload, target_s=2.0):
    """The same strip timing with the oracle on one host core, in a child
    process with OMP_NUM_THREADS=1 (the parent's thread pool is left as it
    is).  Returns (evals/s, evals, seconds, rows), or None if the child
    fails."""
    code = ("import json, sys; sys.path.insert(0, %r); import bench; "
            "r = bench.oracle_strip_rate(bench.workload_config(%r), target_s=%r); "
            "print(json.dumps([r[0], r[1], r[2], r[3]]))") % (ROOT, workload, float(target_s))
    env = dict(os.environ, OMP_NUM_THREADS="1")
    try:
        out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                             timeout=300)
        if out.returncode != 0:
            return None
        return tuple(json.loads(out.stdout.strip().splitlines()[-1]))
    except Exception:
        return None


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    cfg = workload_config(args.workload)
    from oracle.scene import OracleScene
    orc = OracleScene(first_patch(cfg))
    rates, times, evs = [], [], []
    rows_used = None
    # each step: the oracle's frame update plus a strip of the synthesis,
    # the strip sized once so that the whole run stays within ref_total_seconds
    per_step = min(args.ref_seconds, max(0.05, args.ref_total_seconds / (args.warmup + args.steps)))
    for k in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        orc.step(cfg["dt"])
        rate, ev, dt, rows, threads = oracle_strip_rate(cfg, target_s=per_step, state=orc, rows=rows_used)
        rows_used = rows
        if k >= args.warmup:
            rates.append(rate)
            times.append(time.perf_counter() - t0)
            evs.append(ev)
    value = sum(evs) / sum(times)
    ms = 1000 * sum(times) / len(times)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": describe(cfg),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "cpu": host_cpu(),
                         "sample": f"per step: one oracle frame update of patch 0 (of "
                                   f"{len(cfg['patches'])}) plus the FP64 synthesis of a {rows_used}-row "
                                   f"strip of that {cfg['patches'][0]['width']}-wide patch"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    one = oracle_rate_one_core(args.workload)
    if one is not None:
        line["cpu_baseline"]["value_1core"] = one[0]
        line["cpu_baseline"]["sample_1core"] = (f"a {one[3]}-row strip on one core (OMP_NUM_THREADS=1): "
                                                f"{one[1]} evals in {one[2]:.1f} s")
    print(json.dumps(line))
    return 0


# ---- serving ---------------------------------------------------------------------------
def run_serving(args):
    """Open-loop serving run: Poisson frame-step requests over the serving
    scenes through the frame-step server (continuous batching); latency =
    completion seen by polling minus scheduled arrival."""
    import numpy as np
    import torch
    from paper_2511_02852_gb300 import scwp
    rank = int(os.environ.get("RANK", "0"))
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    scenes = wl.serving()
    sv = scwp.Server(hbm_budget_bytes=int(args.hbm_budget_gb * 1e9), max_inflight=args.inflight)
    t_adm = time.perf_counter()
    sid = [sv.add_scene(c) for c in scenes]
    t_adm = time.perf_counter() - t_adm
    admitted = [k for k, s in enumerate(sid) if s is not None]
    dt = 1.0 / 60.0

    def drain(n_req, first_id):
        got = 0
        while got < n_req:
            sv.tick()
            got += len(sv.poll())
        return got

    rid = 10 ** 9                       # warm-up: every scene twice (both graph-free paths warm)
    for _ in range(2):
        for k in admitted:
            sv.submit(sid[k], dt, rid)
            rid += 1
        drain(len(admitted), 0)
    torch.cuda.synchronize()

    def eval_total():
        tot = 0
        for k in admitted:
            v = sv.scene(sid[k])
            tot += sum(v.stats(p).eval_total for p in range(len(scenes[k]["patches"])))
        return tot

    e0 = eval_total()
    t_arr, s_arr = wl.serving_arrivals(rate=args.rate, seconds=args.serve_seconds, n_scenes=len(scenes))
    keep = np.array([sid[s] is not None for s in s_arr], dtype=bool)
    t_arr, s_arr = t_arr[keep], s_arr[keep]
    n = len(t_arr)
    lat = np.full(n, np.nan)
    clk = ClockSampler(0)
    clk.start()
    i = done = 0
    t0 = time.perf_counter()
    while done < n:
        now = time.perf_counter() - t0
        while i < n and t_arr[i] <= now:
            sv.submit(sid[s_arr[i]], dt, i)
            i += 1
        while sv.tick():
            pass
        fin = sv.poll()
        if fin:
            tnow = time.perf_counter() - t0
            for r in fin:
                lat[r] = tnow - t_arr[r]
            done += len(fin)
    elapsed = time.perf_counter() - t0
    clocks = clk.stop()
    torch.cuda.synchronize()
    evals = eval_total() - e0
    info = sv.info()
    ms = np.sort(lat) * 1e3
    line = {
        "metric": METRIC + " (serving)", "value": evals / elapsed, "unit": UNIT, "n_gpus": 1,
        "steps": n, "warmup": 2, "ms_per_step": 1e3 * elapsed / max(n, 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": f"serving: {len(scenes)} scenes ({len(admitted)} admitted under "
                               f"{args.hbm_budget_gb:g} GB), Poisson {args.rate:g} requests/s for "
                               f"{args.serve_seconds:g} s, one frame step (dt 1/60) per request",
                   "max_inflight_ticks": args.inflight, "admission_s": t_adm,
                   "device_bytes": info.device_bytes},
        "p50_ms": float(ms[len(ms) // 2]), "p99_ms": float(ms[min(len(ms) - 1, int(0.99 * len(ms)))]),
        "max_ms": float(ms[-1]), "requests": n, "requests_per_s": n / elapsed,
        "ticks": int(info.ticks_launched), "evals": int(evals), "clocks": clocks,
    }
    if rank == 0:
        print(json.dumps(line))
    sv.close()
    return 0


# ---- sweeps ----------------------------------------------------------------------------
def run_sweep(args):
    """The paper's Table 2 axes as synthetic sweeps: per point the FFT stage
    alone (FFT-only), the particle stages plus synthesis (WP-only) and the
    whole frame (hybrid), from the library's stage events."""
    import torch
    from paper_2511_02852_gb300 import scwp
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    out = []
    for pt in wl.sweep_points():
        cfg = wl.sweep_point(**pt)
        sc = scwp.Scene(cfg)
        for _ in range(args.warmup):
            sc.step(cfg["dt"])
        torch.cuda.synchronize()
        sc.set_timing(True)
        sc.timing_read()
        evals = 0
        for _ in range(args.steps):
            sc.step(cfg["dt"])
            evals += sc.stats(0).eval_count
        torch.cuda.synchronize()
        st, fr = sc.timing_read()
        sc.set_timing(False)
        fft, wp, frame = st[0] / fr, (st[1] + st[2]) / fr, st[3] / fr
        out.append(dict(pt, fft_ms=fft, wp_ms=wp, frame_ms=frame, fps=1000.0 / frame,
                        evals_per_s=evals / (st[2] / 1000.0) if st[2] > 0 else 0.0,
                        live=sc.stats(0).live_particles))
        sc.close()
    line = {"metric": METRIC + " (sweep)", "value": max(o["evals_per_s"] for o in out), "unit": UNIT,
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
            "data": "synthetic", "dtype": "f32",
            "config": {"workload": "sweep: (n_omega, n_theta) in {8,12,16}^2 at U10 10 m/s, res 512; "
                                   "U10 in {3,5,15}; res in {256,1024}; one 128 m patch, 100k particles"},
            "sweep": out}
    print(json.dumps(line))
    return 0


# ---- ours ----------------------------------------------------------------------------
def host_cpu():
    """The host CPU's model name (lscpu, else /proc/cpuinfo where it has one)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            k, _, v = line.partition(":")
            if k.strip() == "Model name" and v.strip():
                return v.strip()
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                k, _, v = line.partition(":")
                if k.strip() in ("model name", "Model", "Hardware"):
                    return v.strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def tc_roofline(sc, cfg, synth_ms, stage_info, fp16):
    """Tensor roofline of the tile gather (k_synth_tc with its bucket-group
    blend), timed by the library's events around the synthesis stage on the
    stream it launches on.  Executed tensor work: operand stages x the work of
    6 MMAs of 128x128x16 (hi*hi, hi*lo, lo*hi over two K = 16 steps; issued as
    one N = 256 and one N = 128 MMA per step), a third of that with single
    FP16 operands."""
    stages = sum(sc.stats(p).mma_stages for p in range(len(cfg["patches"])))
    mma_flops = stages * FLOPS_PER_STAGE // (3 if fp16 else 1)
    peak, peak_src = tensor_peak()
    achieved = mma_flops / (synth_ms / 1000.0) / 1e12
    return {"bound": "tensor", "kernel": "k_synth_tc", "achieved": achieved, "peak": peak,
            "unit": "TFLOP/s", "frac": achieved / peak, "traffic": profiled_traffic(cfg, "k_synth_tc"),
            "peak_source": peak_src, "flops_per_launch": mma_flops, "operand_stages_per_launch": stages,
            "avg_launch_ms": synth_ms, "stage_ms": stage_info}


def sat_roofline(sc, cfg, synth_ms, stage_info):
    """ALU roofline of the summed-area synthesis (k_synth_sat with its
    bucket-group blend), timed by the library's events around the synthesis
    stage.  Algorithmic work: SAT_OPS_PER_TEXEL_BUCKET operations per (texel,
    bucket) of every patch, against the instruction-issue peak."""
    tb = cand = 0
    for p in range(len(cfg["patches"])):
        H, W = sc.patch_shape(p)
        tb += W * H * sc.info(p).n_buckets
        cand += sc.stats(p).sat_candidates
    ops = tb * SAT_OPS_PER_TEXEL_BUCKET + cand * SAT_OPS_PER_CANDIDATE
    achieved = ops / (synth_ms / 1000.0) / 1e12
    kernel = "k_synth_sat3" if sc.info(0).sat_variant == 1 else "k_synth_sat"
    return {"bound": "alu", "kernel": kernel, "achieved": achieved, "peak": ALU_PEAK_TOPS,
            "unit": "Tops/s", "frac": achieved / ALU_PEAK_TOPS, "traffic": profiled_traffic(cfg, kernel),
            "peak_source": "derived: 152 SMs x 4 schedulers x 32 lanes x 2070 MHz (thread instructions)",
            "ops_per_launch": ops, "texel_buckets_per_launch": tb, "candidates_per_launch": cand,
            "ops_note": f"{SAT_OPS_PER_TEXEL_BUCKET} per (texel, bucket): 9 components x (2 prefix adds + "
                        f"1 conversion) + 21 contraction multiply-adds; {SAT_OPS_PER_CANDIDATE} per (candidate "
                        f"bump, tile): 9 corner weights + 4 x 9 corner adds",
            "avg_launch_ms": synth_ms,
            "stage_ms": stage_info}


def fft_roofline(cfg, fft_ms):
    """HBM roofline of the background FFT (k_spectrum_rows + k_fft_cols with
    the spectrum update fused in), timed by the library's events on the side
    stream it runs on.  Algorithmic bytes per grid point: FFT_BYTES_PER_POINT
    (h0 read, the two complex planes written by the row pass and read by the
    column pass, h, Dx, Dy written)."""
    N = int(cfg["spectrum"]["fft_n"])
    peak, src = hbm_peak()
    nbytes = FFT_BYTES_PER_POINT * N * N
    achieved = nbytes / (fft_ms / 1000.0) / 1e9
    return {"bound": "hbm", "kernel": "k_spectrum_rows + k_fft_cols", "achieved": achieved, "peak": peak,
            "unit": "GB/s", "frac": achieved / peak, "traffic": profiled_traffic(cfg, "fft"),
            "peak_source": src, "bytes_per_launch": nbytes, "grid": f"{N}^2", "avg_launch_ms": fft_ms}


def hbm_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        return float(json.load(open(path))["hbm_gbs"]), "measured: STREAM-style copy (MEASURED_PEAKS.json)"
    except Exception:
        return 6800.0, "fallback: 6.8 TB/s"


def profiled_traffic(cfg, kernel):
    """DRAM bytes per launch of `kernel` on this workload from the committed
    ncu summary (null when there is none for this kernel and workload)."""
    rfile = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        tr = json.load(open(rfile))
    except Exception:
        return None
    for e in (tr if isinstance(tr, list) else [tr]):
        if e.get("workload") == cfg["name"] and e.get("kernel") == kernel:
            return e.get("dram_bytes_per_launch")
    return None


class L2Flush:
    """Between timed steps: write a 256 MiB buffer (twice the 129 MB L2),
    then read another one, so that the written lines leave L2 (and reach
    DRAM) before the timed step starts instead of during it."""

    def __init__(self, torch):
        self.a = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
        self.b = torch.ones(64 << 20, dtype=torch.int32, device="cuda")

    def zero_(self):
        self.a.zero_()
        self.b.sum()


def pct(ms_sorted, q):
    return ms_sorted[min(len(ms_sorted) - 1, max(0, int(math.ceil(q * len(ms_sorted))) - 1))]


def timed_frames(sc, cfg, n, flush, stream):
    """n frames timed one by one with CUDA events on the scene's stream (L2
    flushed before each); returns (sorted ms list, evals)."""
    import torch
    st_ev = [torch.cuda.Event(enable_timing=True) for _ in range(n)]
    en_ev = [torch.cuda.Event(enable_timing=True) for _ in range(n)]
    ev = 0
    for k in range(n):
        flush.zero_()
        st_ev[k].record(stream)
        sc.step(cfg["dt"])
        en_ev[k].record(stream)
        ev += sum(sc.stats(p).eval_count for p in range(len(cfg["patches"])))
    torch.cuda.synchronize()
    return sorted(a.elapsed_time(b) for a, b in zip(st_ev, en_ev)), ev


def tune(sc, args, flush, dt):
    """The summed-area autotuner on the scene's live frame (timed on the
    device), then warm-up frames for the re-captured frame graphs."""
    if args.no_tune or args.synth != "sat":
        return None
    rows, chosen, cached = sc.autotune(reps=3)
    for _ in range(3):
        flush.zero_()
        sc.step(dt)
    names = {0: "persistent nine-plane", 1: "three-group"}
    return {"chosen": {"kernel": names[rows[chosen][0]], "group_multiplier": rows[chosen][1]},
            "from_cache": cached,
            "timed": [{"kernel": names[v], "group_multiplier": g, "synthesis_ms": m} for v, g, m in rows]}


def frame_summary(ms, ev, mode):
    return {"mode": mode, "frames": len(ms), "value": ev / (sum(ms) / 1000.0), "unit": UNIT,
            "ms_per_step": sum(ms) / len(ms), "frames_per_s": 1000.0 * len(ms) / sum(ms),
            "p50_ms": pct(ms, 0.5), "p99_ms": pct(ms, 0.99), "max_ms": ms[-1]}


def batched_vs_plain(args, flush, stream, frames):
    """The metric's "batched vs plain" on the 32-patch batched workload: the
    same scene stepped in batched mode (one synthesis launch over every
    patch, frames replayed as captured CUDA graphs) and in plain mode (one
    synthesis launch per patch, eager launches), `frames` timed frames each."""
    import torch
    from paper_2511_02852_gb300 import scwp
    cfg = workload_config("batched")
    sc = scwp.Scene(cfg)
    sc.set_synth_mode(scwp.SYNTH_SAT)
    out = {"workload": describe(cfg)["workload"]}
    for mode, on in (("batched", True), ("plain", False)):
        sc.set_batched(on)
        for _ in range(5):
            flush.zero_()
            sc.step(cfg["dt"])
        tuned = tune(sc, args, flush, cfg["dt"])
        torch.cuda.synchronize()
        ms, ev = timed_frames(sc, cfg, frames, flush, stream)
        out[mode] = frame_summary(ms, ev, "one synthesis launch over all 32 patches, captured frame graph"
                                  if on else "one synthesis launch per patch, eager launches")
        out[mode]["autotune"] = tuned
    out["speedup_frames_per_s"] = out["batched"]["frames_per_s"] / out["plain"]["frames_per_s"]
    sc.close()
    return out


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist
    from paper_2511_02852_gb300 import scwp

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    cfg = workload_config(args.workload, rank)
    sc = scwp.Scene(cfg, device=local)
    if args.batched:
        sc.set_batched(True)
    modes = {"sat": scwp.SYNTH_SAT, "gather": scwp.SYNTH_GATHER, "fp16": scwp.SYNTH_GATHER_FP16}
    sc.set_synth_mode(modes[args.synth])
    stream = torch.cuda.current_stream()
    flush = L2Flush(torch)
    dt = cfg["dt"]
    npatch = len(cfg["patches"])

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        flush.zero_()
        sc.step(dt)
    tuned = tune(sc, args, flush, dt)
    barrier()
    launches0 = sc.launch_count()
    props = torch.cuda.get_device_properties(local)
    clk = ClockSampler(f"GPU-{props.uuid}" if getattr(props, "uuid", None) else local)
    clk.start()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    evals = []
    barrier()
    for k in range(args.steps):
        flush.zero_()
        starts[k].record(stream)
        sc.step(dt)
        ends[k].record(stream)
        evals.append(sum(sc.stats(p).eval_count for p in range(npatch)))
    barrier()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    launches = sc.launch_count() - launches0
    # stage breakdown: library events force one-kernel-at-a-time launches, so
    # it comes from eager frames after the timed ones
    sc.set_timing(True)
    sc.timing_read()
    for _ in range(min(max(args.steps, 5), 20)):
        flush.zero_()
        sc.step(dt)
    torch.cuda.synchronize()
    stage_ms, frames = sc.timing_read()
    sc.set_timing(False)
    total_s = sum(step_ms) / 1000.0
    total_evals = sum(evals)
    total_s_all, total_evals_all = reduce_over_ranks(total_s, total_evals, world, "cuda")
    value = total_evals_all / total_s_all

    synth_ms = stage_ms[2] / max(frames, 1)
    fft_ms = stage_ms[0] / max(frames, 1)
    evals_per_step = total_evals / args.steps
    stage_info = {"source": "library events on eager frames after the timed ones",
                  "fft": fft_ms, "particles": stage_ms[1] / max(frames, 1),
                  "synth_blend": synth_ms, "frame": stage_ms[3] / max(frames, 1)}
    if args.synth == "sat":
        roofline = sat_roofline(sc, cfg, synth_ms, stage_info)
    else:
        roofline = tc_roofline(sc, cfg, synth_ms, stage_info, args.synth == "fp16")
    roof_fft = fft_roofline(cfg, fft_ms)

    # the same scene in plain mode (one patch per launch, eager launches)
    plain = None
    if args.batched and not args.no_compare:
        sc.set_batched(False)
        for _ in range(3):
            flush.zero_()
            sc.step(dt)
        plain_tune = tune(sc, args, flush, dt)
        ms, ev = timed_frames(sc, cfg, max(10, min(args.steps, 50)), flush, stream)
        sc.set_batched(True)
        plain = frame_summary(ms, ev, "plain: one synthesis launch per patch, eager launches")
        plain["autotune"] = plain_tune

    # the other synthesis on the same scene: the tensor-core gather beside the
    # summed-area default (its own roofline), for comparison
    other = None
    if args.synth == "sat" and not args.no_compare:
        sc.set_synth_mode(scwp.SYNTH_GATHER)
        for _ in range(3):
            flush.zero_()
            sc.step(dt)
        sc.set_timing(True)
        sc.timing_read()
        n_cmp = 10
        ev_c = 0
        for _ in range(n_cmp):
            flush.zero_()
            sc.step(dt)
            ev_c += sum(sc.stats(p).eval_count for p in range(npatch))
        torch.cuda.synchronize()
        ms_c, fr_c = sc.timing_read()
        sc.set_timing(False)
        sc.set_synth_mode(scwp.SYNTH_SAT)
        s_ms = ms_c[2] / max(fr_c, 1)
        other = {"synthesis": "tensor-core tile gather (SCWP_SYNTH_GATHER)", "frames": n_cmp,
                 "value": ev_c / (ms_c[3] / 1000.0), "unit": UNIT, "ms_per_step": ms_c[3] / max(fr_c, 1),
                 "roofline": tc_roofline(sc, cfg, s_ms,
                                         {"source": "library events, eager frames", "fft": ms_c[0] / max(fr_c, 1),
                                          "particles": ms_c[1] / max(fr_c, 1), "synth_blend": s_ms,
                                          "frame": ms_c[3] / max(fr_c, 1)}, False)}

    # batched vs plain on the 32-patch batched workload (the metric's comparison)
    bvp = None
    if rank == 0 and not args.no_compare and args.workload != "batched":
        bvp = batched_vs_plain(args, flush, stream, args.compare_frames)

    # end to end through the C ABI: step + one copy of each patch's three
    # blended planes into pinned host memory
    e2e = None
    if not args.no_e2e:
        shapes = [sc.patch_shape(p) for p in range(npatch)]
        host = [torch.empty((3, H, W), dtype=torch.float32, pin_memory=True) for (H, W) in shapes]
        import ctypes as C
        barrier()
        t0 = time.perf_counter()
        e2e_evals = 0
        for k in range(args.steps):
            sc.step(dt)
            for p, (H, W) in enumerate(shapes):
                scwp.scwp_height_maps(sc.ctx, p, C.c_void_p(host[p].data_ptr()), 3 * H * W, 0)
                e2e_evals += sc.stats(p).eval_count
        torch.cuda.synchronize()
        e2e_s = time.perf_counter() - t0
        plan = sum(sc.info(p).frame_param_bytes for p in range(npatch))
        e2e = {"value": e2e_evals / e2e_s, "unit": UNIT, "h2d_bytes_per_step": 8 + plan,
               "d2h_bytes_per_step": sum(3 * H * W * 4 for (H, W) in shapes),
               "note": "scwp_step + scwp_height_maps (one device-to-host copy of h, Dx, Dy per patch) "
                       "into pinned host memory, wall clock; host-to-device per step: dt and each "
                       "patch's frame plan (injection counts and host-placed spawn points)"}
    clocks = clk.stop()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, ev, secs, rows, threads = oracle_strip_rate(cfg, target_s=args.cpu_seconds)
        cpu = {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle", "cpu": host_cpu(),
               "sample": f"FP64 oracle synthesis of a {rows}-row strip of the "
                         f"{cfg['patches'][0]['width']}-wide patch 0 after one frame "
                         f"({ev} evals in {secs:.1f} s)"}
        one = oracle_rate_one_core(args.workload)
        if one is not None:
            cpu["value_1core"] = one[0]
            cpu["sample_1core"] = (f"the same on one core (OMP_NUM_THREADS=1): a {one[3]}-row strip, "
                                   f"{one[1]} evals in {one[2]:.1f} s")

    if rank == 0:
        ms_sorted = sorted(step_ms)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * total_s_all / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"sat": "f32 (int32 prefix sums)", "gather": "f32 (f16 hi/lo operands)",
                      "fp16": "f16 operands, f32 sums"}[args.synth],
            "data": "synthetic", "config": dict(describe(cfg), parallelism=f"replicas{world}",
                                                mode="batched" if args.batched else "plain",
                                                synthesis=args.synth),
            "p50_ms": pct(ms_sorted, 0.5), "p99_ms": pct(ms_sorted, 0.99), "evals_per_step": evals_per_step,
            # the same evals over the synthesis stage alone (library events)
            "synthesis_evals_per_s": evals_per_step / (synth_ms / 1000.0) if synth_ms > 0 else None,
            "live_particles": sum(sc.stats(p).live_particles for p in range(npatch)),
            "roofline": roofline, "roofline_fft": roof_fft, "cpu_baseline": cpu, "e2e": e2e,
            "plain": plain, "batched_vs_plain": bvp, "gather_tc": other,
            "gpu_launches": launches, "clocks": clocks, "autotune": tuned,
            # bucket groups of each patch's own (one patch per launch) plan;
            # a batched frame plans its groups over all patches at once
            "synth_groups_per_patch_plan": [sc.info(p).sat_groups if args.synth == "sat" else sc.info(p).synth_groups
                                            for p in range(npatch)],
        }
        print(json.dumps(line))
    sc.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=600)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="mixed_large", choices=sorted(wl.ALL) + ["serving", "sweep"])
    ap.add_argument("--compare-frames", type=int, default=200,
                    help="frames timed in each mode of the batched-vs-plain comparison")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--rate", type=float, default=2000.0, help="serving: requests per second")
    ap.add_argument("--serve-seconds", type=float, default=60.0)
    ap.add_argument("--inflight", type=int, default=3, help="serving: ticks outstanding")
    ap.add_argument("--hbm-budget-gb", type=float, default=120.0)
    ap.add_argument("--synth", default="sat", choices=["sat", "gather", "fp16"],
                    help="synthesis: summed-area (default, SCWP_SYNTH_SAT), tensor-core gather "
                         "(SCWP_SYNTH_GATHER) or its single-FP16 operands (SCWP_SYNTH_GATHER_FP16)")
    ap.add_argument("--fp16", action="store_true", help="same as --synth fp16")
    ap.add_argument("--no-compare", action="store_true",
                    help="skip the tensor-core gather measured beside the summed-area default")
    ap.add_argument("--batched", action="store_true",
                    help="one synthesis launch over all patches of the frame, frames replayed as CUDA "
                         "graphs (scwp_set_batched; the default)")
    ap.add_argument("--plain", action="store_true",
                    help="one synthesis launch per patch, frames launched eagerly")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-tune", action="store_true",
                    help="skip the summed-area autotuner (scwp_autotune) before the timed frames")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--ref-seconds", type=float, default=2.0, help="reference: strip seconds per step at most")
    ap.add_argument("--ref-total-seconds", type=float, default=60.0, help="reference: strip seconds in all")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    args.batched = not args.plain
    if args.fp16:
        args.synth = "fp16"
    if args.impl == "reference":
        if args.workload in ("serving", "sweep"):
            print(json.dumps({"impl": "reference", "unavailable": f"no oracle counterpart of the {args.workload} "
                                                                  "mode; it is measured on the GPU path only"}))
            return 0
        return run_reference(args)
    if args.workload == "serving":
        return run_serving(args)
    if args.workload == "sweep":
        return run_sweep(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
