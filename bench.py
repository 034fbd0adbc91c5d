"""Benchmark of the 4D SlingBAG hot path on GB300.

Headline (one JSON line on rank 0): ball-sensor-sample contributions per
second of one forward + FP64 loss/residual + adjoint step on the static
100k-ball workload (vessel tree in a 30 mm cube, 576 sensors on a 55 mm
hemisphere, 4096 samples at 40 MHz), inputs resident in HBM, L2 flushed
before every timed step.  Extra keys: end-to-end through host buffers, the
dominant kernel's roofline, the FP64 oracle timed on the host cores, 4D IR
iterations/s (100k balls x 20 frames) batched in a CUDA graph vs plain
per-frame launches, 16 uneven scenes in persistent launches, the imaging
tools (UBP, splat, MAP, SSIM) on the simulated heart, and the 4D
reconstruction quality against ground truth next to UBP, and the 4D IR
iteration on 1M balls x 50 frames, batched in a CUDA graph vs per-frame.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs under torchrun as independent replicas (the path needs no
exchange at one scene per GPU); value = all ranks' contributions / max time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ball-sensor-sample contributions/sec (fwd+adjoint) and 4D IR iterations/sec vs per-frame"
UNIT = "contributions/s"
# Algorithmic FP32 operations per contribution (one in-window (frame, sensor,
# ball, sample) term), an FMA counting as one operation: forward 6 (tau step,
# tau^2, scale, A*tau, *E, accumulate) and adjoint 10, each plus one ex2 on the
# SFU.  These are the per-contribution counts the roofline is reported on.
FWD_OPS = 6
ADJ_OPS = 10
EX2_PER_CONTRIB = 1
SM_MAX_MHZ_NOMINAL = 2070.0
FP32_LANES_NOMINAL = 128

# DRAM traffic per launch (ncu dram__bytes_read.sum + dram__bytes_write.sum)
# of the static-100k step's kernels, recorded with the SHA-256 of the sources
# the kernel was built from; a recorded figure is reported only while those
# sources are unchanged.
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "traffic_static100k.json")
KERNEL_SOURCES = {
    "forward": ["pa_forward.cu", "pa_common.cuh", "pa_internal.h"],
    "adjoint": ["pa_adjoint.cu", "pa_common.cuh", "pa_internal.h"],
}


def sources_sha256(kind: str) -> str:
    """SHA-256 of the kernel's sources with comments and blank lines removed,
    so that edits to comments alone keep a recorded capture valid."""
    import hashlib
    import re
    h = hashlib.sha256()
    for name in KERNEL_SOURCES[kind]:
        with open(os.path.join(ROOT, "paper_2412_03898_gb300", "csrc", name)) as fh:
            src = fh.read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        code = "\n".join(line.rstrip() for line in src.splitlines() if line.strip())
        h.update(code.encode())
    return h.hexdigest()


def recorded_traffic(kind: str):
    """Bytes per launch of the `kind` kernel(s) from the recorded ncu capture,
    or None when there is none or the sources changed since."""
    try:
        with open(TRAFFIC_FILE) as fh:
            rec = json.load(fh)[kind]
    except (OSError, ValueError, KeyError):
        return None
    if rec.get("sources_sha256") != sources_sha256(kind):
        return None
    return rec.get("bytes_per_step")


def fp32_peak(rates: dict, sms: int) -> dict:
    """FP32 and ex2 peaks of this GPU from its measured unit rates: the faster
    of the scalar and packed FMA lane rates, and the SFU ex2 rate, per SM per
    clock, times the SM count and the clock seen during the probe."""
    lanes = max(rates["ffma_lanes_per_sm_clk"], rates["ffma2_lanes_per_sm_clk"])
    mhz = rates["sm_mhz"]
    return {"lanes_per_sm_clk": lanes, "sm_mhz": mhz, "ops_per_s": lanes * sms * mhz * 1e6,
            "ex2_per_s": rates["ex2_per_sm_clk"] * sms * mhz * 1e6}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-4d", action="store_true", help="skip the 4D IR comparison")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle cpu_baseline leg")
    ap.add_argument("--steps-4d", type=int, default=3)
    ap.add_argument("--no-batched", action="store_true", help="skip the 16-scene batched comparison")
    ap.add_argument("--steps-batched", type=int, default=2)
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--no-spatial-order", action="store_true",
                    help="keep the generator's ball order instead of storing the cloud in Morton order")
    ap.add_argument("--no-imaging", action="store_true", help="skip the UBP / splat / MAP / SSIM leg")
    ap.add_argument("--no-static", action="store_true",
                    help="skip the static-100k headline step (prints the other legs only; for profiling a leg)")
    ap.add_argument("--no-large4d", action="store_true",
                    help="skip the 1M-ball, 50-frame IR iterations (4d-1m-50f; batched graph vs per-frame)")
    ap.add_argument("--heart-ir", type=int, default=0, metavar="ITERS",
                    help="add the simulated-heart 4D reconstruction (Sec. 3.1) with this many IR iterations")
    ap.add_argument("--ir-quality-iters", type=int, default=160,
                    help="IR iterations of the 4D reconstruction-quality leg (0 = skip)")
    a = ap.parse_args()
    a.warmup = max(a.warmup, 3)
    return a


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        sm, smax, power = [], [], []
        reasons = set()
        names = ["active", "hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                    power.append(float(parts[3]))
                except ValueError:
                    continue
                for nm, val in zip(names[1:], parts[5:9]):
                    if val.lower().startswith("active"):
                        reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        # samples under load: drawing well above the idle floor
        pmin = min(power)
        loaded = [s for s, p in zip(sm, power) if p >= pmin + 0.25 * (max(power) - pmin)] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm), "power_w_max": max(power)}


# ---------------------------------------------------------------------------
# distributed helpers (replicas; barrier + max over ranks only)
# ---------------------------------------------------------------------------
def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl == "ours" else "gloo"
        dist.init_process_group(backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(v: float, world: int, device) -> float:
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------------------
# CPU baseline: the FP64 oracle on a bounded sample of the same workload
# ---------------------------------------------------------------------------
def oracle_sample_step(sc, pick, g):
    import oracle
    t0 = time.perf_counter()
    y, n = oracle.forward(sc.balls, sc.sensors[:, pick], sc.c, sc.fs, sc.t0, sc.n_samples, sc.kappa)
    t1 = time.perf_counter()
    oracle.adjoint_state(sc.balls, sc.sensors[:, pick], sc.c, sc.fs, sc.t0, sc.n_samples, sc.kappa, g)
    t2 = time.perf_counter()
    return n, t1 - t0, t2 - t1


def cpu_baseline(sc, n_sensors_sample=None, seed=0):
    import oracle
    rng = np.random.default_rng(seed)
    k = sc.n_sensors if n_sensors_sample is None else n_sensors_sample
    pick = np.sort(rng.choice(sc.n_sensors, k, replace=False))
    g = rng.standard_normal((1, len(pick), sc.n_samples)).astype(np.float32)
    n, tf, ta = oracle_sample_step(sc, pick, g)
    return {"value": n / (tf + ta), "unit": UNIT, "cores": oracle.max_threads(), "kind": "oracle",
            "sample": f"{sc.name}: all {sc.n_balls} balls x {len(pick)} of {sc.n_sensors} sensors x "
                      f"{sc.n_samples} samples, forward + adjoint in FP64 ({n} contributions, "
                      f"{tf + ta:.1f} s)"}


def cpu_baseline_single_core(sc, n_sensors_sample=36, seed=0):
    """The oracle on one host core, on a sensor sample of the same workload
    (the multi-core figure above uses every core)."""
    import oracle
    cores = oracle.max_threads()
    rng = np.random.default_rng(seed)
    pick = np.sort(rng.choice(sc.n_sensors, n_sensors_sample, replace=False))
    g = rng.standard_normal((1, len(pick), sc.n_samples)).astype(np.float32)
    t0 = time.perf_counter()
    _, n = oracle.forward(sc.balls, sc.sensors[:, pick], sc.c, sc.fs, sc.t0, sc.n_samples, sc.kappa, nthreads=1)
    oracle.adjoint_state(sc.balls, sc.sensors[:, pick], sc.c, sc.fs, sc.t0, sc.n_samples, sc.kappa, g, nthreads=1)
    dt = time.perf_counter() - t0
    # the thread count set above persists in the oracle library: put it back
    oracle.forward(sc.balls[:, :4], sc.sensors[:, :1], sc.c, sc.fs, sc.t0, sc.n_samples, sc.kappa, nthreads=cores)
    return {"value": n / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{sc.name}: all {sc.n_balls} balls x {len(pick)} of {sc.n_sensors} sensors x "
                      f"{sc.n_samples} samples, forward + adjoint in FP64 ({n} contributions, {dt:.1f} s)"}


def run_reference(args):
    world, rank, local = dist_setup(args)
    if rank != 0:
        return 0
    import oracle
    import pa_inputs
    sc = pa_inputs.config_scene(2)
    rng = np.random.default_rng(1)
    nsamp = 64  # ~1/9 of the workload per step (about a second on 16 cores)
    total_n, total_t = 0, 0.0
    for i in range(args.warmup + args.steps):
        pick = np.sort(rng.choice(sc.n_sensors, nsamp, replace=False))
        g = rng.standard_normal((1, nsamp, sc.n_samples)).astype(np.float32)
        n, tf, ta = oracle_sample_step(sc, pick, g)
        if i >= args.warmup:
            total_n += n
            total_t += tf + ta
    value = total_n / total_t
    sample = (f"{sc.name}: all {sc.n_balls} balls x {nsamp} random sensors x {sc.n_samples} samples per step, "
              f"forward + adjoint in FP64")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total_t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": CONFIG_DESC, "sample": sample},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.max_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


CONFIG_DESC = ("static-100k: 100,000-ball synthetic vessel tree (20 branching tubes, radii 0.2-1.5 mm, 30 mm cube), "
               "a~U(0.1,0.4) mm, p~U(0.2,1.0); 576 sensors on a 55 mm Fibonacci hemisphere; c=1.5 mm/us, 40 MHz, "
               "4096 samples, kappa=5; forward + FP64 loss/residual + adjoint")


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def run_legs(args, pa, pa_inputs, dev, flush) -> dict:
    """The legs beside the headline (each skipped by its --no-* switch)."""
    out = {}
    if not args.no_4d:
        out["ir4d"] = bench_4d(args, pa, pa_inputs, dev, flush)
    if not args.no_batched:
        out["batched"] = bench_batched(args, pa, pa_inputs, dev, flush)
    if not args.no_imaging:
        out["imaging"] = bench_imaging(args, pa, pa_inputs, dev, flush)
    if args.ir_quality_iters > 0 and not args.no_4d:
        out["ir_quality"] = bench_ir_quality(args, pa, pa_inputs, dev)
    if not args.no_large4d:
        out["large4d"] = bench_large4d(args, pa, pa_inputs, dev)
    if args.heart_ir > 0:
        out["heart_ir"] = bench_heart_ir(args, pa, pa_inputs, dev)
    return out


def run_ours(args):
    import torch
    world, rank, local = dist_setup(args)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import pa_inputs
    import paper_2412_03898_gb300 as pa

    if args.no_static:
        flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
        legs = run_legs(args, pa, pa_inputs, dev, flush)
        if rank == 0:
            print(json.dumps({"metric": METRIC, "note": "legs only (--no-static): no headline value", **legs}))
        return 0

    sc = pa_inputs.config_scene(2)
    n = sc.n_balls
    to_dev = lambda a: pa.pad_last(torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(dev))
    state = to_dev(sc.balls)[None].contiguous()
    if not args.no_spatial_order:
        # storage layout (set-up, not timed): the cloud in Morton order of its
        # centres, by the library's own pa_spatial_order; every sum of the step
        # is over all balls, so only the forward's tile boxes change
        state = pa.gather_rows(state, pa.spatial_order(state, n))
    sensors = torch.from_numpy(sc.sensors).to(dev)
    geom = pa.Geometry(sensors, sc.c, sc.fs, sc.t0, sc.n_samples, sc.kappa)
    # measured data: the forward of a perturbed cloud (GT differs from the model)
    gt = sc.balls.copy()
    rng = np.random.default_rng(42)
    gt[4] *= rng.uniform(0.9, 1.1, n).astype(np.float32)
    gt[:3] += rng.normal(0, 0.01, (3, n)).astype(np.float32)
    meas = pa.forward(geom, to_dev(gt)[None].contiguous(), n)
    torch.cuda.synchronize()
    C = pa.count_contributions(geom, state, n)
    tiles = None
    if not args.no_autotune:
        from paper_2412_03898_gb300.autotune import tune_forward
        tiles = tune_forward(geom, state, n)  # set-up, not timed
    plan = pa.forward_plan(geom, state, n, tiles=tiles)
    # measured unit rates of this GPU (set-up, not timed): the roofline's
    # denominator
    rates = pa.measure_unit_rates()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    fws = torch.empty(max(pa.forward_workspace_size(geom, state, n, tiles=tiles), 16), dtype=torch.uint8, device=dev)
    lws = torch.empty(1 << 20, dtype=torch.uint8, device=dev)
    traces = torch.empty(1, geom.n_sensors, geom.n_samples, device=dev)
    resid = torch.empty_like(traces)
    loss = torch.empty(1, dtype=torch.float64, device=dev)
    gstate = torch.empty_like(state)
    aws = torch.empty(256, dtype=torch.uint8, device=dev)  # the adjoint's work-queue counter
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def step(ev=None):
        if ev is not None:
            ev[0].record(stream)
        pa.forward(geom, state, n, out=traces, workspace=fws, tiles=tiles)
        if ev is not None:
            ev[1].record(stream)
        pa.residual_loss(traces, meas, want_loss=True, want_resid=True, loss_out=loss, resid_out=resid,
                         workspace=lws)
        if ev is not None:
            ev[2].record(stream)
        pa.adjoint(geom, resid, state=state, n=n, out=gstate, workspace=aws)
        if ev is not None:
            ev[3].record(stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    pa.device_error()

    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(args.steps)]
    barrier(world)
    torch.cuda.synchronize()
    for k in range(args.steps):
        flush.zero_()  # write 512 MB > L2 between timed steps (not timed)
        step(evs[k])
    torch.cuda.synchronize()
    barrier(world)
    t_fwd = [e[0].elapsed_time(e[1]) for e in evs]
    t_loss = [e[1].elapsed_time(e[2]) for e in evs]
    t_adj = [e[2].elapsed_time(e[3]) for e in evs]
    t_step = [e[0].elapsed_time(e[3]) for e in evs]
    total_ms = max_over_ranks(sum(t_step), world, dev)
    ms_per_step = total_ms / args.steps
    value = world * C * args.steps / (total_ms * 1e-3)

    # end to end through host buffers: inputs H2D from pinned memory, result D2H
    h_state = state.cpu().pin_memory()
    h_meas = meas.cpu().pin_memory()
    h_sens = sensors.cpu().pin_memory()
    h_loss = torch.empty(1, dtype=torch.float64).pin_memory()
    h_grad = torch.empty(gstate.shape, dtype=torch.float32).pin_memory()
    e2e_in = h_state.numel() * 4 + h_meas.numel() * 4 + h_sens.numel() * 4
    e2e_out = h_loss.numel() * 8 + h_grad.numel() * 4
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e2e_ms = 0.0
    for k in range(args.steps):
        flush.zero_()
        e0.record(stream)
        state.copy_(h_state, non_blocking=True)
        meas.copy_(h_meas, non_blocking=True)
        sensors.copy_(h_sens, non_blocking=True)
        step()
        h_loss.copy_(loss, non_blocking=True)
        h_grad.copy_(gstate, non_blocking=True)
        e1.record(stream)
        e1.synchronize()
        e2e_ms += e0.elapsed_time(e1)
    e2e_ms = max_over_ranks(e2e_ms, world, dev)
    pa.device_error()

    legs = run_legs(args, pa, pa_inputs, dev, flush)
    clocks = sampler.stop()

    fwd_avg = statistics.mean(t_fwd)
    adj_avg = statistics.mean(t_adj)
    peak = fp32_peak(rates, sms)
    if fwd_avg >= adj_avg:
        dom, ops, dur, kind = "forward (k_forward + split reduce)", FWD_OPS, fwd_avg, "forward"
    else:
        dom, ops, dur, kind = "adjoint (k_adjoint_static)", ADJ_OPS, adj_avg, "adjoint"
    achieved = C * ops / (dur * 1e-3)
    launches_per_step = 1 + (1 if plan["n_splits"] > 1 else 0) + 2 + 1
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": CONFIG_DESC, "n_balls": n, "n_sensors": geom.n_sensors,
                   "n_samples": geom.n_samples, "contributions_per_step": C,
                   "l2": "flushed (512 MB write) before every timed step", "forward_plan": plan,
                   "forward_tiles": "autotuned" if tiles is not None else "default",
                   "ball_order": "generator (tubes)" if args.no_spatial_order
                   else "Morton order of the centres (pa_spatial_order, set-up)",
                   "parallelism": f"replicas x{world}"},
        "clocks": clocks,
        "e2e": {"value": world * C * args.steps / (e2e_ms * 1e-3), "unit": UNIT, "h2d_bytes_per_step": e2e_in,
                "d2h_bytes_per_step": e2e_out},
        "gpu_launches": launches_per_step * args.steps,
        "roofline": {"bound": "alu", "kernel": dom, "achieved": achieved / 1e12, "peak": peak["ops_per_s"] / 1e12,
                     "unit": "TFLOP/s", "frac": achieved / peak["ops_per_s"], "traffic": recorded_traffic(kind),
                     "note": f"FP32 operations (FMA = 1) per contribution: forward {FWD_OPS}, adjoint {ADJ_OPS} "
                             f"(+{EX2_PER_CONTRIB} ex2 each); peak = measured FP32 FMA rate "
                             f"{peak['lanes_per_sm_clk']:.1f} lane ops per SM per clock x {sms} SMs x "
                             f"{peak['sm_mhz']:.0f} MHz (pa_measure_unit_rates, of measured)",
                     "per_kernel_frac": {"forward": C * FWD_OPS / (fwd_avg * 1e-3) / peak["ops_per_s"],
                                         "adjoint": C * ADJ_OPS / (adj_avg * 1e-3) / peak["ops_per_s"]},
                     "ex2_frac": {"forward": C * EX2_PER_CONTRIB / (fwd_avg * 1e-3) / peak["ex2_per_s"],
                                  "adjoint": C * EX2_PER_CONTRIB / (adj_avg * 1e-3) / peak["ex2_per_s"]}},
        "unit_rates": rates,
        "kernels_ms": {"forward": fwd_avg, "loss": statistics.mean(t_loss), "adjoint": adj_avg},
        "fwd_contrib_per_s": C / (fwd_avg * 1e-3), "adj_contrib_per_s": C / (adj_avg * 1e-3),
    }
    line.update(legs)
    if rank == 0 and world == 1 and not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline(sc)
        line["cpu_baseline_single_core"] = cpu_baseline_single_core(sc)
    if rank == 0:
        print(json.dumps(line))
    return 0


def bench_4d(args, pa, pa_inputs, dev, flush):
    """4D IR iterations/s on 100k canonical balls x 20 frames (576 sensors,
    4096 samples): batched + CUDA graph vs plain per-frame launches."""
    import torch
    from paper_2412_03898_gb300.ir import GGBallIR, init_deformation
    sc = pa_inputs.config_scene(3)
    n = sc.n_balls
    F = sc.n_frames
    to_dev = lambda a: pa.pad_last(torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(dev))
    sensors = torch.from_numpy(sc.sensors).to(dev)
    geom = pa.Geometry(sensors, sc.c, sc.fs, sc.t0, sc.n_samples, sc.kappa)
    gt = to_dev(sc.frames).contiguous()
    meas = pa.forward(geom, gt, n)
    t = torch.from_numpy(pa_inputs.frame_times(F)).to(dev)
    canon = to_dev(sc.balls).contiguous()
    nb = 65
    deform = init_deformation(nb, canon.shape[-1], dev, omega_scale=0.02, seed=1)
    if not args.no_spatial_order:
        # storage layout (set-up): Morton order of the canonical centres
        perm = pa.spatial_order(canon, n)
        canon, deform = pa.gather_rows(canon, perm), pa.gather_rows(deform, perm)
    del gt
    out = {"workload": f"{sc.name}: {n} canonical balls, {F} frames, Nb={nb}, {sc.n_sensors} sensors, "
                       f"{sc.n_samples} samples", "steps": args.steps_4d,
           "ball_order": "generator (tubes)" if args.no_spatial_order else "Morton (pa_spatial_order, set-up)"}
    C = pa.count_contributions(geom, pa.deform_balls(canon, deform[0], deform[1], deform[2], t, n), n)
    out["contributions_per_iter"] = C
    res = {}
    for mode in ("batched_graph", "per_frame"):
        ir = GGBallIR(geom, canon.clone(), deform.clone(), t, meas, n)
        fn = ir.step_graph if mode == "batched_graph" else ir.step_per_frame
        for _ in range(2):
            fn()
        torch.cuda.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ms = 0.0
        for _ in range(args.steps_4d):
            flush.zero_()
            ev[0].record()
            fn()
            ev[1].record()
            ev[1].synchronize()
            ms += ev[0].elapsed_time(ev[1])
        pa.device_error()
        res[mode] = args.steps_4d / (ms * 1e-3)
        out[f"{mode}_iters_per_s"] = res[mode]
        out[f"{mode}_launches_per_iter"] = ir.launches_per_step(per_frame=(mode == "per_frame"))
        out[f"{mode}_loss"] = float(ir.loss.sum().item())
        del ir
    out["speedup_batched_vs_per_frame"] = res["batched_graph"] / res["per_frame"]
    out["frames_per_launch"] = GGBallIR(geom, canon, deform, t, meas, n).frames_per_chunk()
    out["contrib_per_s_batched"] = C * res["batched_graph"]
    out["contrib_per_s_per_frame"] = C * res["per_frame"]
    return out


# Algorithmic FP32 operations per UBP (voxel, sensor) pair: r - r_s (3),
# |r - r_s|^2 (3), n . (r - r_s) (3), d and cos/d^2 (4), fractional sample (1),
# interpolation (2), weighted sums (2) = 18 (+1 rsqrt on the SFU).
UBP_OPS = 18


def bench_imaging(args, pa, pa_inputs, dev, flush):
    """Imaging on the simulated heart (Sec. 3.1: 72,006 balls, 1,024 sensors on
    a full 60 mm Fibonacci sphere, 4,096 samples): UBP of frame 0 onto 256^3
    voxels of 0.2 mm over the (-25.6, 25.6) mm cube, the ball cloud splatted
    onto the same grid, the XY / YZ / XZ MAPs of both and their SSIMs."""
    import torch
    sc = pa_inputs.heart_phantom()
    n = sc.n_balls
    st = pa.pad_last(torch.from_numpy(sc.frames[0]).to(dev)).contiguous()
    geom = pa.Geometry(torch.from_numpy(sc.sensors).to(dev), sc.c, sc.fs, sc.t0, sc.n_samples, sc.kappa)
    y = pa.forward(geom, st[None], n)[0].contiguous()
    nvox = 256
    grid = pa.Grid.cube(25.6, nvox)
    b = torch.empty_like(y)
    vol = torch.empty(grid.shape, dtype=torch.float32, device=dev)
    gt = torch.empty_like(vol)

    def timed(fn, reps):
        fn()
        torch.cuda.synchronize()
        ms = []
        for _ in range(reps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        return statistics.median(ms)

    out = {"workload": f"heart-sim1 frame 0: {n} balls, {geom.n_sensors} sensors (60 mm sphere), "
                       f"{geom.n_samples} samples; grid {nvox}^3 x {grid.h:.2f} mm"}
    out["ubp_filter_ms"] = timed(lambda: pa.ubp_filter(y, sc.fs, sc.t0, out=b), 5)
    ubp_ms = timed(lambda: pa.ubp(geom, b, grid, out=vol), 3)
    pairs = geom.n_sensors * nvox ** 3
    out["ubp_ms"] = ubp_ms
    out["ubp_voxel_sensor_pairs_per_s"] = pairs / (ubp_ms * 1e-3)
    rates = pa.measure_unit_rates()
    peak = fp32_peak(rates, torch.cuda.get_device_properties(dev).multi_processor_count)["ops_per_s"]
    out["ubp_alu_frac"] = pairs * UBP_OPS / (ubp_ms * 1e-3) / peak
    out["splat_ms"] = timed(lambda: pa.splat(st, grid, sc.kappa, n, out=gt), 3)
    out["maps_ms"] = timed(lambda: pa.maps(vol, grid), 5)
    mu, mg = pa.maps(vol, grid), pa.maps(gt, grid)
    out["ssim_ms"] = timed(lambda: [pa.ssim(u, g, minmax=True) for u, g in zip(mu, mg)], 5)
    out["ubp_vs_gt_map_ssim"] = {k: float(pa.ssim(u, g, minmax=True)) for k, u, g in zip(("xy", "yz", "xz"), mu, mg)}
    pa.device_error()
    return out


def bench_heart_ir(args, pa, pa_inputs, dev):
    """The paper's first simulation (Sec. 3.1) on synthetic data: the 17-frame
    simulated heart seen by 1,024 sensors on a 60 mm sphere, reconstructed by
    the 4D IR loop from the ground-truth frame 0 with zero deformation, and by
    UBP frame by frame; XY / YZ / XZ MAP-SSIM against the splatted ground truth
    at the first, middle and last frames (Fig. 5-7)."""
    import torch
    from paper_2412_03898_gb300.ir import GGBallIR, init_deformation
    sc = pa_inputs.heart_phantom()
    n, F = sc.n_balls, sc.n_frames
    to_dev = lambda a: pa.pad_last(torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(dev))
    geom = pa.Geometry(torch.from_numpy(sc.sensors).to(dev), sc.c, sc.fs, sc.t0, sc.n_samples, sc.kappa)
    gt = to_dev(sc.frames).contiguous()
    meas = pa.forward(geom, gt, n)
    t = torch.from_numpy(pa_inputs.frame_times(F)).to(dev)
    ir = GGBallIR(geom, to_dev(sc.frames[0]).contiguous(), init_deformation(65, gt.shape[-1], dev), t, meas, n)
    grid = pa.Grid.cube(25.6, 256)
    frames = [0, F // 2, F - 1]
    vol = torch.empty(grid.shape, dtype=torch.float32, device=dev)
    bfilt = torch.empty(geom.n_sensors, geom.n_samples, dtype=torch.float32, device=dev)
    gt_m = {}
    for f in frames:
        pa.splat(gt[f], grid, sc.kappa, n, out=vol)
        gt_m[f] = [m.clone() for m in pa.maps(vol, grid)]

    def ssim_model():
        state = pa.deform_balls(ir.canon, ir.deform[0], ir.deform[1], ir.deform[2], t, n)
        out = {}
        for f in frames:
            pa.splat(state[f], grid, sc.kappa, n, out=vol)
            out[f] = [float(pa.ssim(u, g, minmax=True)) for u, g in zip(pa.maps(vol, grid), gt_m[f])]
        return out

    before = ssim_model()
    loss0 = float(ir.step().sum())
    ir.capture()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ev[0].record()
    for _ in range(args.heart_ir - 2):
        ir.step_graph()
    ev[1].record()
    ev[1].synchronize()
    loss1 = float(ir.loss.sum())
    after = ssim_model()
    ubp = {}
    for f in frames:
        pa.ubp_filter(meas[f], sc.fs, sc.t0, out=bfilt)
        pa.ubp(geom, bfilt, grid, out=vol)
        ubp[f] = [float(pa.ssim(u, g, minmax=True)) for u, g in zip(pa.maps(vol, grid), gt_m[f])]
    pa.device_error()
    views = ("xy", "yz", "xz")
    fmt = lambda d: {f"frame{f + 1}": dict(zip(views, v)) for f, v in d.items()}
    return {"workload": f"{sc.name}: {n} balls, {F} frames, Nb = 65, {geom.n_sensors} sensors; MAPs on "
                        f"{grid.shape[0]}^3 x {grid.h:.2f} mm", "iterations": args.heart_ir,
            "ms_per_iteration": ev[0].elapsed_time(ev[1]) / max(args.heart_ir - 2, 1),
            "loss_first": loss0, "loss_last": loss1, "map_ssim_4d_before": fmt(before),
            "map_ssim_4d_after": fmt(after), "map_ssim_ubp": fmt(ubp)}


def bench_large4d(args, pa, pa_inputs, dev):
    """The paper's large-scale case (4d-1m-50f): one 4D IR iteration (deform,
    forward, FP64 loss, adjoint, chain rule, Adam) over 1,000,000 balls x 50
    frames with 1,024 sensors and 4,096 samples, in its two execution forms:
    all frames per launch replayed from one CUDA graph, and 50 plain per-frame
    launch sequences; CUDA events on the launching stream, one warm-up of each
    form first.  L2 is not flushed (an iteration moves tens of GB)."""
    import torch
    from paper_2412_03898_gb300.ir import GGBallIR, init_deformation
    sc = pa_inputs.config_scene(4)
    n, F = sc.n_balls, sc.n_frames
    to_dev = lambda a: pa.pad_last(torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(dev))
    geom = pa.Geometry(torch.from_numpy(sc.sensors).to(dev), sc.c, sc.fs, sc.t0, sc.n_samples, sc.kappa)
    # ground-truth motion (radial pulsation and drift), generated here: the
    # workload stores no frames
    gt = to_dev(pa_inputs.gt_motion_frames(sc.balls, sc.axis, F)).contiguous()
    meas = pa.forward(geom, gt, n)
    C = pa.count_contributions(geom, gt, n)
    del gt
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    torch.cuda.reset_peak_memory_stats(dev)
    base = torch.cuda.memory_allocated(dev)
    t = torch.from_numpy(pa_inputs.frame_times(F)).to(dev)
    canon = to_dev(sc.balls).contiguous()
    if not args.no_spatial_order:
        # storage layout (set-up): Morton order of the canonical centres (the
        # initial deformation is the same for every ball)
        canon = pa.gather_rows(canon, pa.spatial_order(canon, n))
    ir = GGBallIR(geom, canon, init_deformation(65, canon.shape[-1], dev), t, meas, n)
    out = {"workload": f"{sc.name}: {n} balls, {F} frames, Nb = 65, {geom.n_sensors} sensors, {geom.n_samples} "
                       "samples", "contributions_per_iteration": C,
           "ball_order": "generator (tubes)" if args.no_spatial_order else "Morton (pa_spatial_order, set-up)"}

    def timed(fn, iters):
        torch.cuda.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev[0].record()
        for _ in range(iters):
            fn()
        ev[1].record()
        ev[1].synchronize()
        return ev[0].elapsed_time(ev[1]) * 1e-3 / iters

    ir.step()
    ir.capture()
    s_graph = timed(ir.step_graph, 2)
    ir.step_per_frame()
    s_pf = timed(ir.step_per_frame, 1)
    pa.device_error()
    out["frames_per_launch"] = ir.frames_per_chunk()
    out.update({"iters_per_s": 1.0 / s_graph, "seconds_per_iteration": s_graph,
                "per_frame_iters_per_s": 1.0 / s_pf, "per_frame_seconds_per_iteration": s_pf,
                "speedup_batched_vs_per_frame": s_pf / s_graph,
                "contrib_per_s": C / s_graph, "per_frame_contrib_per_s": C / s_pf,
                "iterations_timed": {"batched_graph": 2, "per_frame": 1},
                "device_memory_gb": (torch.cuda.max_memory_allocated(dev) - base) / 1e9,
                "device_memory_note": "peak bytes allocated by the IR beyond the measurements: parameters, Adam "
                                      "moments, gradients, traces, residual and one frame chunk of states; no "
                                      "[F][5][N] buffer"})
    return out


def bench_ir_quality(args, pa, pa_inputs, dev):
    """Reconstruction quality of the 4D IR loop (Sec. 2.2 stage 2, Sec. 3.2
    hyper-parameters) on 4d-100k-20f: the canonical cloud starts at the
    ground-truth frame 0 with zero deformation, the measurements are the
    forward projections of the 20 ground-truth frames (radial pulsation and
    drift), and the whole iteration replays from one CUDA graph.  Reports the
    loss, the RMS position error against the ground-truth motion, and the SSIM
    of XY / YZ / XZ MAPs of the splatted model against the splatted ground
    truth at the first, middle and last frames, next to UBP from the same
    576-sensor measurements (the paper's Tab. 1 columns, on synthetic data)."""
    import torch
    from paper_2412_03898_gb300.ir import GGBallIR, init_deformation
    sc = pa_inputs.config_scene(3)
    n, F = sc.n_balls, sc.n_frames
    to_dev = lambda a: pa.pad_last(torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(dev))
    geom = pa.Geometry(torch.from_numpy(sc.sensors).to(dev), sc.c, sc.fs, sc.t0, sc.n_samples, sc.kappa)
    gt = to_dev(sc.frames).contiguous()
    meas = pa.forward(geom, gt, n)
    t = torch.from_numpy(pa_inputs.frame_times(F)).to(dev)
    canon = to_dev(sc.frames[0]).contiguous()
    deform = init_deformation(65, canon.shape[-1], dev)
    ir = GGBallIR(geom, canon, deform, t, meas, n)
    grid = pa.Grid.cube(15.0, 192)
    frames = [0, F // 2, F - 1]
    vol = torch.empty(grid.shape, dtype=torch.float32, device=dev)
    ref = torch.empty_like(vol)
    bfilt = torch.empty(geom.n_sensors, geom.n_samples, dtype=torch.float32, device=dev)

    def gt_maps(f):
        pa.splat(gt[f], grid, sc.kappa, n, out=ref)
        return pa.maps(ref, grid)

    gt_m = {f: [m.clone() for m in gt_maps(f)] for f in frames}

    def model_quality():
        state = pa.deform_balls(ir.canon, ir.deform[0], ir.deform[1], ir.deform[2], t, n)
        err = (state[:, :3, :n] - gt[:, :3, :n]).pow(2).sum(1).mean().sqrt().item()
        ss = {}
        for f in frames:
            pa.splat(state[f], grid, sc.kappa, n, out=vol)
            ss[f] = [float(pa.ssim(u, g, minmax=True)) for u, g in zip(pa.maps(vol, grid), gt_m[f])]
        return err, ss

    pos0, ss0 = model_quality()
    loss0 = float(ir.step().sum())
    ir.capture()
    for _ in range(args.ir_quality_iters - 2):
        ir.step_graph()
    loss1 = float(ir.loss.sum())
    pos1, ss1 = model_quality()
    ubp = {}
    for f in frames:
        pa.ubp_filter(meas[f], sc.fs, sc.t0, out=bfilt)
        pa.ubp(geom, bfilt, grid, out=vol)
        ubp[f] = [float(pa.ssim(u, g, minmax=True)) for u, g in zip(pa.maps(vol, grid), gt_m[f])]
    pa.device_error()
    views = ("xy", "yz", "xz")
    fmt = lambda d: {f"frame{f + 1}": dict(zip(views, v)) for f, v in d.items()}
    return {"workload": f"{sc.name}: {n} balls, {F} frames, Nb = 65, {geom.n_sensors} sensors; MAPs on "
                        f"{grid.shape[0]}^3 x {grid.h:.3f} mm",
            "iterations": args.ir_quality_iters, "loss_first": loss0, "loss_last": loss1,
            "position_rmse_mm_first": pos0, "position_rmse_mm_last": pos1,
            "map_ssim_4d_before": fmt(ss0), "map_ssim_4d_after": fmt(ss1), "map_ssim_ubp": fmt(ubp)}


def bench_batched(args, pa, pa_inputs, dev, flush):
    """16 uneven scenes (N log-uniform in [1e4, 5e5], S in {256, 576, 1024},
    T in [2048, 4096], 1-10 frames): forward + static adjoint of all scenes
    as two persistent launches replayed from one CUDA graph, vs plain
    per-scene launches."""
    import torch
    from paper_2412_03898_gb300.autotune import tune_batched
    raw = pa_inputs.config_scene(5)
    to_dev = lambda a: pa.pad_last(torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(dev))
    scenes = []
    C = 0
    for sc in raw:
        st = to_dev(sc.frames if sc.frames is not None else sc.balls[None]).contiguous()
        geom = pa.Geometry(torch.from_numpy(sc.sensors).to(dev), sc.c, sc.fs, sc.t0, sc.n_samples, sc.kappa)
        C += pa.count_contributions(geom, st, sc.n_balls)
        b = pa.Scene(geom, st, sc.n_balls)
        b.traces = torch.empty(b.F, geom.n_sensors, geom.n_samples, device=dev)
        b.trace_grad = b.traces  # any residual: the work does not depend on its values
        b.grad_state = torch.empty_like(st)
        scenes.append(b)
    plan = tune_batched(scenes) if not args.no_autotune else None
    arr = (pa._lib.pa_scene * len(scenes))(*[b.struct() for b in scenes])
    ws = torch.empty(int(pa._LIB.pa_batched_workspace_size(arr, len(scenes), plan.handle if plan else None)),
                     dtype=torch.uint8, device=dev)
    ws2 = torch.empty(256, dtype=torch.uint8, device=dev)

    def batched_step():
        pa.forward_batched(scenes, plan=plan, workspace=ws)
        pa.adjoint_batched(scenes, plan=plan, workspace=ws2)

    per_ws = {}
    for b in scenes:
        need = pa.forward_workspace_size(b.geom, b.state, b.n)
        per_ws[id(b)] = torch.empty(max(need, 16), dtype=torch.uint8, device=dev)

    def per_scene_step():
        for b in scenes:
            pa.forward(b.geom, b.state, b.n, out=b.traces, workspace=per_ws[id(b)])
            pa.adjoint(b.geom, b.trace_grad, state=b.state, n=b.n, out=b.grad_state)

    batched_step()
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        batched_step()
    torch.cuda.current_stream().wait_stream(s)
    with torch.cuda.graph(g):
        batched_step()
    out = {"workload": "batched-16: " + ", ".join(f"{b.n}x{b.geom.n_sensors}x{b.geom.n_samples}x{b.F}"
                                                   for b in scenes),
           "contributions_per_step": C, "plan": plan.values() if plan is not None else None, "steps": args.steps_batched}
    for mode, fn in (("graph_persistent", g.replay), ("per_scene", per_scene_step)):
        fn()
        torch.cuda.synchronize()
        ms = 0.0
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for _ in range(args.steps_batched):
            flush.zero_()
            e0.record()
            fn()
            e1.record()
            e1.synchronize()
            ms += e0.elapsed_time(e1)
        out[f"{mode}_ms_per_step"] = ms / args.steps_batched
        out[f"{mode}_contrib_per_s"] = C * args.steps_batched / (ms * 1e-3)
    pa.device_error()
    out["speedup_persistent_vs_per_scene"] = out["per_scene_ms_per_step"] / out["graph_persistent_ms_per_step"]
    return out


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
