"""Throughput of the averaged-Yee field advance on GB300.

Workload (one "step" = one full pass of the hot path: current filter, source,
Algorithm 1, E update, Faraday update): a 2D periodic 4096 x 4096 grid, FP32
storage (FP64 only in reductions), dt = 0.5 dt_CFL, random-phase field
spectrum with power ~ |n|^-2 up to |n| = N/8, a static divergence-free
current (curl of a smooth random potential, Gaussian spectrum of width 16
cells) re-filtered by a 3-pass binomial filter every step, m = 4 sweeps.
All inputs are seeded and synthetic.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line.  Under torchrun (N > 1) every rank advances its own
grid (independent replicas, weak scaling, no collective on the data path).
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

NX = NY = 4096
M_SWEEPS = 4
PASSES = 3
COURANT = 0.5
KMAX = NX // 8
SEED = 1907002
BYTES_PER_CELL = 15 * 4  # read E, B, j (9 x 4 B) + write E, B (6 x 4 B)
METRIC = "Gcell-updates/s per full step (curl+iteration+filter) and % HBM roofline, 1 GB300"
UNIT = "Gcell-updates/s"
WORKLOAD = ("2D periodic 4096x4096 FP32 (FP64 reductions), dt=0.5 dt_CFL, power-law spectrum k_max=N/8, "
            "static solenoidal J (curl of Gaussian-spectrum potential, width 16), 3-pass binomial current "
            "filter every step, m=4 sweeps")
FALLBACK_HBM_GBS = 6800.0
# FP32 work of one 3D cell-step as the z-march kernels evaluate it (an FMA is
# 2 flops, an add or multiply 1): the 1-pass filter of the current, per
# component three x-y rows of (1, 2, 1), their (1, 2, 1) along y and z and the
# scaled subtraction (3 x 21 = 63); the source with the averaged curl factored
# into in-plane terms and 3-point z-combinations (53); each sweep of Algorithm
# 1 with A factored the same way, its 21 in-plane second differences and
# mixed differences and the z-combinations of three components, plus dE'
# (112; four sweeps 448); the E update (3); Faraday, 2 terms x 2 taps x 3
# components (24).  The 27-point stencils as written, one FMA per tap, would
# take 963.
FLOPS_PER_CELL_STEP_3D = 63 + 53 + 4 * 112 + 3 + 24
# FP32 FMA peak from the unit counts and clock: 152 SMs x 128 lanes x 2 flops x 2.07 GHz
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(x, world, device):
    """The largest of every rank's x (a time): an all-reduce MAX when world > 1
    (NCCL on the GPU runs, gloo in the CPU tests)."""
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(cells_per_rank, steps, seconds_max, world):
    """Gcell-updates/s of the whole job: the cell updates of all ranks over the
    slowest rank's time (replicas: every rank advances its own grid)."""
    return world * cells_per_rank * steps / seconds_max / 1e9


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        try:
            with open(path) as f:
                d = json.load(f)
            for key in ("hbm_gbs", "hbm_GBps", "hbm_bandwidth_gbs"):
                if key in d and d[key]:
                    return float(d[key]), f"measured ({key} of MEASURED_PEAKS.json)"
        except Exception:
            pass
    return FALLBACK_HBM_GBS, "fallback (6.8 TB/s, no MEASURED_PEAKS.json)"


def alu_roofline(cells, seconds_per_step, flops_per_cell_step=FLOPS_PER_CELL_STEP_3D):
    """FP32 arithmetic achieved against the FMA peak (the 3D step's flops per
    algorithmic byte, 591 / 60, lie below the ridge 80.5 TFLOP/s / 6.76 TB/s:
    its roof is HBM, this is the secondary one)."""
    achieved = flops_per_cell_step * cells / seconds_per_step / 1e12
    return {"bound": "alu", "achieved": round(achieved, 2), "peak": round(FP32_PEAK_TFLOPS, 1), "unit": "TFLOP/s",
            "frac": round(achieved / FP32_PEAK_TFLOPS, 4), "flops_per_cell_step": flops_per_cell_step,
            "peak_source": "152 SMs x 128 FP32 lanes x 2 flops x 2.07 GHz (unit counts and maximum SM clock)"}


def _ncu_traffic(kernel_name):
    """dram bytes (read + write) per launch of a kernel from the committed ncu
    summary, or None when absent or taken on another version of the kernel."""
    path = os.path.join(ROOT, "profiles", "fused2d_pol_4096_traffic.json")
    if not os.path.exists(path):
        return None
    try:
        with open(path) as f:
            d = json.load(f)
        from ncu_report import kernel_hash
        if d.get("kernel_sha256_16") != kernel_hash():
            return None
        return float(d["dram_bytes_per_launch"][kernel_name])
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 100 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.samples = []
        self.proc = None
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append((time.time(), line.strip()))

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self, t0, t1):
        rows = [s for (t, s) in self.samples if t0 - 0.05 <= t <= t1 + 0.05] or [s for _, s in self.samples[-3:]]
        if not rows:
            return None
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for r in rows:
            parts = [p.strip() for p in r.split(",")]
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except Exception:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def gpu_numa_cpus(index):
    """CPUs of the NUMA node the GPU hangs off (from its PCI device's sysfs
    entry), or None when that is not known."""
    try:
        bus = subprocess.run(["nvidia-smi", "-i", str(index), "--query-gpu=pci.bus_id", "--format=csv,noheader"],
                             capture_output=True, text=True, timeout=20).stdout.strip()
        dom, rest = bus.split(":", 1)
        dev = f"{int(dom, 16):04x}:{rest}".lower()
        with open(f"/sys/bus/pci/devices/{dev}/numa_node") as f:
            node = int(f.read().strip())
        if node < 0:
            return None
        with open(f"/sys/devices/system/node/node{node}/cpulist") as f:
            spec = f.read().strip()
        cpus = set()
        for part in spec.split(","):
            if "-" in part:
                a, b = part.split("-")
                cpus.update(range(int(a), int(b) + 1))
            elif part:
                cpus.add(int(part))
        return (node, cpus) if cpus else None
    except Exception:
        return None


def make_inputs():
    import numpy as np
    from paper_1907_13088_gb300 import synth
    E, B = synth.power_law_fields((NX, NY), KMAX, SEED, dtype=np.float32)
    J = synth.solenoidal_current((NX, NY), SEED + 1, width=16.0, rms=1e-3, dtype=np.float32)
    return E, B, J


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    rank, world, local = _dist()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    from paper_1907_13088_gb300 import build
    if rank == 0 or world == 1:
        build.build()
    if world > 1:
        dist.barrier()
    from paper_1907_13088_gb300 import fmx

    E, B, J = make_inputs()
    g = fmx.Grid((NX, NY), precision=fmx.FMX_F32, m=M_SWEEPS, filter_passes=PASSES, courant=COURANT,
                 engine=fmx.FMX_ENGINE_FUSED)
    g.set_fields(E, B)
    g.set_current(J)
    stream = g.stream
    cells = NX * NY

    def barrier():
        if world > 1:
            dist.barrier()

    # warm-up
    g.step(args.warmup)
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    if rank == 0:
        sampler.start()
        time.sleep(0.3)
    barrier()
    torch.cuda.synchronize()
    l0 = g.launches
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    t0 = time.time()
    ev0.record(stream)
    g.step(args.steps)
    ev1.record(stream)
    torch.cuda.synchronize()
    t1 = time.time()
    barrier()
    launches = g.launches - l0
    ms = ev0.elapsed_time(ev1)
    ms_max = max_over_ranks(ms, world, "cuda")
    clocks = sampler.summary(t0, t1) if rank == 0 else None
    sampler.stop()

    # end to end through the C ABI (fmx_step_host): every step uploads E, B, j
    # from pinned host memory, advances one step and reads E, B back into
    # pinned memory; the upload of step k+1 overlaps the read-back of step k.
    # The pinned buffers are allocated (first touched) from the CPUs of the
    # GPU's own NUMA node.
    e2e_steps = max(3, min(50, args.steps // 20))
    numa = gpu_numa_cpus(local)
    old_aff = os.sched_getaffinity(0)
    if numa:
        try:
            os.sched_setaffinity(0, numa[1])
        except Exception:
            numa = None
    hin = torch.empty((9, 1, NY, NX), dtype=torch.float32).pin_memory().numpy()
    hin[0:3], hin[3:6], hin[6:9] = E, B, J
    hout = torch.empty((6, 1, NY, NX), dtype=torch.float32).pin_memory().numpy()
    hout[:] = 0.0
    g.step_host([(hin, hout)] * 2)
    barrier()
    torch.cuda.synchronize()
    te0 = time.perf_counter()
    g.step_host([(hin, hout)] * e2e_steps)
    torch.cuda.synchronize()
    te1 = time.perf_counter()
    os.sched_setaffinity(0, old_aff)
    e2e_value = whole_job_rate(cells, e2e_steps, max_over_ranks(te1 - te0, world, "cuda"), world)

    # per-kernel durations, CUDA events on the launching stream, after the timed region
    prof_steps = max(50, min(500, args.steps))
    g.profile(True)
    g.step(prof_steps)
    kstats = g.profile_read()
    g.profile(False)

    cpu = cpu_baseline(E, B, J) if (rank == 0 and args.cpu_baseline) else None

    if rank == 0:
        value = whole_job_rate(cells, args.steps, ms_max / 1e3, world)
        peak, peak_src = _peaks()
        dom = max(kstats, key=lambda k: k["total_ms"])
        per_launch_s = dom["total_ms"] / 1e3 / dom["launches"]
        achieved = dom["bytes_per_launch"] / per_launch_s / 1e9
        step_s = (ms / 1e3) / args.steps
        kernels = [{"name": k["name"], "ms_per_launch": round(k["total_ms"] / k["launches"], 5),
                    "algorithmic_bytes_per_launch": k["bytes_per_launch"],
                    "achieved_gbs": round(k["bytes_per_launch"] / (k["total_ms"] / 1e3 / k["launches"]) / 1e9, 1),
                    "ncu_dram_bytes_per_launch": _ncu_traffic(k["name"])} for k in kstats]
        line = {
            "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms_max / args.steps, 6), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "grid": [NX, NY], "cells_per_gpu": cells, "m": M_SWEEPS,
                       "filter_passes": PASSES, "courant": COURANT, "engine": "fused2d (TE + TM kernels)",
                       "l2": "inputs larger than L2 (1.0 GB of fields per step vs 129 MB L2)",
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
            "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                         "frac": round(achieved / peak, 4), "traffic": _ncu_traffic(dom["name"]),
                         "kernel": dom["name"], "peak_source": peak_src,
                         "bytes_per_cell_step": BYTES_PER_CELL,
                         "step": {"achieved": round(BYTES_PER_CELL * cells / step_s / 1e9, 1),
                                  "frac": round(BYTES_PER_CELL * cells / step_s / 1e9 / peak, 4)},
                         "kernels": kernels, "timing": f"CUDA events around each launch, {prof_steps} steps"},
            "cpu_baseline": cpu,
            "e2e": {"value": round(e2e_value, 4), "unit": UNIT, "h2d_bytes_per_step": 9 * 4 * cells,
                    "d2h_bytes_per_step": 6 * 4 * cells, "steps": e2e_steps,
                    "path": "fmx_step_host: per step E, B, j pinned host -> device, one step, E, B -> pinned host; "
                            "upload of step k+1 overlapping read-back of step k",
                    "pinned_numa_node": numa[0] if numa else None},
            "gpu_launches": int(launches),
            "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_batch(args):
    """256 independent 2D grids (sizes log-uniform in 64..1024 per side,
    Courant fractions uniform in 0.3..0.9, FP32, vacuum, m = 4), advanced by
    one persistent launch per step (column-pair TE/TM tiles) replayed from
    CUDA graphs, with the tile
    rows picked by the autotuner; the same grids stepped one fmx_step call per
    grid are timed beside it."""
    import numpy as np
    import torch
    from paper_1907_13088_gb300 import build, synth
    build.build()
    from paper_1907_13088_gb300 import fmx
    sizes = synth.batch_sizes(256, 1907004)
    shapes = [(a, b) for a, b, _ in sizes]
    cfs = [c for _, _, c in sizes]
    cells = sum(a * b for a, b in shapes)
    bt = fmx.Batch(shapes, cfs, m=4)
    chosen = bt.tune(trial_steps=10)
    tiles = bt.tiles()
    # grid-size classes of the tuned work list: which grids run on narrow tiles
    narrow_grids = [i for i in range(len(shapes)) if bt.grid_width(i) < 200]
    size_classes = {}
    for i, (a, b_) in enumerate(shapes):
        cls = "nx<128" if a < 128 else ("nx<256" if a < 256 else ("nx<512" if a < 512 else "nx>=512"))
        d = size_classes.setdefault(cls, {"grids": 0, "narrow_tiles": 0})
        d["grids"] += 1
        d["narrow_tiles"] += int(i in narrow_grids)
    fields = [synth.power_law_fields(sh, max(2, min(sh) // 8), 1907004 + i) for i, sh in enumerate(shapes)]
    for i, (E, B) in enumerate(fields):
        bt.set_fields(i, E, B)
    bt.step(args.warmup)
    bt.sync()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    l0 = bt.launches
    sampler = ClockSampler(0)
    sampler.start()
    time.sleep(0.3)
    t0 = time.time()
    ev0.record(bt.stream)
    bt.step(args.steps)
    ev1.record(bt.stream)
    bt.sync()
    t1 = time.time()
    ms = ev0.elapsed_time(ev1)
    clocks = sampler.summary(t0, t1)
    sampler.stop()
    launches = bt.launches - l0
    # the same grids, one fmx_step call per grid per step (single-grid path)
    grids = []
    for i, (sh, cf) in enumerate(zip(shapes, cfs)):
        g = fmx.Grid(sh, with_current=False, precision=0, m=4, courant=cf, engine=fmx.FMX_ENGINE_FUSED)
        g.set_fields(*fields[i])
        grids.append(g)
    single_steps = max(5, min(50, args.steps // 10))
    for g in grids:
        g.step(2)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(single_steps):
        for g in grids:
            g.step(1)
    e1.record()
    torch.cuda.synchronize()
    single = cells * single_steps / (e0.elapsed_time(e1) / 1e3) / 1e9
    value = cells * args.steps / (ms / 1e3) / 1e9
    peak, peak_src = _peaks()
    achieved = 48 * cells / (ms / 1e3 / args.steps) / 1e9
    line = {
        "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 6), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "batch of 256 independent 2D periodic grids, sizes log-uniform 64..1024 per side "
                               "(seed 1907004), Courant U[0.3, 0.9], FP32, vacuum, m = 4, one persistent launch "
                               "per step replayed from CUDA graphs, autotuned tile rows",
                   "cells_total": cells, "grids": len(shapes), "tuned_tile_rows": chosen or "auto",
                   "tuned_tile_rule": {0: "wide tiles only", 1: "narrow tiles where they compute fewer columns",
                                       2: "narrow tiles everywhere"}[tiles["narrow_rule"]],
                   "tiles": {"wide": tiles["wide"], "narrow": tiles["narrow"], "single_column": tiles["single"]},
                   "size_classes": size_classes,
                   "work_items": bt.items, "single_grid_path_gcells": round(single, 3)},
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 4), "traffic": None,
                     "kernel": "k_pol2d_batch<4,0,false,128> (whole step)",
                     "peak_source": peak_src, "bytes_per_cell_step": 48},
        "gpu_launches": int(launches), "clocks": clocks,
    }
    print(json.dumps(line), flush=True)


def run_adjoint(args):
    """Differentiable 1024^2 FP32 run: 64 Gaussian-envelope sources
    (amplitude parameters theta), loss = field energy in the window
    [448, 576)^2 at the final step, forward + hand-written adjoint with a
    checkpoint every 50 steps.  Reports forward-only and forward+adjoint
    cell-updates/s on the same GPU."""
    import numpy as np
    import torch
    from paper_1907_13088_gb300 import build, synth
    build.build()
    from paper_1907_13088_gb300 import fmx
    from paper_1907_13088_gb300.adjoint import GaussSourceRun, make_function
    shape, N = (1024, 1024), args.steps
    cxy, phases, theta = synth.gauss_sources(64, shape, seed=1907005)
    E0, B0, _ = synth.random_fields(shape, seed=1907006)
    e0 = torch.from_numpy(0.01 * E0[:, 0]).to("cuda", torch.float32)
    b0 = torch.from_numpy(0.01 * B0[:, 0]).to("cuda", torch.float32)
    mask = torch.zeros((3, 1024, 1024), device="cuda")
    mask[:, 448:576, 448:576] = 1.0
    run = GaussSourceRun(shape, cxy, phases, N, width=8.0, omega0=0.2, m=4, passes=3, courant=0.5,
                         precision=fmx.FMX_F32, checkpoint_every=50)
    FieldRun = make_function()
    th = torch.tensor(theta, dtype=torch.float64, requires_grad=True)
    # warm-up: one full forward + adjoint pass (first launches load the kernels)
    EN, BN = FieldRun.apply(th, e0, b0, run, False)
    (0.5 * ((EN * EN * mask).sum() + (BN * BN * mask).sum())).backward()
    th.grad = None
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()  # the grid's stream: fmx.Grid takes the current one
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    l0 = run.launches
    sampler = ClockSampler(0)
    sampler.start()
    time.sleep(0.3)
    tc0 = time.time()
    ev[0].record(stream)
    run.forward(theta, e0, b0)
    ev[1].record(stream)
    torch.cuda.synchronize()
    l1 = run.launches
    ev[2].record(stream)
    EN, BN = FieldRun.apply(th, e0, b0, run, False)
    loss = 0.5 * ((EN * EN * mask).sum() + (BN * BN * mask).sum())
    loss.backward()
    ev[3].record(stream)
    torch.cuda.synchronize()
    tc1 = time.time()
    clocks = sampler.summary(tc0, tc1)
    sampler.stop()
    t_fwd = ev[0].elapsed_time(ev[1]) / 1e3
    t_both = ev[2].elapsed_time(ev[3]) / 1e3
    cells = shape[0] * shape[1]
    peak, peak_src = _peaks()
    # algorithmic bytes per cell of one forward and one adjoint step: forward
    # reads and writes E, B (48 B) and writes then reads the synthesised j_z
    # (8 B); adjoint reads and writes Ebar, Bbar (48 B), writes jbar_z and the
    # projection reads it (8 B)
    bpc = 56 + 56
    achieved = bpc * cells * N / t_both / 1e9
    line = {
        "metric": METRIC, "value": round(cells * N / t_both / 1e9, 4), "unit": UNIT, "n_gpus": 1, "steps": N,
        "warmup": N, "ms_per_step": round(t_both / N * 1e3, 4), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "differentiable 2D 1024x1024 FP32, 64 Gaussian-envelope sources, loss = window "
                               "energy [448,576)^2 at the final step, forward + adjoint, checkpoint every 50",
                   "forward_only_gcells": round(cells * N / t_fwd / 1e9, 4),
                   "forward_plus_adjoint_gcells": round(cells * N / t_both / 1e9, 4),
                   "l2": "fields 1024^2 x 4 B x 15 arrays = 63 MB: inside the 129 MB L2 (the small differentiable "
                         "workload as specified)",
                   "timing": "CUDA events on the grid's stream around whole passes (forward; forward + adjoint "
                             "with the loss and autograd bookkeeping)"},
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 4), "traffic": None, "kernel": "forward + adjoint steps",
                     "peak_source": peak_src, "bytes_per_cell_step": bpc},
        "gpu_launches": int(run.launches - l1 + (l1 - l0)), "clocks": clocks,
    }
    print(json.dumps(line), flush=True)


def run_3d(args):
    """3D periodic 512^3 FP32, six components, power-law spectrum up to
    k_max = N/8, solenoidal current (width 16), m = 4, one binomial pass on
    the current every step, dt = 0.5 dt_CFL.  --n3d picks another cube side
    (for profiler captures on a smaller case; the benchmark line is 512)."""
    import numpy as np
    import torch
    from paper_1907_13088_gb300 import build, synth
    build.build()
    from paper_1907_13088_gb300 import fmx
    n = args.n3d
    t0 = time.perf_counter()
    E, B = synth.power_law_fields((n, n, n), n // 8, 1907003, dtype=np.float32)
    J = synth.solenoidal_current((n, n, n), 1907013, width=16.0, rms=1e-3, dtype=np.float32)
    gen_s = time.perf_counter() - t0
    g = fmx.Grid((n, n, n), precision=fmx.FMX_F32, m=4, filter_passes=1, courant=0.5)
    g.set_fields(E, B)
    g.set_current(J)
    del E, B, J
    g.step(args.warmup)
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    l0 = g.launches
    sampler = ClockSampler(0)
    sampler.start()
    time.sleep(0.3)
    t0 = time.time()
    ev0.record(g.stream)
    g.step(args.steps)
    ev1.record(g.stream)
    torch.cuda.synchronize()
    t1 = time.time()
    ms = ev0.elapsed_time(ev1)
    clocks = sampler.summary(t0, t1)
    sampler.stop()
    launches = g.launches - l0
    # the other setting of sweeps per z-march pass, timed the same way
    spp = g.get_option(fmx.FMX_OPT_SWEEPS_PER_PASS)
    other = 2 if spp == 1 else 1
    g.set_option(fmx.FMX_OPT_SWEEPS_PER_PASS, other)
    g.step(args.warmup)
    torch.cuda.synchronize()
    l1 = g.launches
    ev0.record(g.stream)
    g.step(args.steps)
    ev1.record(g.stream)
    torch.cuda.synchronize()
    ms_other = ev0.elapsed_time(ev1)
    launches_other = g.launches - l1
    g.set_option(fmx.FMX_OPT_SWEEPS_PER_PASS, spp)
    cells = n ** 3
    peak, peak_src = _peaks()
    achieved = BYTES_PER_CELL * cells / (ms / 1e3 / args.steps) / 1e9
    line = {
        "metric": METRIC, "value": round(cells * args.steps / (ms / 1e3) / 1e9, 3), "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"3D periodic {n}^3 FP32, power-law spectrum k_max=N/8, solenoidal J (width 16), "
                               "m=4, 1 binomial pass on J each step, dt=0.5 dt_CFL",
                   "engine": "z-marching kernels", "sweeps_per_pass": spp,
                   "launches_per_step": round(launches / args.steps, 2),
                   "other_sweeps_per_pass": {"sweeps_per_pass": other, "ms_per_step": round(ms_other / args.steps, 4),
                                             "value": round(cells * args.steps / (ms_other / 1e3) / 1e9, 3),
                                             "launches_per_step": round(launches_other / args.steps, 2)},
                   "input_generation_s": round(gen_s, 1)},
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 4), "traffic": None, "kernel": "whole step",
                     "peak_source": peak_src, "bytes_per_cell_step": BYTES_PER_CELL,
                     "alu": alu_roofline(cells, ms / 1e3 / args.steps)},
        "gpu_launches": int(launches), "clocks": clocks,
    }
    print(json.dumps(line), flush=True)


# FP64 arithmetic of one 2D cell-step of the fused FP64 kernel as executed
# (halo and warm-up rows included): (DADD + DMUL + 2 x DFMA) thread
# instructions of one launch over its output cells, from the ncu capture of
# k_fused2d<double, 4, 3> at 2048^2 (profiles/k_fused2d_f64_2048.md):
# (562.4 M + 17.4 M + 2 x 463.8 M) / 2048^2 = 359
FP64_FLOPS_PER_CELL_STEP_2D = 359


def run_f64(args):
    """The 2D benchmark recipe in FP64: 4096^2, power-law spectrum up to
    k_max = N/8, static solenoidal current (width 16) re-filtered by 3
    binomial passes every step, m = 4, dt = 0.5 dt_CFL, on the fused engine
    (one launch per step, all six components).  Two rooflines: HBM (15
    values of 8 bytes per cell-step) and FP64 arithmetic against the FMA rate
    measured in this run (fmx_fma_peak)."""
    import numpy as np
    import torch
    from paper_1907_13088_gb300 import build, synth
    build.build()
    from paper_1907_13088_gb300 import fmx
    n = args.n2d
    E, B = synth.power_law_fields((n, n), n // 8, SEED, dtype=np.float64)
    J = synth.solenoidal_current((n, n), SEED + 1, width=16.0, rms=1e-3, dtype=np.float64)
    g = fmx.Grid((n, n), precision=fmx.FMX_F64, m=M_SWEEPS, filter_passes=PASSES, courant=COURANT,
                 engine=fmx.FMX_ENGINE_FUSED)
    g.set_fields(E, B)
    g.set_current(J)
    del E, B, J
    g.step(args.warmup)
    torch.cuda.synchronize()
    fp64_peak = fmx.fma_peak(fmx.FMX_F64, g.stream)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    l0 = g.launches
    sampler = ClockSampler(0)
    sampler.start()
    time.sleep(0.3)
    t0 = time.time()
    ev0.record(g.stream)
    g.step(args.steps)
    ev1.record(g.stream)
    torch.cuda.synchronize()
    t1 = time.time()
    ms = ev0.elapsed_time(ev1)
    clocks = sampler.summary(t0, t1)
    sampler.stop()
    launches = g.launches - l0
    prof_steps = max(20, min(100, args.steps))
    g.profile(True)
    g.step(prof_steps)
    ks = g.profile_read()
    g.profile(False)
    cells = n * n
    peak, peak_src = _peaks()
    bpc = 15 * 8
    dom = max(ks, key=lambda k: k["total_ms"])
    per_launch_s = dom["total_ms"] / 1e3 / dom["launches"]
    achieved = dom["bytes_per_launch"] / per_launch_s / 1e9
    flops = FP64_FLOPS_PER_CELL_STEP_2D * cells / per_launch_s / 1e12
    line = {
        "metric": METRIC, "value": round(cells * args.steps / (ms / 1e3) / 1e9, 3), "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"2D periodic {n}x{n} FP64, dt=0.5 dt_CFL, power-law spectrum k_max=N/8, static "
                               "solenoidal J (width 16), 3-pass binomial current filter every step, m=4 sweeps",
                   "engine": "fused2d (one kernel per step, k_fused2d<double>)",
                   "l2": f"inputs larger than L2 ({15 * 8 * cells / 1e9:.2f} GB of fields per step vs 129 MB L2)"},
        "roofline": {"bound": "alu", "achieved": round(flops, 3), "peak": round(fp64_peak / 1e12, 3),
                     "unit": "TFLOP/s", "frac": round(flops / (fp64_peak / 1e12), 4), "traffic": None,
                     "kernel": dom["name"], "flops_per_cell_step": FP64_FLOPS_PER_CELL_STEP_2D,
                     "peak_source": "FP64 FMA rate measured in this run (fmx_fma_peak: independent FMA chains on "
                                    "every SM, CUDA events)",
                     "hbm": {"achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                             "frac": round(achieved / peak, 4), "peak_source": peak_src, "bytes_per_cell_step": bpc},
                     "timing": f"CUDA events around each launch, {prof_steps} steps"},
        "gpu_launches": int(launches), "clocks": clocks,
    }
    print(json.dumps(line), flush=True)


def run_res64(args):
    """The 64 x 64 FP64 plane-wave case: 8 TM plane waves (|n| <= 8), no
    current, no filter, the solve to a relative residual of 1e-13 every step
    (Algorithm 1), 200 steps, on the resident engine (all 200 steps and
    their residual stops in one cluster launch); beside it the staged engine
    (one launch per stage, one residual read-back per step) and the staged
    Chebyshev residual mode.  The grid fits in L2: a latency case, reported
    without a roofline."""
    import torch
    from paper_1907_13088_gb300 import build, synth
    build.build()
    from paper_1907_13088_gb300 import fmx
    shape, nsteps = (64, 64), 200
    out = {}
    variants = (("resident", fmx.FMX_ITER_RESIDUAL, fmx.FMX_ENGINE_RESIDENT),
                ("staged", fmx.FMX_ITER_RESIDUAL, fmx.FMX_ENGINE_STAGED),
                ("chebyshev", fmx.FMX_ITER_CHEB_RESIDUAL, fmx.FMX_ENGINE_STAGED))
    for name, mode, engine in variants:
        g = fmx.Grid(shape, with_current=False, precision=fmx.FMX_F64, iter_mode=mode, tol=1e-13, m_max=10000,
                     courant=0.5, engine=engine)
        E, B, _ = synth.tm_plane_waves(shape, g.dt, seed=1907001)
        reps = []
        for rep_ in range(max(args.warmup, 3) + 1):  # warm-up passes, then the timed one
            g.set_fields(E, B)
            s0 = g.diagnostics()["total_sweeps"]
            l0 = g.launches
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            ev0.record(g.stream)
            g.step(nsteps)
            ev1.record(g.stream)
            torch.cuda.synchronize()
            nl = g.launches - l0
            reps.append((ev0.elapsed_time(ev1) * 1e-3, g.diagnostics()["total_sweeps"] - s0, nl))
        if engine == fmx.FMX_ENGINE_RESIDENT:
            clusters = g.get_option(fmx.FMX_OPT_RESIDENT_CLUSTERS)
        out[name] = reps[-1]
        g.close()
    secs, sweeps, launches = out["resident"]
    value = 64 * 64 * nsteps / secs / 1e9
    ctx = {k: {"ms_per_step": round(v[0] / nsteps * 1e3, 4), "sweeps_per_step": round(v[1] / nsteps, 2),
               "launches": int(v[2])} for k, v in out.items()}
    line = {
        "metric": METRIC, "value": round(value, 6), "unit": UNIT, "n_gpus": 1, "steps": nsteps,
        "warmup": max(args.warmup, 3), "ms_per_step": round(secs / nsteps * 1e3, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "2D periodic 64x64 FP64, 8 TM plane waves |n|<=8 (seed 1907001), no current, "
                               "no filter, residual 1e-13 every step (Algorithm 1), 200 steps, dt=0.5 dt_CFL",
                   "engine": f"resident (all steps in one launch of {clusters} thread-block cluster(s))",
                   "sweeps_per_step": round(sweeps / nsteps, 2),
                   "variants": ctx,
                   "timing": "CUDA events on the grid's stream around the 200 steps (the call reads the "
                             "solver status back once at its end)"},
        "roofline": None, "gpu_launches": int(launches),
    }
    print(json.dumps(line), flush=True)


def _oracle_sample_rate(n, nsteps, threads):
    """Runs the FP64 oracle on an n x n periodic sample of the workload;
    returns (cell-updates/s, threads used, seconds)."""
    import numpy as np
    from oracle import core
    from paper_1907_13088_gb300 import synth
    used = core.threads(threads)
    E, B = synth.power_law_fields((n, n), max(1, n // 8), SEED, dtype=np.float64)
    J = synth.solenoidal_current((n, n), SEED + 1, width=16.0, rms=1e-3, dtype=np.float64)
    p = core.Params(shape=(n, n), courant=COURANT, m=M_SWEEPS, filter_passes=PASSES, coef_f32=True)
    t0 = time.perf_counter()
    core.step(p, E, B, J, nsteps)
    dt = time.perf_counter() - t0
    return n * n * nsteps / dt, used, dt


def cpu_baseline(E, B, J):
    """The oracle, as it stands, on the benchmark's own 4096^2 inputs: one
    step to size the run, then enough steps for about 12 s of CPU work."""
    import numpy as np
    from oracle import core
    used = core.threads(os.cpu_count() or 1)
    p = core.Params(shape=(NX, NY), courant=COURANT, m=M_SWEEPS, filter_passes=PASSES, coef_f32=True)
    E64, B64, J64 = (a.astype(np.float64) for a in (E, B, J))
    t0 = time.perf_counter()
    E1, B1, _, _ = core.step(p, E64, B64, J64, 1)
    t1 = time.perf_counter() - t0
    n = int(max(1, min(30, round(12.0 / max(t1, 1e-3)))))
    t0 = time.perf_counter()
    core.step(p, E1, B1, J64, n)
    secs = time.perf_counter() - t0
    rate = NX * NY * n / secs
    # the same oracle on one core, on a 1024^2 periodic sample (two steps)
    core.threads(1)
    try:
        one, _, one_s = _oracle_sample_rate(1024, 2, 1)
    finally:
        core.threads(os.cpu_count() or 1)
    return {"value": round(rate / 1e9, 6), "unit": UNIT, "cores": used, "kind": "oracle",
            "sample": f"the full 4096x4096 workload, {n} steps after one sizing step, FP64 C oracle "
                      f"({secs:.1f} s, OpenMP over rows)",
            "cpu_model": _cpu_model(),
            "one_core": {"value": round(one / 1e9, 6), "unit": UNIT,
                         "sample": f"1024x1024 periodic sample, 2 steps ({one_s:.1f} s)"}}


def _cpu_model():
    """The host CPU as /proc/cpuinfo names it (x86: model name; Arm: the
    implementer and part numbers), with the architecture."""
    import platform
    info = {}
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if ":" in line:
                    k, v = (x.strip() for x in line.split(":", 1))
                    info.setdefault(k, v)
    except OSError:
        pass
    name = info.get("model name") or (
        f"CPU implementer {info['CPU implementer']} part {info['CPU part']}" if "CPU part" in info else "")
    return f"{platform.machine()} {name}".strip()


def run_reference(args):
    rank, world, local = _dist()
    if rank != 0:
        return
    from oracle import core
    core.build()
    threads = os.cpu_count() or 1
    # size the per-step sample so the whole run stays within about two minutes
    n = 256
    rate, used, secs = _oracle_sample_rate(n, 1, threads)
    budget = 120.0 / max(1, args.steps + args.warmup)
    while n > 32 and n * n / rate > budget:
        n //= 2
    _oracle_sample_rate(n, args.warmup, threads) if args.warmup else None
    rate, used, secs = _oracle_sample_rate(n, args.steps, threads)
    value = rate / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(secs / args.steps * 1e3, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample": f"{n}x{n} periodic sample per step"},
        "cpu_baseline": {"value": round(value, 6), "unit": UNIT, "cores": used, "kind": "oracle",
                         "sample": f"{n}x{n} periodic sample of the workload per step, FP64 C oracle"},
        "e2e": {"value": round(value, 6), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def _parser():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--warmup", type=int, default=50)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--workload", choices=("2d4096", "batch256", "adjoint1024", "3d512", "res64", "2d4096f64"),
                    default="2d4096")
    ap.add_argument("--n2d", type=int, default=NX, help="grid side of the 2d4096f64 workload (profiler captures only)")
    ap.add_argument("--n3d", type=int, default=512, help="cube side of the 3d512 workload (profiler captures only)")
    return ap


def main():
    ap = _parser()
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch256":
        run_batch(args)
    elif args.workload == "adjoint1024":
        run_adjoint(args)
    elif args.workload == "3d512":
        run_3d(args)
    elif args.workload == "2d4096f64":
        run_f64(args)
    elif args.workload == "res64":
        run_res64(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
