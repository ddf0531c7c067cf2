"""Benchmark of the device-resident LLG + N-cavity Dormand-Prince integrator.

One benchmark step = one persistent launch of A adaptive Dormand-Prince attempts (6 stage
passes each) over the whole problem.  Two more legs follow the timed region: `adjoint` (the
gradient of a cavity-to-cavity energy transfer on the 64^3 sphere, backward / forward wall time)
and `batch` (a field sweep of independent spheres in one persistent launch, sims/s, against the
same instances one at a time).  `value` is cell-stage updates per second (magnetic cells
x right-hand-side evaluations) summed over ranks, device-timed with CUDA events on the stream
the integrator runs on, L2 flushed between timed steps.  `e2e` times the same work through the
public API from pinned host buffers: set_state (H2D of m, a), the launch, and get_a/get_m (D2H)
every step.  `roofline` relates the algorithmic bytes of one launch to the measured HBM copy
bandwidth; `cpu_baseline` times the FP64 oracle on a bounded sample of the same workload.

--impl reference times the FP64 CPU oracle itself (the only other implementation there is) on
the same workload and metric.  Multi-GPU runs (torchrun) are independent replicas: the
single-problem path has no data exchange between GPUs.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("cell-stage updates/s and % of HBM peak; batched sweep sims/s; "
          "adjoint/forward time ratio")
UNIT = "cell-stage updates/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="cmx", choices=["cmx", "reference"])
    ap.add_argument("--workload", default="afm_film",
                    choices=["multimode_sphere", "afm_film", "full_box", "single_sphere"])
    ap.add_argument("--attempts", type=int, default=0, help="DP attempts per launch (0: auto)")
    ap.add_argument("--box", default="256,256,128", help="full_box grid nx,ny,nz")
    ap.add_argument("--tiling", default="", help="bx,by,bz override")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-sub", action="store_true",
                    help="skip the other single-problem workloads and the 8^3 sphere record")
    ap.add_argument("--adjoint-T", type=float, default=20e-9,
                    help="end time of the adjoint measurement (64^3 sphere, 3 modes)")
    ap.add_argument("--adjoint-every", type=int, default=200)
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--batch-n", type=int, default=512, help="instances of the batched sweep")
    ap.add_argument("--batch-T", type=float, default=30e-9, help="end time of every instance")
    return ap.parse_args()


def make_workload(name, box):
    from paper_2603_03706_b300 import workloads as W
    if name == "multimode_sphere":
        return W.multimode_sphere()
    if name == "afm_film":
        return W.afm_film()
    if name == "single_sphere":
        return W.single_sphere()
    nx, ny, nz = (int(v) for v in box.split(","))
    p = W.multimode_sphere(nx=nx, ny=ny, nz=nz)
    p = p.replace(mask=W.full_mask(nx, ny, nz), name=f"full_box_{nx}x{ny}x{nz}")
    return p.replace(dt_max=W.stable_dt_max(p))


def bytes_per_cell_attempt(p):
    """Algorithmic DRAM bytes per magnetic cell and Dormand-Prince attempt (FP32 SoA, FSAL):
    stage s = 2..6 reads m_n and the slopes with nonzero coupling and writes k_s; stage 7 reads
    m_n, k1, k3..k6 (a_72 = 0) and writes k7 and the new m.  Per sublattice 3 floats per vector:
    36 + 48 + 60 + 72 + 84 + 96 = 396 B; profiles add 4 B per mode and stage when present."""
    per_sub = 12 * (3 + 4 + 5 + 6 + 7 + 8)
    prof = 6 * 4 * p.nmodes if p.u is not None else 0
    return p.nsub * per_sub + prof


# Sources that define the single-problem integrator launch (kernel, engine, stage code, the
# host code that lays out the cells and partitions the blocks).
KERNEL_SOURCES = ("cmx_internal.cuh", "cmx_stage.cuh", "cmx_dense.cuh", "cmx_dense_maps.cu",
                  "cmx_engine.cuh", "cmx_demag.cuh",
                  "cmx_single_kernel.cuh", "cmx_single_t1x4.cu", "cmx_single_t1x8.cu",
                  "cmx_single_t1x16.cu", "cmx_single_t2x4.cu", "cmx_single_t2x8.cu",
                  "cmx_single_t2x16.cu", "cmx_single.cu", "cmx_kernels.h", "cmx_layout.cu",
                  "cmx_layout.h")


def kernel_source_hash():
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2603_03706_b300", "csrc")
    for fn in KERNEL_SOURCES:
        h.update(open(os.path.join(d, fn), "rb").read())
    h.update(open(os.path.join(ROOT, "include", "cmx.h"), "rb").read())
    return h.hexdigest()[:16]


def recorded_traffic(workload, attempts):
    """DRAM bytes per launch from a committed ncu capture, if it was taken on the current kernel
    source (profiles/traffic.json: workload -> {bytes per launch at the bench's attempts, or
    bytes per attempt for workloads whose traffic grows with the attempts, source_hash, ...})."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        rec = json.load(open(path)).get(workload)
    except (OSError, ValueError):
        return None
    if not rec or rec.get("source_hash") != kernel_source_hash():
        return None
    if rec.get("bytes_per_launch_at_bench_attempts") is not None:
        return rec["bytes_per_launch_at_bench_attempts"]
    if rec.get("bytes_per_attempt") is not None:
        return rec["bytes_per_attempt"] * attempts
    return None


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            f = [v.strip() for v in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        load = [v for v in sm if mx and v > 0.3 * mx] or sm
        return {"sm_mhz": statistics.median(load), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup(n):
    import torch
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    elif torch.cuda.is_available():
        torch.cuda.set_device(0)
    return rank, world, local


def barrier_and_max(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda")
    dist.barrier()
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def cpu_baseline(p, seconds):
    """FP64 oracle, adaptive, on all host cores, on a bounded number of attempts of the same
    workload; cell-stage updates per second."""
    from oracle import oracle as O
    cores = os.cpu_count() or 1
    os.environ.setdefault("OMP_NUM_THREADS", str(cores))
    op = O.OracleProblem(p)
    it = O.Integrator(op)
    it.run(p.T, max_attempts=1)               # first attempt incl. the initial slope
    t0 = time.perf_counter()
    it.run(p.T, max_attempts=3)               # attempt rate of the steady state
    per = max((time.perf_counter() - t0) / 3, 1e-4)
    n = max(1, int(seconds / per))
    s0 = it.state()
    t0 = time.perf_counter()
    it.run(p.T, max_attempts=n)
    dt = time.perf_counter() - t0
    s1 = it.state()
    rhs = 6 * (s1["attempts"] - s0["attempts"])
    return {"value": rhs * p.ncells / dt, "unit": UNIT, "cores": int(os.environ["OMP_NUM_THREADS"]),
            "kind": "oracle",
            "sample": f"{p.name}: {s1['attempts'] - s0['attempts']} adaptive FP64 attempts "
                      f"({rhs} RHS evaluations x {p.ncells} cells) in {dt:.1f} s"}


def adjoint_ratio(T, every, stream):
    """Adjoint form on the 64^3 sphere with three profiled modes: wall time of the forward run
    (adaptive, to T) and of the gradient of the cavity 1 -> 3 energy transfer with respect to
    g~_n, kappa_n, omega_n, alpha, u_n(r), a_0 and m_0 (recompute + reverse sweep), each
    bracketed by device synchronisation."""
    import numpy as np
    import torch
    from paper_2603_03706_b300 import cmx
    from paper_2603_03706_b300 import workloads as W
    p = W.adjoint_sphere(T=T)
    sim = cmx.Simulation.from_problem(p, stream=stream, log_cap=400000)
    # warm-up: a short recorded run and its gradient (allocations, module load)
    sim.adjoint_record(every, 400000)
    sim.run(20 * p.dt_max)
    sim.adjoint(None, None, want_u=False, want_m0=False)
    # plain forward
    sim.set_state(p.m0, p.a0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st_plain = sim.run(p.T)
    torch.cuda.synchronize()
    t_plain = time.perf_counter() - t0
    # recorded forward + backward
    sim.set_state(p.m0, p.a0)
    sim.adjoint_record(every, 400000)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st = sim.run(p.T)
    torch.cuda.synchronize()
    t_fwd = time.perf_counter() - t0
    log = sim.get_log(cap=st["attempts"])
    acc = log["accepted"]
    n = int(acc.sum())
    aT = log["a"][acc][-1]
    e0 = abs(p.a0[0]) ** 2
    la = np.zeros((n + 1, 2 * p.nmodes))
    la[-1, 4:6] = 2 * np.array([aT[2].real, aT[2].imag]) / e0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    g = sim.adjoint(la, None)
    torch.cuda.synchronize()
    t_bwd = time.perf_counter() - t0
    sim.close()
    return {"ratio": t_bwd / t_plain, "unit": "backward s / forward s",
            "forward_s": t_plain, "forward_recorded_s": t_fwd, "backward_s": t_bwd,
            "total_over_forward": (t_fwd + t_bwd) / t_plain,
            "workload": p.name, "T": p.T, "accepted_steps": n, "attempts": st_plain["attempts"],
            "checkpoint_every": every, "cells": p.ncells, "modes": p.nmodes,
            "loss": "energy transfer |a_3(T)|^2/|a_1(0)|^2",
            "energy_transfer": float(abs(aT[2]) ** 2 / e0),
            "dL_dg_re": [float(v) for v in g["g_re"]], "timing": "wall clock, synchronised"}


def batch_sweep(n_inst, T, stream):
    """Field sweep across the anticrossing: n_inst independent spheres of 24^3 .. 96^3 cells
    with 1-3 modes each, all integrated to T in one persistent launch sequence (CUDA graph), and
    the same instances one after the other through the single-problem path.  Wall time,
    synchronised; instance creation (layout, uploads) is outside both timed regions."""
    import torch
    from paper_2603_03706_b300 import cmx
    from paper_2603_03706_b300 import workloads as W
    probs = W.batch_sweep(n_inst=n_inst, T=T)
    cells = sum(p.ncells for p in probs)
    # launch shape from the batch autotuner (trial batches of every k-th instance)
    tuned = cmx.batch_autotune(probs, sample=64, attempts=20, stream=stream)
    shape = dict(bx=tuned["bx"], by=tuned["by"], team=tuned["team"])
    # warm-up of both paths on a few instances
    b = cmx.BatchSimulation(probs[:8], stream=stream, **shape)
    b.run()
    b.close()
    b = cmx.BatchSimulation(probs, stream=stream, **shape)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st = b.run()
    torch.cuda.synchronize()
    t_batch = time.perf_counter() - t0
    info = b.info()
    b.close()
    sims = [cmx.Simulation.from_problem(p, stream=stream) for p in probs]
    sims[0].run(T)
    sims[0].set_state(probs[0].m0, probs[0].a0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    seq_updates = 0
    for s in sims:
        seq_updates += s.run(T)["cell_stage_updates"]
    torch.cuda.synchronize()
    t_seq = time.perf_counter() - t0
    for s in sims:
        s.close()
    # algorithmic bytes of the batched run: the single-problem bytes model per magnetic cell and
    # attempt (uniform profiles), times the cell-attempts it performed
    peaks = measured_peaks()
    peak_gbs = peaks.get("hbm_gbs", 6400.0)
    achieved = bytes_per_cell_attempt(probs[0]) * st["cell_stage_updates"] / 6.0 / t_batch / 1e9
    return {"value": n_inst / t_batch, "unit": "sims/s", "sequential": n_inst / t_seq,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak_gbs, "unit": "GB/s",
                         "frac": achieved / peak_gbs, "traffic": None,
                         "bytes_per_cell_attempt": bytes_per_cell_attempt(probs[0]),
                         "timing": "wall clock of the whole batched run"},
            "speedup_vs_sequential": t_seq / t_batch, "instances": n_inst, "T": T,
            "cells_total": cells, "batch_s": t_batch, "sequential_s": t_seq,
            "cell_stage_updates_per_s": st["cell_stage_updates"] / t_batch,
            "sequential_cell_stage_updates_per_s": seq_updates / t_seq,
            "teams": info["teams"], "team_size": info["team_size"], "blocks": info["blocks"],
            "graph": bool(info["graph"]), "window": [shape["bx"], shape["by"]],
            "autotune_us": tuned["us"], "workload": "batch_sweep (spheres 24^3..96^3, 1-3 modes)",
            "timing": "wall clock, synchronised"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    p = make_workload(args.workload, args.box)
    from oracle import oracle as O
    cores = os.cpu_count() or 1
    os.environ.setdefault("OMP_NUM_THREADS", str(cores))
    op = O.OracleProblem(p)
    it = O.Integrator(op)
    t0 = time.perf_counter()
    it.run(p.T, max_attempts=1)
    per = max(time.perf_counter() - t0, 1e-4)
    budget = 150.0 / max(args.steps + args.warmup, 1)
    att = max(1, int(budget / per))
    for _ in range(args.warmup):
        it.run(p.T, max_attempts=att)
    t0 = time.perf_counter()
    s0 = it.state()
    for _ in range(args.steps):
        it.run(p.T, max_attempts=att)
    dt = time.perf_counter() - t0
    s1 = it.state()
    rhs = 6 * (s1["attempts"] - s0["attempts"])
    v = rhs * p.ncells / dt
    line = {"metric": METRIC, "value": v, "unit": UNIT, "impl": "reference", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": p.name, "cells": p.ncells,
                                            "attempts_per_step": att},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": int(os.environ["OMP_NUM_THREADS"]),
                             "kind": "oracle",
                             "sample": f"{args.steps} steps x {att} adaptive FP64 attempts"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def time_workload(p, stream, steps, warmup, attempts=0, tiling=None, clocks_for=None):
    """Device-timed launches of one workload: autotuned window (unless given), A attempts per
    launch (about 20 ms of work at the HBM roofline, 8..2000), L2 flushed before every timed
    launch, CUDA events on the integrator's stream.  Returns the record and the open handle."""
    import torch
    from paper_2603_03706_b300 import cmx
    sim = cmx.Simulation.from_problem(p, stream=stream, tiling=tiling)
    tuned = None
    if tiling is None:
        tuned = sim.autotune(20)        # measured window choice, state restored afterwards
        torch.cuda.synchronize()
    ncell = sim.ncells()[0]
    bpa = bytes_per_cell_attempt(p) * ncell
    peaks = measured_peaks()
    peak_gbs = peaks.get("hbm_gbs", 6400.0)
    A = attempts or max(8, min(2000, int(0.02 * peak_gbs * 1e9 / bpa)))
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")   # 256 MiB > L2
    with torch.cuda.stream(stream):
        for _ in range(warmup):
            flush.zero_()
            sim.launch(1.0, A)           # T = 1 s is never reached within a launch
        st0 = sim.sync()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(steps)]
        torch.cuda.synchronize()
        if clocks_for is not None:
            clocks_for()
        with ClockSampler(int(os.environ.get("LOCAL_RANK", "0"))) as clk:
            for i in range(steps):
                flush.zero_()
                evs[i][0].record(stream)
                sim.launch(1.0, A)
                evs[i][1].record(stream)
            torch.cuda.synchronize()
        st1 = sim.sync()
    del flush
    times = [a.elapsed_time(b) * 1e-3 for a, b in evs]
    t_total = sum(times)
    updates = st1["cell_stage_updates"] - st0["cell_stage_updates"]
    attempts_done = st1["attempts"] - st0["attempts"]
    achieved = bpa * (attempts_done / steps) / (t_total / steps) / 1e9
    rec = {
        "workload": p.name, "value": updates / t_total, "unit": UNIT,
        "ms_per_step": 1e3 * t_total / steps, "steps": steps, "warmup": warmup,
        "us_per_attempt": 1e6 * t_total / max(attempts_done, 1),
        "cells": ncell, "grid": [p.nx, p.ny, p.nz], "nsub": p.nsub, "modes": p.nmodes,
        "attempts_per_step": A, "rhs_evals_per_step": updates / ncell / steps,
        "dt_max": p.dt_max, "l2": "flushed between timed steps (256 MiB write)",
        "tiling": sim.get_tiling(), "autotune_us_per_attempt": tuned and tuned["us_per_attempt"],
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak_gbs, "unit": "GB/s",
                     "frac": achieved / peak_gbs,
                     "traffic": recorded_traffic(p.name, A),
                     "bytes_per_cell_attempt": bytes_per_cell_attempt(p),
                     "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)" if peaks else
                     "fallback 6400 GB/s"},
        "clocks": clk.summary(),
    }
    return rec, sim, t_total, updates


def single_sphere_record(stream):
    """Latency-bound 8^3 sphere (280 cells, one mode): device time per attempt of one long
    launch, and the wall time of the whole 20 ns integration through cmx_run."""
    import torch
    from paper_2603_03706_b300 import cmx
    from paper_2603_03706_b300 import workloads as W
    p = W.single_sphere(T=20e-9)
    sim = cmx.Simulation.from_problem(p, stream=stream)
    sim.run(0.2e-9)                                   # warm-up
    sim.set_state(p.m0, p.a0)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sim.launch(1.0, 2000)
    e1.record(stream)
    torch.cuda.synchronize()
    us = e0.elapsed_time(e1) * 1e3 / 2000
    sim.set_state(p.m0, p.a0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st = sim.run(p.T)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    tl = sim.get_tiling()
    sim.close()
    return {"workload": p.name, "cells": p.ncells, "us_per_attempt": us,
            "cell_stage_updates_per_s": 6 * p.ncells / (us * 1e-6),
            "T": p.T, "wall_s_to_T": wall, "attempts_to_T": st["attempts"],
            "accepted_to_T": st["accepted"], "launches_to_T": st["launches"], "tiling": tl,
            "timing": "us_per_attempt: CUDA events over one 2000-attempt launch; wall_s_to_T: "
                      "cmx_run from t = 0 to T, synchronised"}


def demag_record(stream):
    """Full magnetostatic demag (FFT convolution with the Newell tensor) against the diagonal
    factors on a 64 x 64 x 8 film (non-ellipsoidal: the diagonal factors are only approximate):
    device time per attempt both ways on the 32 x 8 tiles, the demag passes' share, and the bytes
    the five FFT passes move per stage (complex FP32 work array of nz planes of Ly x Lx, three
    components, read and written once per pass; the tensor spectrum read once)."""
    import torch
    from paper_2603_03706_b300 import cmx
    from paper_2603_03706_b300 import workloads as W
    nx, ny, nz = 64, 64, 8
    p = W.make_problem(nx, ny, nz, 3e-9, W.full_mask(nx, ny, nz), Ms=1.4e5, B0=(0.0, 0.0, 0.3),
                       Nd=(0.0, 0.0, 1.0), omega=[2 * 3.141592653589793 * 5e9],
                       kappa=[2 * 3.141592653589793 * 2e6], g_re=[2 * 3.141592653589793 * 50e6],
                       g_im=[0.0], m0=W.tilted_state(1, nx, ny, nz, 2.0, 0.0), T=1.0)
    p = p.replace(dt_max=W.stable_dt_max(p))
    out = {"workload": "film_64x64x8 (full mask, 3 nm cells)", "cells": p.ncells}
    for full in (False, True):
        sim = cmx.Simulation.from_problem(p, stream=stream, tiling=(32, 8, 4))
        sim.set_demag(full)
        sim.run(1.0, max_attempts=5)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sim.launch(1.0, 200)
        e1.record(stream)
        torch.cuda.synchronize()
        st = sim.sync()
        sim.close()
        out["us_per_attempt_" + ("full" if full else "diagonal")] = e0.elapsed_time(e1) * 1e3 / 200
    Lx, Ly, Lz = 128, 128, 16
    c8 = 3 * 8                                   # three complex FP32 components
    half, full = nz * ny * Lx * c8, nz * Ly * Lx * c8
    out["fft_grid"] = [Lx, Ly, Lz]
    # pass 1: stage values in, x lines out; 2: x lines in, y lines out; 3: y lines in and out
    # plus the six real tensor spectra; 4: y lines in, x lines out; 5: x lines in, field out
    out["demag_bytes_per_stage"] = ((p.ncells * 12 + half) + (half + full) +
                                    (2 * full + 6 * Lx * Ly * Lz * 4) + (full + half) +
                                    (half + p.ncells * 12))
    out["demag_share"] = 1.0 - out["us_per_attempt_diagonal"] / out["us_per_attempt_full"]
    out["timing"] = "CUDA events over one 200-attempt launch each, same tiles"
    return out


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import numpy as np
    import torch

    rank, world, local = dist_setup(args.gpus)
    p = make_workload(args.workload, args.box)
    stream = torch.cuda.Stream()
    tiling = tuple(int(v) for v in args.tiling.split(",")) if args.tiling else None

    def sync_ranks():
        if world > 1:
            torch.distributed.barrier()

    rec, sim, t_total, updates = time_workload(p, stream, args.steps, args.warmup,
                                               args.attempts, tiling, clocks_for=sync_ranks)
    A = rec["attempts_per_step"]
    t_total_max = barrier_and_max(t_total, world)
    value = updates * world / t_total_max

    # end to end through the public API: pinned host buffers in and out every step
    e2e = None
    if not args.no_e2e:
        m_host = torch.from_numpy(np.asarray(p.m0, np.float32).copy()).pin_memory()
        m_out = torch.empty_like(m_host).pin_memory()
        a0 = np.asarray(p.a0)
        for _ in range(2):
            sim.set_state(m_host, a0)
            sim.launch(1.0, A)
            sim.get_a()
            sim.get_m(out=m_out)
        torch.cuda.synchronize()
        sync_ranks()
        u0 = 0
        t0 = time.perf_counter()
        for _ in range(args.steps):
            sim.set_state(m_host, a0)
            sim.launch(1.0, A)
            st = sim.sync()
            u0 += st["cell_stage_updates"]
            sim.get_a()
            sim.get_m(out=m_out)
        torch.cuda.synchronize()
        te = barrier_and_max(time.perf_counter() - t0, world)
        h2d = m_host.numel() * 4 + 16 * p.nmodes
        d2h = m_out.numel() * 4 + 16 * p.nmodes
        e2e = {"value": u0 * world / te, "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h}
    sim.close()

    line = None
    if rank == 0:
        config = {k: rec[k] for k in ("workload", "cells", "grid", "nsub", "modes",
                                      "attempts_per_step", "rhs_evals_per_step", "dt_max", "l2",
                                      "tiling", "autotune_us_per_attempt")}
        config["parallelism"] = "replicas" if world > 1 else "single"
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_total_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": config, "roofline": rec["roofline"],
            "clocks": rec["clocks"], "gpu_launches": 2 * args.steps, "e2e": e2e,
        }
        def leg(fn, *a):
            # a sub-record that fails reports its error instead of taking the headline line
            # with it
            from paper_2603_03706_b300 import cmx
            try:
                return fn(*a)
            except (cmx.CmxError, RuntimeError, ValueError) as e:
                return {"error": f"{type(e).__name__}: {e}"}

        def sub_workloads():
            # the other single-problem workloads, each with its own roofline record
            subs = []
            for name in ("multimode_sphere", "full_box"):
                if name == args.workload:
                    continue
                q = make_workload(name, "256,256,128")
                r, s2, _, _ = time_workload(q, stream, 5, 3)
                s2.close()
                subs.append(r)
            return subs

        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(p, args.cpu_seconds)
        if not args.no_sub:
            line["workloads"] = leg(sub_workloads)
            line["single_sphere"] = leg(single_sphere_record, stream)
            line["demag"] = leg(demag_record, stream)
        if not args.no_adjoint:
            line["adjoint"] = leg(adjoint_ratio, args.adjoint_T, args.adjoint_every, stream)
        if not args.no_batch:
            line["batch"] = leg(batch_sweep, args.batch_n, args.batch_T, stream)
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
