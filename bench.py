"""Benchmark of the Godunov hydro step on GB300.

Default workload: 3D periodic turbulence box 256^3 (rho = 1, p = 0.6,
random-phase Gaussian velocity field with a k^-4 shell spectrum, rms Mach 1),
mixed precision (FP32 reconstruction/HLLC, FP64 state), CFL 0.3.  One
benchmark step = one Heun step of the whole grid = ncell cell-updates.
The same grid is also timed on the all-FP64 path, the all-FP32 path and
with the memory-optimized van Leer integrator (mixed).

Prints ONE JSON line.  ``--impl reference`` times the CPU oracle instead (the
reference arm: a plain FP64 C program on the host cores).

Multi-GPU: the path does not shard here (replicas only): each rank runs the
same workload on its own GPU, the barrier and max-over-ranks timing are the
only collectives, and ``value`` adds the ranks' cell-updates.
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

METRIC = "cell-updates/s (mixed vs FP64, 1 GB300, % HBM roofline); p99 solve latency"
UNIT = "cell-updates/s"
BYTES_PER_CELL_UPDATE_3D = 200  # stage 1: read Un, write U1; stage 2: read U1 and Un, write Un+1 (5 x 8 B each)
# all-FP32 Heun: the same five array passes of 5 x 4 B
BYTES_PER_CELL_UPDATE_3D_FP32 = 100
# van Leer, mixed: predictor reads Un (40 B), writes W (5 x 4 B); corrector
# reads W and Un, writes Un+1
BYTES_PER_CELL_UPDATE_3D_VL2 = 160


# the translation unit of the mixed stage kernels and every file it includes
STAGE_SOURCES = ("khy_mixed.cu", "khy_launch.cuh", "khy_internal.h", "khy_stage.cuh", "khy_kernels.cuh",
                 "khy_mixed_kernels.cuh", "khy_packed.cuh", "khy_single_kernels.cuh")


def stage_sources_sha256(sources=STAGE_SOURCES) -> str:
    import hashlib
    h = hashlib.sha256()
    for name in sources:
        with open(os.path.join(ROOT, "paper_2501_02317_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def _recorded_traffic(workload: str):
    """DRAM bytes (read + write) of the stage-kernel pair from the committed
    ncu capture, or None when the stage kernels' sources changed since it was
    taken."""
    try:
        with open(os.path.join(ROOT, "profiles", "stage_traffic.json")) as f:
            rec = json.load(f)
        if rec.get("stage_sources_sha256") != stage_sources_sha256() or rec.get("workload") != workload:
            return None
        return float(rec["stage1_dram_bytes"]) + float(rec["stage2_dram_bytes"])
    except Exception:
        return None


# independent simulations stepped at once in the end-to-end leg: the host
# link copies in both directions at once (host->device and device->host of
# different problems), so three pipelines keep both directions busy
E2E_PIPELINES = 3

# GB300 HBM3e nominal bandwidth (GB/s), the second denominator of the roofline
NOMINAL_HBM_GBS = 7900.0


def _recorded_warp_inst(workload: str):
    """Warp instructions the stage-kernel pair executes per step, from the
    committed ncu capture, or None when the sources changed since."""
    try:
        with open(os.path.join(ROOT, "profiles", "stage_traffic.json")) as f:
            rec = json.load(f)
        if rec.get("stage_sources_sha256") != stage_sources_sha256() or rec.get("workload") != workload:
            return None
        return float(rec["stage1_warp_inst"]) + float(rec["stage2_warp_inst"])
    except Exception:
        return None


def issue_roofline(stage_ms: float, ncell: int, workload: str, sms: int, sm_mhz: float):
    """The resource that bounds the mixed stage pair: instruction issue.
    Executed warp instructions of the pair (ncu count) over its event-timed
    duration, against one warp instruction per clock per SM sub-partition
    (4 per SM) at the maximum SM clock.  Executed, not algorithmic,
    instructions: this shows how close the kernel runs to its issue limit."""
    inst = _recorded_warp_inst(workload)
    peak = 4.0 * sms * sm_mhz * 1e6
    if inst is None:
        return {"bound": "issue", "achieved": None, "peak": peak, "unit": "warp-inst/s", "frac": None}
    ach = inst / (stage_ms * 1e-3)
    return {"bound": "issue", "achieved": ach, "peak": peak, "unit": "warp-inst/s", "frac": ach / peak,
            "thread_inst_per_cell_update": inst * 32.0 / ncell,
            "note": "executed instructions (ncu count of the committed capture), 4 warp-instructions per clock per SM"}


def _sm_max_mhz() -> float:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["sm_max_mhz"])
    except Exception:
        return 2070.0


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def host_cpu() -> dict:
    """Host CPU model and logical CPU count (lscpu / nproc)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    return {"model": model, "nproc": os.cpu_count()}


# the translation unit of the all-FP64 stage kernels and every file it includes
FP64_SOURCES = ("khy_fp64.cu", "khy_launch.cuh", "khy_internal.h", "khy_stage.cuh", "khy_kernels.cuh",
                "khy_mixed_kernels.cuh", "khy_packed.cuh", "khy_single_kernels.cuh")
# FP64 instructions a GB300 SM retires per clock (DFMA, DADD, DMUL: two
# lanes per clock per SM, the rate behind the part's nominal 1.25 TFLOP/s
# of FP64 FMA at 152 SMs and 2.07 GHz)
FP64_PER_CLK_PER_SM = 2


def fp64_ops_per_cell_update(workload: str):
    """Thread-level FP64 instructions (DFMA + DADD + DMUL) per cell-update of
    the all-FP64 stage pair, from the committed ncu count, or None when the
    FP64 kernels' sources changed since it was taken."""
    try:
        with open(os.path.join(ROOT, "profiles", "fp64_stage_ops.json")) as f:
            rec = json.load(f)
        if rec.get("sources_sha256") != stage_sources_sha256(FP64_SOURCES) or rec.get("workload") != workload:
            return None
        return float(rec["fp64_inst_per_cell_update"])
    except Exception:
        return None


def fp64_roofline(stage_ms: float, ncell: int, workload: str, sms: int, sm_mhz: float):
    """Bound of the all-FP64 leg: counted FP64 instructions per cell-update x
    cells over the stage pair's event-timed duration, against the FP64 pipe's
    peak (FP64_PER_CLK_PER_SM x SMs x the maximum SM clock)."""
    ops = fp64_ops_per_cell_update(workload)
    peak = FP64_PER_CLK_PER_SM * sms * sm_mhz * 1e6
    if ops is None:
        return {"bound": "fp64", "achieved": None, "peak": peak / 1e12, "unit": "T FP64 inst/s", "frac": None,
                "ops_per_cell_update": None, "note": "no FP64 instruction count recorded for these sources"}
    ach = ops * ncell / (stage_ms * 1e-3)
    return {"bound": "fp64", "achieved": ach / 1e12, "peak": peak / 1e12, "unit": "T FP64 inst/s",
            "frac": ach / peak, "ops_per_cell_update": ops, "peak_kind": "nominal (2 per clock per SM)"}


class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.QUERY, "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        except Exception:
            pass
        finally:
            try:
                os.unlink(self.path)
            except Exception:
                pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows),
                "power_w_max": max(float(r[3]) for r in rows if r[3].replace(".", "").isdigit())
                if any(r[3].replace(".", "").isdigit() for r in rows) else None}


def cpu_oracle_rate(steps: int = 10, n: int = 256, threads: int = 0):
    """Oracle cell-updates/s over `steps` Heun steps of the n^3 turbulence
    box (the headline workload) with `threads` host threads (0: all cores).
    Returns (rate, threads used, sample description, final state, mesh, W)."""
    import oracle
    from paper_2501_02317_gb300 import workloads as wl
    cores = threads or os.cpu_count() or 1
    used = oracle.set_threads(cores)
    mesh, W = wl.turbulence(n, prec=wl.PREC_FP64)
    U = oracle.prim_to_cons(mesh, W)
    t = 0.0
    t0 = time.perf_counter()
    for _ in range(steps):
        U, t, _, _ = oracle.heun_step(mesh, U, t, 1e30)
    el = time.perf_counter() - t0
    sample = "%d Heun step%s of the %d^3 turbulence box (the headline workload, seed 2)" % (
        steps, "" if steps == 1 else "s", n)
    return mesh.ncell * steps / el, used, sample, U, mesh, W


def parity_against_oracle(khydro, wl, mesh0, W, Uo, steps: int):
    """Per-field relative L1 (sum |q - q_ref| / sum |q_ref|, conserved fields
    and the pressure) of the mixed and all-FP64 paths after `steps` Heun steps
    of the headline workload against the oracle's state after the same steps
    (the state the CPU-baseline leg computed)."""
    out = {}
    for name, prec in (("mixed", wl.PREC_MIXED), ("fp64", wl.PREC_FP64)):
        mesh = mesh0.replace(prec=prec)
        with khydro.Sim(mesh) as sim:
            sim.set_primitive(W)
            sim.step_to(1e30, steps)
            U = sim.conserved()
        errs = {}
        names = ["rho"] + ["m_%s" % "xyz"[d] for d in range(mesh.ndim)] + ["E"]
        for q, nm in enumerate(names):
            errs[nm] = float(np.abs(U[q] - Uo[q]).sum() / np.abs(Uo[q]).sum())

        def pres(V):
            ke = 0.5 * sum(V[1 + d] ** 2 for d in range(mesh.ndim)) / V[0]
            return (mesh.gamma - 1.0) * (V[mesh.nvar - 1] - ke)
        po = pres(Uo)
        errs["p"] = float(np.abs(pres(U) - po).sum() / np.abs(po).sum())
        errs["bitwise"] = bool(np.array_equal(U, Uo))
        out[name] = errs
    out["steps"] = steps
    out["gates"] = {"fp64": "1e-12 every field", "mixed": "rho 1e-5, p 1e-4"}
    return out


# 2D Heun cell-update: stage 1 reads Un, writes U1; stage 2 reads U1 and Un,
# writes Un+1 (four fields of 8 B each)
BYTES_PER_CELL_UPDATE_2D = 160


def bench_batch(khydro, wl, torch, steps: int = 200, peak_gbs: float = None):
    """Batched workload: 4096 independent 2D blast grids (sides log-uniform in
    [32, 256], seed 3), mixed precision, one launch per stage for all grids,
    tile variant picked by the autotuner; `steps` Heun steps of every grid.
    The HBM fraction divides the algorithmic bytes by the whole step (clock
    launch included), a lower bound on the stage kernels' own fraction."""
    grids = wl.batch_blasts(4096)
    meshes = [m for m, _ in grids]
    cells = sum(m.ncell for m in meshes)
    stream = torch.cuda.Stream()
    with khydro.Batch(meshes, stream=stream.cuda_stream) as b:
        b.set_primitive([W for _, W in grids])
        variant, tune_ms = b.autotune(2)
        _, ctas_per_slot = b.schedule()
        b.set_target(1e30, steps)
        b.enqueue_steps(3)
        torch.cuda.synchronize()
        b.set_target(1e30, steps)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        b.enqueue_steps(steps)
        e1.record(stream)
        e1.synchronize()
        el = e0.elapsed_time(e1) / 1e3
        info = b.info()
        done = all(b.clock(k)[1] == steps + 3 for k in (0, len(meshes) // 2, len(meshes) - 1))
    return {"workload": "4096 2D blast grids, sides log-U[32,256] (seed 3), mixed, periodic", "grids": len(meshes),
            "cells": cells, "steps": steps, "value": cells * steps / el, "unit": UNIT, "ms_per_step": 1e3 * el / steps,
            "variant": variant, "ctas_per_slot": ctas_per_slot, "ctas": info["nblocks"], "launches_per_step": 3, "all_grids_stepped": done,
            "bytes_per_cell_update": BYTES_PER_CELL_UPDATE_2D,
            "hbm_achieved_gbs": BYTES_PER_CELL_UPDATE_2D * cells * steps / el / 1e9,
            "hbm_frac": (BYTES_PER_CELL_UPDATE_2D * cells * steps / el / 1e9 / peak_gbs) if peak_gbs else None}


def serving_prefix(jobs, avail_bytes):
    """How many jobs of the stream to serve: all of them when their FP64
    initial states take at most half of `avail_bytes` of free host memory
    (None: unknown, serve all), else the longest prefix that does.  Returns
    (count, note or None)."""
    ic_bytes = [(j.ndim + 2) * j.side ** j.ndim * 8 for j in jobs]
    if avail_bytes is None or 2 * sum(ic_bytes) <= avail_bytes:
        return len(jobs), None
    keep, acc = 0, 0
    while keep < len(jobs) and 2 * (acc + ic_bytes[keep]) <= avail_bytes:
        acc += ic_bytes[keep]
        keep += 1
    return keep, "first %d of %d jobs: their initial states fill half the %.0f GB of free host memory" % (
        keep, len(jobs), avail_bytes / 1e9)


def bench_serving(khydro, wl, njobs: int = 2000, budget_bytes: int = 16 << 30, slots: int = 64):
    """Serving: the first `njobs` jobs of the seeded Poisson stream (mean 200
    jobs/s; 2D 64^2-512^2 and 3D 32^3-128^3, KH / blast / turbulence, t_end
    U[0.05, 0.5]) submitted at their arrival times; then the same jobs as
    Poisson streams at 50% and 90% of the capacity measured in the first run
    (the stream's exponential inter-arrival times rescaled to the lower rate).
    Time-to-solution = finish - submit."""
    jobs = wl.serving_stream(njobs, seed=4)
    # the initial states are generated before the clock starts (submissions
    # keep to the arrival times): keep them within half the host memory
    # available, else serve the longest prefix of the stream that fits
    try:
        avail = os.sysconf("SC_AVPHYS_PAGES") * os.sysconf("SC_PAGE_SIZE")
    except (ValueError, OSError):
        avail = None
    keep, note = serving_prefix(jobs, avail)
    jobs = jobs[:keep]
    ics = [wl.job_initial_state(j) for j in jobs]

    def run(arrivals, offered):
        with khydro.Server(budget_bytes, slots) as srv:
            t0 = time.perf_counter()
            ids = []
            for (m, W), j, at in zip(ics, jobs, arrivals):
                delay = at - (time.perf_counter() - t0)
                if delay > 0:
                    time.sleep(delay)
                ids.append(srv.submit(m, W, j.t_end))
            for i in ids:
                srv.wait(i, 1800.0)
            lat = []
            for i in ids:
                _, (ts, ta, td), _ = srv.poll(i)
                lat.append(td - ts)
            st = srv.stats()
        makespan = st["elapsed_s"]
        return {"arrivals": "poisson", "offered_jobs_per_s": offered, "achieved_jobs_per_s": len(ids) / makespan,
                "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
                "value": st["cell_updates"] / makespan, "jobs": len(ids), "makespan_s": makespan,
                "cell_updates": st["cell_updates"]}

    base = [j.arrival for j in jobs]
    rate0 = 200.0
    sat = run(base, rate0)
    cap = sat["achieved_jobs_per_s"]  # jobs/s the server sustained while saturated
    out = {"workload": "Poisson 200 jobs/s (seed 4), first %d jobs, mixed, HBM budget %d GiB, %d slots"
                       % (len(jobs), budget_bytes >> 30, slots),
           "offered_200_per_s": sat, "capacity_jobs_per_s": cap}
    if note:
        out["note"] = note
    for frac in (0.5, 0.9):
        rate = frac * cap
        arr = [a * rate0 / rate for a in base]  # the same exponential gaps, mean 1/rate
        out["load_%d%%" % int(frac * 100)] = run(arr, rate)
    out["unit"] = UNIT
    return out


class Ranks:
    """Collectives of the replica harness (one process per GPU, each stepping
    its own copy of the workload): a barrier, and the maximum of a host value
    over ranks -- the timed region ends when the slowest rank ends.  `dist`
    is torch.distributed after init_process_group (NCCL on GPUs, gloo in the
    CPU tests) or None for one process."""

    def __init__(self, dist=None, device: str = "cpu"):
        self.dist = dist
        self.device = device
        self.world = dist.get_world_size() if dist is not None else 1
        self.rank = dist.get_rank() if dist is not None else 0

    def barrier(self) -> None:
        if self.dist is not None:
            self.dist.barrier()

    def max(self, x: float) -> float:
        if self.dist is None:
            return x
        import torch
        t = torch.tensor([x], dtype=torch.float64, device=self.device)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return float(t.item())


def whole_job_rate(world: int, units_per_rank: float, seconds: float) -> float:
    """Units all ranks processed per second of the slowest rank (weak scaling)."""
    return world * units_per_rank / seconds


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    from paper_2501_02317_gb300 import workloads as wl
    cores = os.cpu_count() or 1
    used = oracle.set_threads(cores)
    n = args.n
    mesh, W = wl.turbulence(n, prec=wl.PREC_FP64)
    U = oracle.prim_to_cons(mesh, W)
    t = 0.0
    for _ in range(args.warmup):
        U, t, _, _ = oracle.heun_step(mesh, U, t, 1e30)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        U, t, _, _ = oracle.heun_step(mesh, U, t, 1e30)
    el = time.perf_counter() - t0
    value = mesh.ncell * args.steps / el
    sample = "one oracle Heun step of the whole %d^3 turbulence box (the headline workload) per step" % n
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "turbulence-3d-%d^3-mixed" % n, "cells": mesh.ncell,
                   "sample": "oracle (FP64) on the same %d^3 box, %d cells, %d threads" % (n, mesh.ncell, used)},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": used, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--side", "--n", dest="n", type=int, default=256, help="side of the 3D turbulence box")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-grids measurement")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving measurement")
    ap.add_argument("--no-legs", action="store_true",
                    help="skip the FP64, FP32, van Leer and lean-Heun legs (headline only)")
    ap.add_argument("--serve-jobs", type=int, default=2000, help="jobs of the serving stream")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    ranks = Ranks(dist, "cuda")
    barrier, max_over_ranks = ranks.barrier, ranks.max

    from paper_2501_02317_gb300 import build as kbuild
    kbuild.build()
    from paper_2501_02317_gb300 import khydro
    from paper_2501_02317_gb300 import workloads as wl

    peak_gbs, peak_kind = _peaks()
    stream = torch.cuda.Stream()
    mesh, W = wl.turbulence(args.n, prec=wl.PREC_MIXED)
    ncell = mesh.ncell
    K, Wm = args.steps, args.warmup
    T_END = 1e30

    def timed_steps(sim, k):
        barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sim.enqueue_steps(T_END, k)
        e1.record(stream)
        e1.synchronize()
        torch.cuda.synchronize()
        barrier()
        return e0.elapsed_time(e1) / 1e3

    # ---------------------------------------------------------- mixed (headline)
    sim = khydro.Sim(mesh, stream=stream.cuda_stream)
    sim.set_primitive(W)
    sim.enqueue_steps(T_END, Wm)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        el = timed_steps(sim, K)
    clocks = clk.summary()
    el = max_over_ranks(el)
    value = whole_job_rate(world, ncell * K, el)
    flags, floors = sim.flags()
    ms = sim.profile_steps(T_END, 5)
    stage_ms = ms[1] + ms[2]
    achieved = BYTES_PER_CELL_UPDATE_3D * ncell / (stage_ms * 1e-3) / 1e9
    # DRAM bytes of the stage pair from the committed ncu capture (None when
    # the stage kernels' sources changed since)
    traffic = _recorded_traffic("turbulence-3d-%d^3-mixed" % args.n)

    # ---------------------------------------------------------- all-FP64 path
    fp64 = None
    value64 = None
    if not args.no_legs:
        mesh64 = mesh.replace(prec=wl.PREC_FP64)
        sim64 = khydro.Sim(mesh64, stream=stream.cuda_stream)
        sim64.set_primitive(W)
        sim64.enqueue_steps(T_END, 2)
        torch.cuda.synchronize()
        k64 = max(3, K // 10)
        el64 = max_over_ranks(timed_steps(sim64, k64))
        value64 = whole_job_rate(world, ncell * k64, el64)
        ms64 = sim64.profile_steps(T_END, 2)
        sim64.close()
        fp64 = {"value": value64, "unit": UNIT, "steps": k64, "ms_per_step": 1e3 * el64 / k64,
                "stage_ms": [ms64[1], ms64[2]],
                "roofline": fp64_roofline(ms64[1] + ms64[2], ncell, "turbulence-3d-fp64",
                                          torch.cuda.get_device_properties(local).multi_processor_count,
                                          _sm_max_mhz())}

    # ---------------------------------------------------------- all-FP32 path, van Leer (mixed)
    def leg(prec, integrator, k, bytes_per_cu):
        m = mesh.replace(prec=prec, integrator=integrator)
        s = khydro.Sim(m, stream=stream.cuda_stream)
        s.set_primitive(W)
        s.enqueue_steps(T_END, 3)
        torch.cuda.synchronize()
        t = max_over_ranks(timed_steps(s, k))
        pm = s.profile_steps(T_END, 3)
        state_bytes = s.device_bytes()[0]
        s.close()
        ach = bytes_per_cu * ncell / ((pm[1] + pm[2]) * 1e-3) / 1e9
        return {"value": whole_job_rate(world, ncell * k, t), "unit": UNIT, "steps": k, "ms_per_step": 1e3 * t / k,
                "stage_ms": [pm[1], pm[2]], "state_bytes": state_bytes, "bytes_per_cell_update": bytes_per_cu,
                "hbm_achieved_gbs": ach, "hbm_frac": ach / peak_gbs}

    fp32 = vl2 = lean = None
    if not args.no_legs:
        fp32 = dict(leg(wl.PREC_FP32, wl.INT_HEUN, K, BYTES_PER_CELL_UPDATE_3D_FP32),
                    workload="turbulence-3d-%d^3-fp32 (FP32 state and flux)" % args.n)
        vl2 = dict(leg(wl.PREC_MIXED, wl.INT_VL2, K, BYTES_PER_CELL_UPDATE_3D_VL2),
                   workload="turbulence-3d-%d^3-mixed, memory-optimized van Leer integrator" % args.n)
        lean = dict(leg(wl.PREC_MIXED, wl.INT_HEUN_LEAN, K, BYTES_PER_CELL_UPDATE_3D),
                    workload="turbulence-3d-%d^3-mixed, Heun without stored primitives" % args.n)

    # ---------------------------------------------------------- end to end (host buffers)
    # Each e2e step is one whole problem through the public API with host
    # buffers: khy_set_conserved from pinned host memory (the full 256^3
    # state), one Heun step, khy_get_conserved back to pinned host memory.
    # E2E_PIPELINES independent simulations, each with its own stream and
    # host thread, keep the host link busy in both directions at once
    # (host->device and device->host copies of different problems overlap,
    # and with the compute of a third); one pipeline is reported beside it.
    e2e = None
    if not args.no_e2e:
        import threading

        ke = max(3, min(K, 10))
        sims_e2e = [sim]
        streams_e2e = [stream]
        for _ in range(E2E_PIPELINES - 1):
            st = torch.cuda.Stream()
            s = khydro.Sim(mesh, stream=st.cuda_stream)
            s.set_primitive(W)
            s.enqueue_steps(T_END, 1)  # graphs captured before the threads start
            sims_e2e.append(s)
            streams_e2e.append(st)
        bufs = []
        for s in sims_e2e:
            Uh = torch.empty(mesh.shape, dtype=torch.float64, pin_memory=True).numpy()
            s.conserved(Uh)
            bufs.append(Uh)
        torch.cuda.synchronize()

        errors = []

        def pipeline(i, nsteps):
            try:
                torch.cuda.set_device(local)
                for _ in range(nsteps):
                    sims_e2e[i].set_conserved(bufs[i])
                    sims_e2e[i].enqueue_steps(T_END, 1)
                    sims_e2e[i].conserved(bufs[i])
            except Exception as e:  # re-raised on the main thread: no number from a failed pipeline
                errors.append(e)

        def run_e2e(npipe):
            barrier()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            th = [threading.Thread(target=pipeline, args=(i, ke)) for i in range(npipe)]
            for t in th:
                t.start()
            for t in th:
                t.join()
            torch.cuda.synchronize()
            if errors:
                raise errors[0]
            return max_over_ranks(time.perf_counter() - t0)

        el1 = run_e2e(1)
        elp = run_e2e(len(sims_e2e))
        e2e = {"value": whole_job_rate(world, ncell * ke * len(sims_e2e), elp), "unit": UNIT,
               "h2d_bytes_per_step": int(bufs[0].nbytes), "d2h_bytes_per_step": int(bufs[0].nbytes),
               "steps": ke * len(sims_e2e), "pipelines": len(sims_e2e),
               "single_pipeline": {"value": whole_job_rate(world, ncell * ke, el1), "steps": ke},
               "api": "khy_set_conserved(host) + khy_enqueue_steps(1) + khy_get_conserved(host); "
                      "%d independent simulations, one stream and one host thread each" % len(sims_e2e)}
        for s in sims_e2e[1:]:
            s.close()
    sim.close()

    batch = None if args.no_batch or world > 1 else bench_batch(khydro, wl, torch, peak_gbs=peak_gbs)
    serving = None if args.no_serve or world > 1 else bench_serving(khydro, wl, njobs=args.serve_jobs)

    cpu = None
    parity = None
    if rank == 0 and world == 1 and not args.no_cpu:
        csteps = 10
        v, cores, sample, Uo, _, W0 = cpu_oracle_rate(steps=csteps, n=args.n)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
               "host": host_cpu()}
        # the plain single-thread oracle beside the OpenMP build (same bits)
        v1, _, sample1, _, _, _ = cpu_oracle_rate(steps=1, n=args.n, threads=1)
        cpu["single_thread"] = {"value": v1, "unit": UNIT, "cores": 1, "sample": sample1}
        # the oracle's state after those steps is the reference of the
        # per-field errors of both GPU paths over the same steps
        parity = parity_against_oracle(khydro, wl, mesh, W0, Uo, csteps)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": Wm,
            "ms_per_step": 1e3 * el / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64 state, f32 reconstruction/flux", "data": "synthetic",
            "config": {"workload": "turbulence-3d-%d^3-mixed" % args.n, "cells": ncell, "prec": "mixed",
                       "cfl": mesh.cfl, "parallelism": "replicas" if world > 1 else "single",
                       "l2": "inputs larger than L2: two 5x8xN-byte states (%.0f MB each)" % (mesh.nvar * 8 * ncell / 1e6)},
            "fp64": fp64,
            "mixed_over_fp64": value / value64 if value64 else None,
            "fp32": fp32,
            "vl2_mixed": vl2,
            "heun_lean_mixed": lean,
            "parity_256": parity,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak_gbs, "unit": "GB/s",
                         "frac": achieved / peak_gbs,
                         "nominal_peak": NOMINAL_HBM_GBS, "frac_of_nominal": achieved / NOMINAL_HBM_GBS,
                         "traffic": traffic,
                         "traffic_gbs": traffic / (stage_ms * 1e-3) / 1e9 if traffic else None,
                         "algorithmic_bytes": BYTES_PER_CELL_UPDATE_3D * ncell,
                         "kernel": "stage_kernel (stage 1 + stage 2 of one Heun step)",
                         "bytes_per_cell_update": BYTES_PER_CELL_UPDATE_3D, "stage_ms": [ms[1], ms[2]],
                         "clock_ms": ms[0], "peak_kind": peak_kind},
            "issue_roofline": issue_roofline(stage_ms, ncell, "turbulence-3d-%d^3-mixed" % args.n,
                                             torch.cuda.get_device_properties(local).multi_processor_count,
                                             _sm_max_mhz()),
            "cpu_baseline": cpu,
            "batch": batch,
            "serving": serving,
            "e2e": e2e,
            "clocks": clocks,
            "gpu_launches": 3 * K,
            "gpu_launches_note": "timed region of the headline: clock + stage 1 + stage 2 per step",
            "status_flags": flags, "floor_hits": floors,
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
