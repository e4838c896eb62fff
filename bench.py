#!/usr/bin/env python
"""Benchmark of the GB300 MHD hot path: Mcell-updates/s of the RK2 Godunov
step (PLM-MC + HLLD + upwind CT + RK2 + device CFL) on the 3D decaying
turbulence box, 256^3 periodic, mixed FP32/FP64 precision.

One "step" is one full RK2 step (both fused stage kernels, with the CFL
max-reduction fused into stage 1 and the self-computed dt used by stage 2)
over the whole box.  Inputs are generated from the seeded turbulence recipe
(synthetic; the paper's runs use no dataset).  The resident buffers (4.1 GB:
state, stage increment, primitives) are far larger than the 129 MB L2, so no
flush is needed between steps.

Prints ONE JSON line on rank 0.  ``--impl reference`` times the FP64 CPU
oracle instead (on a bounded sample of the same workload).
Multi-GPU (torchrun, N > 1): every rank advances its own replica box (the
single-box path is not sharded); value = cells x steps x N / max-over-ranks
time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Mcell-updates/s on 1 GB300 at 256^3 MHD; % HBM roofline; vs plain FP64 at L1 error"
UNIT = "Mcell-updates/s"
# Minimum algorithmic HBM bytes per cell per stage launch (the roofline's
# numerator): only the conserved states move, halos come from cache.  RK2:
# stage 1 reads U^n (8 values) and writes U*, stage 2 reads U* and U^n and
# writes U^{n+1}; U^n and U^{n+1} are FP64 in the FP64 and mixed forms, U*
# is FP64 / FP32 / FP32.  FP64 128 + 192 = 320 B per cell-update, mixed
# 96 + 160 = 256, FP32 64 + 96 = 160.
MIN_STAGE_BYTES = {"fp64": (128, 192), "mixed": (96, 160), "fp32": (64, 96)}
# SSP-RK3 the same way: U1 and U2 in the bulk precision, U^n re-read by stages 2 and 3
MIN_STAGE_BYTES_RK3 = {"fp64": (128, 192, 192), "mixed": (96, 128, 160), "fp32": (64, 96, 96)}
# What this design's stage kernels move (reported beside the minimum): the
# primitives W (11 arrays) are stored once per state instead of recomputed in
# every halo copy, and RK2's stage increment K1 is stored in the bulk
# precision.  Stage 1 reads W and U^n, writes K1 and W(U*); stage 2 reads
# W(U*), U^n and K1, writes U^{n+1} and W(U^{n+1}).
STAGE_BYTES = {"fp64": (304, 368), "mixed": (184, 248), "fp32": (152, 184)}
# SSP-RK3 stages: read W(U_in), U_in (and U^n in stages 2, 3), write U_out, W(U_out)
STAGE_BYTES_RK3 = {"fp64": (304, 368, 368), "mixed": (216, 280, 280), "fp32": (152, 184, 184)}
# the host-core oracle legs (cpu_baseline and --impl reference) step one
# sample box of this edge per process
CPU_SAMPLE_N = 64
# the paper's own run of this workload (FP64, RK3, 3D OT 352^3, 10 steps): context, not a target
PAPER_OT352 = {"time_10_steps_s": 13.9, "hardware": "NVIDIA A100 64 GB (Leonardo), NVHPC 24.5 OpenACC, managed memory",
               "note": "total time of 10 steps of the paper's 3D Orszag-Tang test (Sec. 4, its figure of total "
                       "execution time); other hardware and a whole-application time: context only"}
# Algorithmic flops per cell-update (one full step with its CFL maximum),
# counted by the operation-counting build of the oracle on 32^3 patterns of
# each workload's start state (oracle/opcount_table.py writes the table these
# figures are copied from; a CPU test keeps the two equal).  "fp64" is the part
# the mixed form computes in FP64 (primitive recoveries, RK accumulation), the
# rest is FP32 there; the FP64 form computes all of it in FP64.
FLOPS = {
    ("turbulence", "primitive", "rk2"): {"total": 3438.012, "fp64_in_mixed": 112.0},
    ("turbulence", "characteristic", "rk2"): {"total": 10301.774, "fp64_in_mixed": 112.0},
    ("orszag_tang", "primitive", "rk2"): {"total": 3293.019, "fp64_in_mixed": 112.0},
    ("orszag_tang", "primitive", "rk3"): {"total": 4934.793, "fp64_in_mixed": 192.0},
}
# the learned switch's network per face: 2 (16*32 + 32*32 + 32) flops, on the
# lower x-, y- and z-faces of every cell in both stages
MLP_FLOPS_PER_FACE = 2 * (16 * 32 + 32 * 32 + 32)
# nominal arithmetic peaks from unit counts and the maximum SM clock: 152 SMs
# x 2070 MHz x (2 FP64 FMA lanes per SM per clock, 128 FP32 FMA lanes) x 2
# flops per FMA (the FP64 figure is GB300's 1.25 TFLOP/s FP64 rating)
SMS, SM_MAX_GHZ = 152, 2.070
FP64_NOMINAL_TFLOPS = SMS * SM_MAX_GHZ * 2 * 2 / 1e3
FP32_NOMINAL_TFLOPS = SMS * SM_MAX_GHZ * 128 * 2 / 1e3
CLOCK_QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
               "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
               "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="turbulence256",
                   choices=["turbulence256", "turbulence256_learned", "ot2d128", "ot3d512", "ot3d352_rk3",
                            "riemann2d3200_hll", "blast_batch64"])
    p.add_argument("--precision", default=None, choices=["mixed", "fp64", "fp32"])
    p.add_argument("--n", type=int, default=None)
    p.add_argument("--tile", default="0,0,0")
    p.add_argument("--compare-steps", type=int, default=10)
    p.add_argument("--e2e-steps", type=int, default=40)
    p.add_argument("--cpu-seconds", type=float, default=12.0)
    p.add_argument("--no-extras", action="store_true", help="skip the FP64 comparison, e2e and CPU legs")
    p.add_argument("--recon", default="primitive", choices=["primitive", "characteristic"],
                   help="reconstruction of single-box workloads")
    p.add_argument("--switch-faces", type=int, default=10_000_000, help="training faces of the learned switch")
    p.add_argument("--switch-steps", type=int, default=3000, help="Adam steps of the learned switch")
    return p.parse_args()


# instruction issue: one warp-instruction per clock per scheduler, 4 schedulers per SM
ISSUE_PEAK_WARP_INST_PER_S = SMS * 4 * SM_MAX_GHZ * 1e9
SLOWDOWNS = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown")


def clocks_disqualify(clocks) -> bool:
    """Whether a timed run's clock samples rule it out: a hardware or thermal
    slowdown, or an SM clock well below its maximum with no reason given (a
    clock lock left behind).  A power cap alone does not (a 1.4 kW part under
    a dense load); no samples cannot decide either way."""
    if not clocks:
        return False
    if set(clocks["reasons"]) & set(SLOWDOWNS):
        return True
    return not clocks["reasons"] and clocks["sm_mhz"] < 0.9 * clocks["sm_max_mhz"]


def max_over_ranks(value: float, world: int, device="cuda") -> float:
    """MAX of a per-rank float over all ranks of the process group (one
    collective; the timing rule takes the slowest rank)."""
    if world <= 1:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_rate(cells_per_rank: int, steps: int, ms_max: float, world: int) -> float:
    """Whole-job Mcell-updates/s: every rank advances its own replica of the
    workload (replicas only: the single-box path does not shard), timed by
    the slowest rank."""
    return world * cells_per_rank * steps / (ms_max / 1e3) / 1e6


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def flop_counts(args, box):
    """Algorithmic flops per cell-update of this run's workload, or None
    (uncounted workloads; the learned switch, whose HLL/HLLD mix varies)."""
    if args.workload == "turbulence256_learned":
        return None
    kind = "turbulence" if box.name.startswith("turbulence") else (
        "orszag_tang" if box.name.startswith("orszag_tang_3d") else None)
    key = (kind, args.recon, "rk3" if args.workload == "ot3d352_rk3" else "rk2")
    return FLOPS.get(key)


def pipe_report(args, box, value_mcells, measured):
    """FP64 and FP32 arithmetic rates of the run (algorithmic flops x
    cell-updates/s) against the nominal and the measured pipe peaks."""
    fl = flop_counts(args, box)
    if fl is None:
        return None
    if args.precision == "fp64":
        f64, f32 = fl["total"], 0.0
    elif args.precision == "mixed":
        f64, f32 = fl["fp64_in_mixed"], fl["total"] - fl["fp64_in_mixed"]
    else:
        f64, f32 = 0.0, fl["total"]
    rate = value_mcells * 1e6
    rep = {"flops_per_cell_update": fl["total"], "source": "operation-counting build of the oracle"}
    for name, fpc, nom, meas in (("fp64", f64, FP64_NOMINAL_TFLOPS, measured.get("fp64_fma_tflops")),
                                 ("fp32", f32, FP32_NOMINAL_TFLOPS, measured.get("fp32_fma_tflops"))):
        ach = rate * fpc / 1e12
        rep[name] = {"flops_per_cell_update": fpc, "achieved_tflops": ach, "peak_tflops": nom,
                     "frac": ach / nom, "measured_peak_tflops": meas,
                     "frac_of_measured": ach / meas if meas else None}
    return rep


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 50 ms with
    timestamps.  Started before the warm-up (it waits for its first sample),
    marked around the timed region; the summary keeps the samples inside the
    timed region, widened back into the warm-up that ran just before it when
    fewer than 3 fell inside (the window used is reported)."""

    def __init__(self, index, interval_ms=50):
        self.index = index
        self.interval_ms = interval_ms
        self.proc = None
        self.t0 = self.t1 = None
        out = os.environ.get("MHD_CLOCKS_DIR") or tempfile.gettempdir()   # where the raw samples go
        self.path = os.path.join(out, f"clocks_bench_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu=timestamp,{CLOCK_QUERY}",
                                          "--format=csv,noheader,nounits", "-i", str(self.index),
                                          "-lms", str(self.interval_ms)], stdout=self.f, stderr=subprocess.DEVNULL)
            deadline = time.time() + 3.0
            while time.time() < deadline and os.path.getsize(self.path) == 0:
                time.sleep(0.02)
        except Exception:
            self.proc = None
        return self

    def mark_start(self):
        self.t0 = time.time()

    def mark_end(self):
        self.t1 = time.time()

    def stop(self):
        if self.proc is not None:
            time.sleep(self.interval_ms / 1000.0)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def _samples(self):
        import datetime
        out = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 10:
                continue
            try:
                ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                out.append((ts, float(parts[2]), float(parts[3]), parts[6:10]))
            except ValueError:
                continue
        return out

    def summary(self):
        if self.proc is None or self.t0 is None or self.t1 is None:
            return None
        try:
            samples = self._samples()
        except FileNotFoundError:
            return None
        lo, window = self.t0, "timed region"
        inside = [x for x in samples if lo <= x[0] <= self.t1]
        while len(inside) < 3 and lo > self.t0 - 2.0:
            lo -= 0.1
            inside = [x for x in samples if lo <= x[0] <= self.t1]
            window = f"timed region + the preceding {self.t0 - lo:.1f} s of warm-up"
        if not inside:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for x in inside:
            for nm, val in zip(names, x[3]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(x[1] for x in inside), "sm_max_mhz": max(x[2] for x in inside),
                "reasons": sorted(reasons), "samples": len(inside), "window": window,
                "timed_s": round(self.t1 - self.t0, 3)}


def kernel_source_digest() -> str:
    """Hash of the CUDA sources with comments and blank space removed, and of
    the compiler flags (without machine paths), so that only a change of what
    is compiled invalidates a recorded capture."""
    import hashlib
    import re
    from paper_2606_12753_gb300 import _build
    h = hashlib.sha1()
    for p in _build._deps():
        if p.endswith((".cu", ".cuh")):
            src = open(p, encoding="utf-8").read()
            src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
            src = re.sub(r"//[^\n]*", " ", src)
            h.update(" ".join(src.split()).encode())
    flags = [x for x in _build.ARCH + _build.NVCC_FLAGS if not os.path.isabs(x)]
    flags += _build.FAST_FP32_FLAGS + sorted(_build.FAST_FP32_UNITS)
    h.update(" ".join(flags).encode())
    return h.hexdigest()[:12]


def profile_record(kernel_tag):
    """The fields profiles/traffic.txt records for this kernel (ncu counts per
    launch), if the kernel code is unchanged since the capture; else None."""
    digest = kernel_source_digest()
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    try:
        for line in open(path):
            f = dict(kv.split("=", 1) for kv in line.split() if "=" in kv)
            if f.get("kernel") == kernel_tag and f.get("src") == digest:
                return f, digest
    except FileNotFoundError:
        pass
    return None, digest


def traffic_from_profiles(kernel_tag):
    """ncu DRAM bytes per launch recorded for this kernel (None when stale)."""
    rec, digest = profile_record(kernel_tag)
    return (float(rec["dram_bytes_per_launch"]) if rec else None), digest


def _oracle_worker(n, warmup, steps, barrier, seconds=None):
    """One host process: the FP64 oracle (as it stands) on its own n^3 sample
    of the turbulence workload; `warmup` untimed steps, then `steps` timed
    steps (or as many as fit in `seconds`).  Returns (cells x steps, seconds)."""
    import oracle as O
    from paper_2606_12753_gb300 import inputs as I
    box = I.turbulence_3d(n)
    cfg = O.Config(box.nx, box.ny, box.nz, box.dx, box.dy, box.dz, box.gamma, 0.4, box.bc)
    cell, face = box.cell, box.face
    for _ in range(warmup):
        cell, face, _ = O.step(cfg, cell, face, -1.0, nsteps=1)
    if barrier is not None:
        barrier.wait()
    done, t0 = 0, time.perf_counter()
    while done < steps or (seconds is not None and time.perf_counter() - t0 < seconds):
        cell, face, _ = O.step(cfg, cell, face, -1.0, nsteps=1)
        done += 1
    return box.ncell * done, time.perf_counter() - t0


def oracle_throughput(n: int, steps: int, warmup: int, workers: int, seconds=None):
    """Whole-host rate of the oracle: `workers` independent processes (spawned,
    so none inherits a CUDA context), each stepping its own sample, released
    together after their warm-up.  Rate = all cell-updates / the slowest
    process's time.  Returns (Mcell-updates/s, cell-updates, seconds)."""
    import concurrent.futures as cf
    import multiprocessing as mp
    import oracle as O
    O.build()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        barrier = mgr.Barrier(workers) if workers > 1 else None
        with cf.ProcessPoolExecutor(max_workers=workers, mp_context=ctx) as ex:
            futs = [ex.submit(_oracle_worker, n, warmup, steps, barrier, seconds) for _ in range(workers)]
            res = [f.result() for f in futs]
    cells = sum(r[0] for r in res)
    el = max(r[1] for r in res)
    return cells / el / 1e6, cells, el


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_oracle_rate(seconds: float, n: int = CPU_SAMPLE_N):
    """The FP64 oracle on the host cores: one process per core, each on its
    own n^3 sample of the turbulence workload, for about ``seconds``; plus the
    same on one core alone."""
    cores = host_cores()
    one, _, el1 = oracle_throughput(n, 0, 0, 1, seconds=seconds / 3)
    allc, cells, el = oracle_throughput(n, 1, 0, cores, seconds=seconds)
    return {"value": allc, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"turbulence_3d recipe at {n}^3 per process, {cores} processes (one per host core) of "
                      f"RK2 steps with CFL dt for {el:.1f} s ({cells / n ** 3:.0f} box-steps)",
            "single_core": {"value": one, "cores": 1, "seconds": round(el1, 1)}}


WORKLOADS = {
    "turbulence256": ("mixed", 256),
    "turbulence256_learned": ("mixed", 256),
    "ot3d352_rk3": ("fp64", 352),
    "riemann2d3200_hll": ("fp64", 3200),
    "ot2d128": ("fp64", 128),
    "ot3d512": ("mixed", 512),
    "blast_batch64": ("fp32", 64),
}


def resolve(args):
    prec, n = WORKLOADS[args.workload]
    args.precision = args.precision or prec
    args.n = args.n or n


def make_box(args):
    from paper_2606_12753_gb300 import inputs as I
    if args.workload == "ot2d128":
        return I.orszag_tang_2d(args.n)
    if args.workload in ("ot3d512", "ot3d352_rk3"):
        return I.orszag_tang_3d(args.n, seed=12753)
    if args.workload == "riemann2d3200_hll":
        return I.riemann_2d(args.n, seed=3200)
    return I.turbulence_3d(args.n, seed=2606)


def workload_config(args):
    text = {
        "turbulence256": f"turbulence_3d_{args.n}: 3D decaying MHD turbulence {args.n}^3 periodic, "
                         f"rho=1 p=0.6 rms Mach 1 beta=1, PLM-MC+HLLD+upwind CT+RK2, CFL 0.4",
        "turbulence256_learned": f"turbulence_3d_{args.n}_learned: 3D decaying MHD turbulence {args.n}^3 periodic "
                                 f"as turbulence256, per-face learned HLL/HLLD switch (BF16 MLP 16-32-32-1, "
                                 f"FP32 accumulation) trained on the GPU on 1e7 faces of FP64 runs (seed 5)",
        "ot2d128": f"orszag_tang_2d_{args.n}: 2D Orszag-Tang {args.n}^2 periodic, PLM-MC+HLLD+upwind CT+RK2, CFL 0.4",
        "ot3d512": f"orszag_tang_3d_{args.n}: 3D Orszag-Tang {args.n}^3 periodic (+1% velocity noise), "
                   f"PLM-MC+HLLD+upwind CT+RK2, CFL 0.4",
        "ot3d352_rk3": f"orszag_tang_3d_{args.n}_rk3: 3D Orszag-Tang {args.n}^3 periodic (+1% velocity noise), "
                       f"PLM-MC+HLLD+upwind CT+SSP-RK3 (the paper's integrator and 3D OT size), CFL 0.4",
        "riemann2d3200_hll": f"riemann2d_{args.n}: seeded four-quadrant 2D MHD Riemann problem {args.n}^2 x 1, "
                             f"outflow, PLM-MC+HLL+upwind CT+RK2, CFL 0.4 (stand-in for the paper's 2D Riemann "
                             f"test, whose quadrant states it does not print)",
        "blast_batch64": f"blast_batch_{args.n}: {args.n} outflow MHD blast boxes, 32-128 cells per axis "
                         f"log-uniform, one persistent launch per call, autotuned tile, per-box CFL 0.4",
    }[args.workload]
    out = {"workload": text, "precision": args.precision, "n": args.n}
    if getattr(args, "recon", "primitive") != "primitive":
        out["recon"] = args.recon
    return out


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    n = CPU_SAMPLE_N
    cores = host_cores()
    value, cells, el = oracle_throughput(n, args.steps, args.warmup, cores)
    sample = (f"turbulence_3d recipe at {n}^3 per process, {cores} processes (one per host core); each step is "
              f"one RK2 step of the FP64 oracle in every process")
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": el * 1e3 / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic",
           "config": dict(workload_config(args), sample=f"{cores} x {n}^3 per step, FP64 oracle on the host cores"),
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
           "gpu_launches": 0}
    print(json.dumps(out), flush=True)


def run_ours(args):
    import numpy as np
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2606_12753_gb300 import inputs as I
    from paper_2606_12753_gb300 import mhd

    tile = tuple(int(x) for x in args.tile.split(","))
    box = make_box(args)
    learned = args.workload == "turbulence256_learned"
    rk3 = args.workload == "ot3d352_rk3"
    stage_bytes = (STAGE_BYTES_RK3 if rk3 else STAGE_BYTES)[args.precision]
    min_bytes = (MIN_STAGE_BYTES_RK3 if rk3 else MIN_STAGE_BYTES)[args.precision]
    switch_rep = None
    if learned:
        # training (not timed): faces of FP64 turbulence runs with seed 5,
        # the library's BF16 forward/backward and Adam kernels
        from paper_2606_12753_gb300 import switch_train as T
        sw, tau, switch_rep = T.train_switch(n=args.n, nfaces=args.switch_faces, seed=5, steps=args.switch_steps,
                                             batch=16384)
    stream = torch.cuda.Stream()
    riemann = "learned" if learned else ("hll" if args.workload == "riemann2d3200_hll" else "hlld")
    solver = mhd.Solver(box, precision=args.precision, riemann=riemann, tile=tile,
                        stream=stream.cuda_stream, integrator="rk3" if rk3 else "rk2", recon=args.recon)
    if learned:
        solver.set_switch(sw.block.data_ptr(), tau)
    solver.set_state(box.cell, box.face)

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
            torch.cuda.synchronize()

    def timed_once():
        """W warm-up steps, then K steps timed with CUDA events on the
        solver's stream, clocks sampled throughout."""
        clk = ClockSampler(local).start()
        solver.step_async(-1.0, args.warmup)
        st_w = solver.stats()
        solver.set_profiling(True)
        solver.profile()
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        clk.mark_start()
        e0.record(stream)
        solver.step_async(-1.0, args.steps)
        e1.record(stream)
        stream.synchronize()
        clk.mark_end()
        clk.stop()
        barrier()
        stage_ms, launches = solver.profile()
        solver.set_profiling(False)
        return e0.elapsed_time(e1), stage_ms, launches, clk.summary(), st_w

    ms_total, stage_ms, launches, clocks, st_w = timed_once()
    if max_over_ranks(1.0 if clocks_disqualify(clocks) else 0.0, world) > 0:
        first = clocks   # measured once more; the first run's clocks are kept for the record
        ms_total, stage_ms, launches, clocks, st_w = timed_once()
        if clocks is not None:
            clocks["remeasured_after"] = first
    e0 = torch.cuda.Event(enable_timing=True)   # for the comparison legs below
    e1 = torch.cuda.Event(enable_timing=True)
    st = solver.stats()
    if st["status"] != 0:
        raise RuntimeError(f"device status {st['status']} after the timed steps")
    ms_total = max_over_ranks(ms_total, world)
    value = job_rate(box.ncell, args.steps, ms_total, world)

    measured = mhd.mhd_measure_pipe_peaks(stream.cuda_stream)
    peak, peak_kind = peaks()
    nst = len(stage_bytes)
    k = max(range(nst), key=lambda i: stage_ms[i] / max(launches[i], 1))
    per_launch_ms = stage_ms[k] / max(launches[k], 1)
    alg_bytes = min_bytes[k] * box.ncell
    achieved = alg_bytes / (per_launch_ms / 1e3) / 1e9
    design_achieved = stage_bytes[k] * box.ncell / (per_launch_ms / 1e3) / 1e9
    kname = "stage_kernel" + ("_learned" if learned else "") + ("_rk3" if rk3 else "") + \
        ("_char" if args.recon == "characteristic" else "")
    tag = f"{kname}<{args.precision},{k + 1}>@{box.name}"
    traffic, src = traffic_from_profiles(tag)
    elem = 4 if args.precision == "fp32" else 8
    kelem = 8 if args.precision == "fp64" else 4
    resident = box.ncell * (8 * (2 * elem + kelem) + 2 * 11 * kelem)
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_total / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": {"mixed": "f32+f64", "fp64": "f64", "fp32": "f32"}[args.precision],
        "data": "synthetic",
        "config": {**workload_config(args),
                   "tile": [solver.cfg.tile_x, solver.cfg.tile_y, solver.cfg.tile_z],
                   "l2": f"inputs larger than L2 (state + stage buffers {resident / 1e9:.1f} GB > 129 MB), no flush",
                   "parallelism": f"replicas x{world}" if world > 1 else "single box"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "kernel": tag, "peak_kind": peak_kind,
                     "bytes_per_cell": min_bytes[k], "bytes_basis": "minimum: conserved states only",
                     "traffic_ratio": traffic / alg_bytes if traffic else None,
                     "frac_design": design_achieved / peak, "design_bytes_per_cell": stage_bytes[k],
                     "step_frac": value * 1e6 / world * sum(min_bytes) / 1e9 / peak},
        "stage_ms_per_launch": [stage_ms[i] / max(launches[i], 1) for i in range(nst)],
        "gpu_launches": nst * args.steps,
    }
    # the same kernel against the SM's instruction-issue rate, from the
    # executed warp-instructions ncu recorded for it (null once stale)
    rec, _ = profile_record(tag)
    out["roofline_issue"] = None
    if rec and "warp_inst_per_launch" in rec:
        inst = float(rec["warp_inst_per_launch"])
        rate = inst / (per_launch_ms / 1e3)
        out["roofline_issue"] = {"bound": "issue", "achieved": rate / 1e9, "peak": ISSUE_PEAK_WARP_INST_PER_S / 1e9,
                                 "unit": "G warp-instructions/s", "frac": rate / ISSUE_PEAK_WARP_INST_PER_S,
                                 "kernel": tag, "warp_instructions_per_launch": inst,
                                 "source": "ncu smsp__inst_executed.sum (profiles/traffic.txt)"}
    out["pipes"] = pipe_report(args, box, value / world, measured)
    if out["pipes"] is not None:
        out["pipes"]["measured_peaks"] = measured
    if args.precision == "fp64" and out["pipes"] is not None:
        # the FP64 form is bound by its FP64 pipe: its roofline is arithmetic,
        # the algorithmic flops of an average stage launch over the mean stage
        # launch time, against the nominal FP64 peak
        mean_ms = sum(stage_ms[i] / max(launches[i], 1) for i in range(nst)) / nst
        fl = out["pipes"]["flops_per_cell_update"] * box.ncell / nst
        ach = fl / (mean_ms / 1e3) / 1e12
        out["roofline_hbm"] = out["roofline"]
        out["roofline"] = {"bound": "alu", "achieved": ach, "peak": FP64_NOMINAL_TFLOPS, "unit": "TFLOP/s",
                           "frac": ach / FP64_NOMINAL_TFLOPS, "traffic": traffic, "kernel": tag,
                           "peak_kind": "nominal (152 SMs x 2070 MHz x 2 FP64 FMA lanes x 2 flops)",
                           "measured_peak": measured["fp64_fma_tflops"],
                           "frac_of_measured": ach / measured["fp64_fma_tflops"],
                           "flops_per_launch": fl}
    if learned:
        mlp = 6 * MLP_FLOPS_PER_FACE * value / world * 1e6 / 1e12
        out["pipes_tensor"] = {"mlp_flops_per_cell_update": 6 * MLP_FLOPS_PER_FACE, "achieved_tflops": mlp,
                               "mma_sync_measured_peak_tflops": measured["bf16_mma_sync_tflops"],
                               "frac_of_mma_sync": mlp / measured["bf16_mma_sync_tflops"]}
    if rk3:
        out["config"]["integrator"] = "SSP-RK3 (3 stage launches per step)"
        out["time_10_steps_s"] = 10 * ms_total / args.steps / 1e3
        out["paper_context"] = PAPER_OT352
    if learned:
        nh = st["faces_hll"] - st_w["faces_hll"]
        nd = st["faces_hlld"] - st_w["faces_hlld"]
        out["switch"] = {**switch_rep, "timed_hll_frac": nh / max(nh + nd, 1)}
    with_extras = rank == 0 and world == 1 and not args.no_extras
    if with_extras:
        # end to end through the public API with host buffers: per step the
        # state goes host -> device, one RK2 step (CFL dt) runs, the new state
        # comes back device -> host (pinned host memory both ways)
        ncell = box.ncell
        dtype = torch.float32 if args.precision == "fp32" else torch.float64
        cell_h = torch.from_numpy(box.cell.astype(np.float32 if args.precision == "fp32" else np.float64)).pin_memory()
        face_h = [torch.from_numpy(f.astype(cell_h.numpy().dtype)).pin_memory() for f in box.face]
        out_c = torch.empty_like(cell_h).pin_memory()
        out_f = [torch.empty_like(f).pin_memory() for f in face_h]
        nbytes = cell_h.numel() * cell_h.element_size() + sum(f.numel() * f.element_size() for f in face_h)
        h = solver.h
        # sequential: set_state, step, get_state, each waiting for the last
        mhd.mhd_set_state(h, [cell_h[v].data_ptr() for v in range(5)], [f.data_ptr() for f in face_h], 0)
        mhd.mhd_step(h, -1.0, 1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            mhd.mhd_set_state(h, [cell_h[v].data_ptr() for v in range(5)], [f.data_ptr() for f in face_h], 0)
            mhd.mhd_step(h, -1.0, 1)
            mhd.mhd_get_state(h, [out_c[v].data_ptr() for v in range(5)], [f.data_ptr() for f in out_f], 0)
        el_seq = time.perf_counter() - t0
        # streamed (mhd_stream_step): a stream of host states, each copied in,
        # stepped and copied out; the copies of one state overlap the step of
        # the next.  Every step's copies are inside the timed region.
        out2 = (torch.empty_like(cell_h).pin_memory(), [torch.empty_like(f).pin_memory() for f in face_h])
        outs = [(out_c, out_f), out2]
        solver.stream_step(cell_h, face_h, out_c, out_f, -1.0)
        solver.stream_sync()
        t0 = time.perf_counter()
        for i in range(args.e2e_steps):
            solver.stream_step(cell_h, face_h, outs[i % 2][0], outs[i % 2][1], -1.0)
        solver.stream_sync()
        el = time.perf_counter() - t0
        out["e2e"] = {"value": ncell * args.e2e_steps / el / 1e6, "unit": UNIT, "h2d_bytes_per_step": nbytes,
                      "d2h_bytes_per_step": nbytes, "steps": args.e2e_steps,
                      "mode": "mhd_stream_step: independent host states (pinned), each copied in, advanced one "
                              "step (CFL dt) and copied out; copies overlap the neighbouring steps",
                      "sequential_value": ncell * args.e2e_steps / el_seq / 1e6,
                      "sequential_mode": "mhd_set_state + mhd_step + mhd_get_state per step, no overlap"}
        # plain FP64 path on the same GPU and the L1 error of this path against it
        cmp = {}
        dt = solver.cfl_dt()
        ref = mhd.Solver(box, precision="fp64", riemann="hll" if riemann == "hll" else "hlld", stream=stream.cuda_stream,
                         integrator="rk3" if rk3 else "rk2", recon=args.recon)
        ref.set_state(box.cell, box.face)
        ref.step(dt, 1)
        ref.set_state(box.cell, box.face)
        torch.cuda.synchronize()
        e0.record(stream)
        ref.step_async(dt, args.compare_steps)
        e1.record(stream)
        stream.synchronize()
        fp64_ms = e0.elapsed_time(e1) / args.compare_steps
        ref.stats()
        rc, rf = ref.get_state()
        ref.close()
        solver.set_state(box.cell, box.face)
        solver.step(dt, args.compare_steps)
        c, f = solver.get_state()
        l1 = {}
        names = ["rho", "mx", "my", "mz", "E", "Bx", "By", "Bz"]
        for v in range(5):
            l1[names[v]] = float(np.abs(c[v] - rc[v]).sum() / np.abs(rc[v]).sum())
        bnorm = sum(float(np.abs(x).sum()) for x in rf)
        for d in range(3):
            l1[names[5 + d]] = float(np.abs(f[d] - rf[d]).sum() / max(np.abs(rf[d]).sum(), 1e-3 * bnorm))
        cmp = {"fp64_value": box.ncell / (fp64_ms / 1e3) / 1e6, "unit": UNIT, "fp64_ms_per_step": fp64_ms,
               "steps": args.compare_steps, "dt": dt, "l1_rel_vs_fp64": l1,
               "note": "FP64 GPU path with the same integrator (parity with the FP64 oracle at 1e-12) as the "
                       "reference"}
        if learned:
            # the method without the switch (HLLD on every face) and HLL on
            # every face, same precision, same dt, same steps
            for name in ("hlld", "hll"):
                alt = mhd.Solver(box, precision=args.precision, riemann=name, stream=stream.cuda_stream)
                alt.set_state(box.cell, box.face)
                alt.step(dt, 1)
                alt.set_state(box.cell, box.face)
                torch.cuda.synchronize()
                e0.record(stream)
                alt.step_async(dt, args.compare_steps)
                e1.record(stream)
                stream.synchronize()
                ams = e0.elapsed_time(e1) / args.compare_steps
                ac, af = alt.get_state()
                alt.close()
                al1 = {}
                for v in range(5):
                    al1[names[v]] = float(np.abs(ac[v] - rc[v]).sum() / np.abs(rc[v]).sum())
                for d in range(3):
                    al1[names[5 + d]] = float(np.abs(af[d] - rf[d]).sum() / max(np.abs(rf[d]).sum(), 1e-3 * bnorm))
                cmp[f"{name}_ms_per_step"] = ams
                cmp[f"{name}_l1_rel_vs_fp64"] = al1
            solver.set_state(box.cell, box.face)
            solver.step(dt, 1)
            solver.set_state(box.cell, box.face)
            torch.cuda.synchronize()
            e0.record(stream)
            solver.step_async(dt, args.compare_steps)
            e1.record(stream)
            stream.synchronize()
            cmp["learned_ms_per_step"] = e0.elapsed_time(e1) / args.compare_steps
        out["vs_fp64"] = cmp
        out["cpu_baseline"] = cpu_oracle_rate(args.cpu_seconds)
    elif rank == 0:
        out["e2e"] = None
    out["clocks"] = clocks
    solver.close()
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def run_batch(args):
    """64 independent outflow blast boxes advanced by one persistent launch
    per call (all K timed steps in one launch, replayed from a CUDA graph)."""
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        torch.distributed.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
            torch.cuda.synchronize()

    from paper_2606_12753_gb300 import inputs as I
    from paper_2606_12753_gb300 import mhd
    boxes = I.blast_batch(args.n, seed=64)
    ncell = sum(b.ncell for b in boxes)
    stream = torch.cuda.Stream()
    batch = mhd.Batch(boxes, precision=args.precision, stream=stream.cuda_stream)
    for i, b in enumerate(boxes):
        batch.set_state(i, b.cell, b.face)
    tile = tuple(int(x) for x in args.tile.split(","))
    if any(tile):
        batch.set_tile(*tile)       # an explicit tile: no autotuning (a fixed launch sequence)
        tune_ms = None
    else:
        cache = os.environ.get("MHD_AUTOTUNE_CACHE") or os.path.join(tempfile.gettempdir(), "mhd_autotune.jsonl")
        tile, tune_ms = batch.autotune(trial_steps=3, cache_path=cache)
    def timed_once():
        clk = ClockSampler(local).start()
        batch.step(-1.0, args.warmup)
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        clk.mark_start()
        e0.record(stream)
        batch.step_async(-1.0, args.steps)
        e1.record(stream)
        stream.synchronize()
        clk.mark_end()
        clk.stop()
        barrier()
        return e0.elapsed_time(e1), clk.summary()

    ms_local, clocks = timed_once()
    if max_over_ranks(1.0 if clocks_disqualify(clocks) else 0.0, world) > 0:
        first = clocks
        ms_local, clocks = timed_once()
        if clocks is not None:
            clocks["remeasured_after"] = first
    ms_total = max_over_ranks(ms_local, world)
    st = batch.stats()
    if st["status"] != 0:
        raise RuntimeError(f"device status {st['status']} after the timed steps")
    value = job_rate(ncell, args.steps, ms_total, world)
    peak, peak_kind = peaks()
    step_bytes = sum(MIN_STAGE_BYTES[args.precision]) * ncell
    achieved = step_bytes * args.steps / (ms_total / 1e3) / 1e9
    design_achieved = sum(STAGE_BYTES[args.precision]) * ncell * args.steps / (ms_total / 1e3) / 1e9
    (tx, ty, tz), items, grid = batch.tile()
    seq = None
    if rank == 0 and world == 1 and not args.no_extras:
        seq = single_box_sequence(args, boxes, stream, barrier)
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_total / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": {"mixed": "f32+f64", "fp64": "f64", "fp32": "f32"}[args.precision], "data": "synthetic",
        "config": {**workload_config(args), "cells": ncell, "tile": [tx, ty, tz], "work_items": items,
                   "persistent_grid": grid, "autotune_ms_per_step": tune_ms,
                   "l2": "inputs larger than L2",
                   "parallelism": (f"replicas x{world}, " if world > 1 else "") + "all boxes of a GPU in one launch"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": None, "kernel": f"batch_kernel<{args.precision},{tx}x{ty}>@blast_batch_{args.n}",
                     "peak_kind": peak_kind, "bytes_per_cell": sum(MIN_STAGE_BYTES[args.precision]),
                     "bytes_basis": "minimum: conserved states only, per cell-update",
                     "frac_design": design_achieved / peak},
        "gpu_launches": 2 if args.steps else 0,
        "e2e": None,
        "clocks": clocks,
    }
    if seq is not None:
        out["vs_single_box_calls"] = {**seq, "batched_value": value, "batched_over_single": value / seq["value"]}
    batch.close()
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def single_box_sequence(args, boxes, stream, barrier):
    """The same boxes advanced through one single-box handle each (the plain
    path): per step, every handle's RK2 step with its own CFL dt (2 stage
    launches per box), all K steps captured in one CUDA graph and replayed,
    timed like the batch.  Returns the rate and how it was taken."""
    import torch
    from paper_2606_12753_gb300 import mhd
    solvers = [mhd.Solver(b, precision=args.precision, stream=stream.cuda_stream) for b in boxes]
    for s, b in zip(solvers, boxes):
        s.set_state(b.cell, b.face)
    for s in solvers:
        s.step_async(-1.0, 2)          # primitives valid, every handle warm
    torch.cuda.synchronize()
    k = args.steps + (args.steps % 2)  # an even count returns each ping-pong buffer to its start
    graph, mode = None, "CUDA graph of K steps x 64 handles"
    try:
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=stream):
            for _ in range(k):
                for s in solvers:
                    s.step_async(-1.0, 1)
    except Exception as exc:                                 # capture refused: time plain launches
        graph, mode = None, f"asynchronous launches (graph capture failed: {type(exc).__name__})"
        torch.cuda.synchronize()

    def run():
        if graph is not None:
            with torch.cuda.stream(stream):   # replay on the stream the events are recorded on
                graph.replay()
        else:
            for _ in range(k):
                for s in solvers:
                    s.step_async(-1.0, 1)

    for _ in range(max(1, args.warmup // 2)):
        run()
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    run()
    e1.record(stream)
    stream.synchronize()
    ms = e0.elapsed_time(e1)
    bad = [s.stats()["status"] for s in solvers if s.stats()["status"] != 0]
    for s in solvers:
        s.close()
    if bad:
        raise RuntimeError(f"device status {bad[0]} in the single-box sequence")
    ncell = sum(b.ncell for b in boxes)
    return {"value": ncell * k / (ms / 1e3) / 1e6, "unit": UNIT, "steps": k, "ms_per_step": ms / k,
            "launches_per_step": 2 * len(boxes), "mode": mode}


def main():
    args = parse()
    resolve(args)
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "blast_batch64":
        run_batch(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
