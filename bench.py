#!/usr/bin/env python
"""Benchmark of the improved-staggered CG on one GB300 (or N replicas).

Workload: the single-mass 32^4 lattice, m = 0.01, seeded random fat/long
links (fat = 0.9 SU(3), long = -1/24 times a product of three SU(3)),
antiperiodic time, one Gaussian source; the mixed-precision CG (FP32 Dslash
and vectors, FP64 x, reductions and reliable updates) solved from x0 = 0 to
a true relative residual of 1e-8. One step = one such solve.

value: sustained Dslash GFLOP/s inside the solve, counting MILC's 1146 flops
per output site for every Dslash application the solve performs (Krylov
loop, reliable updates, initial residual); whole-job over all ranks.
Also reported: the plain FP64 GPU CG time to the same residual, the
Dslash-only HBM roofline of the dominant kernel (FP32 Dslash), an end-to-end
number through the C ABI with host buffers, and the FP64 CPU oracle timed on
the host cores on a bounded sample of the same workload.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Dslash GFLOP/s & HBM-roofline frac; CG time to 1e-8 residual vs plain FP64 CG"
UNIT = "GFLOP/s"
FLOPS_PER_SITE = 1146
LATTICE = (32, 32, 32, 32)
MASS = 0.01
TOL = 1e-8
GAUGE_SEED = 1002   # 1000 + workload number (the 32^4 single-mass case is the second)
SOURCE_SEED = 2200  # 2000 + 100 * workload number + rhs
# least bytes per output site (each link once, input once, output once): 16 links + 2 vectors
BYTES_PER_SITE = {"f64": 16 * 144 + 2 * 48, "f32": 16 * 72 + 2 * 24, "f32_recon12": 8 * 72 + 8 * 48 + 2 * 24}
FALLBACK_HBM_GBS = 6800.0

# DRAM bytes per launch of the FP32 Dslash measured by ncu, with the hash of
# the kernel sources they were taken on (null once the sources change).
NCU_TRAFFIC = {"sources_sha256": None, "bytes_per_launch": None, "lattice": None}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true", help="skip the oracle timing (profiling runs)")
    ap.add_argument("--dslash-only", action="store_true", help="only the Dslash roofline loop (profiling runs)")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# ranks (replicas only: no data exchange; the process group is used for the
# barrier and the max-over-ranks timing)
# ---------------------------------------------------------------------------
class Ranks:
    def __init__(self):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.dist = None
        if self.world > 1:
            import torch
            import torch.distributed as dist

            backend = "nccl" if torch.cuda.is_available() else "gloo"
            dist.init_process_group(backend)
            self.dist = dist
            self.backend = backend

    def barrier(self):
        if self.dist:
            self.dist.barrier()

    def _reduce(self, v: float, op) -> float:
        if not self.dist:
            return v
        import torch

        dev = "cuda" if self.backend == "nccl" else "cpu"
        t = torch.tensor([v], dtype=torch.float64, device=dev)
        self.dist.all_reduce(t, op=op)
        return float(t.item())

    def max(self, v: float) -> float:
        return self._reduce(v, self.dist.ReduceOp.MAX) if self.dist else v

    def sum(self, v: float) -> float:
        return self._reduce(v, self.dist.ReduceOp.SUM) if self.dist else v

    def close(self):
        if self.dist:
            self.dist.destroy_process_group()


def whole_job_rate(flops_per_rank: float, seconds_per_rank: float, ranks: Ranks) -> tuple[float, float]:
    """(GFLOP/s over all ranks, max seconds): total work / slowest rank's time."""
    total = ranks.sum(flops_per_rank)
    tmax = ranks.max(seconds_per_rank)
    return total / tmax / 1e9, tmax


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid: str | None):
        self.uuid = (uuid or "").replace("GPU-", "")
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        rows = [[c.strip() for c in ln.split(",")] for ln in out.strip().splitlines() if ln.count(",") >= 8]
        mine = [r for r in rows if self.uuid and self.uuid in r[0]] or rows
        if not mine:
            return None
        sm = [float(r[1]) for r in mine if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in mine if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in mine for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(mine)}


def hbm_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def sources_sha256() -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1611_00728_gb300", "csrc")
    for name in sorted(os.listdir(csrc)):
        if name.endswith((".cu", ".cuh")):
            with open(os.path.join(csrc, name), "rb") as f:
                h.update(name.encode() + f.read())
    return h.hexdigest()


def workload_config():
    return {"workload": "32^4 single-mass CG, m=0.01, mixed FP32/FP64 with reliable updates, to true rel. residual 1e-8",
            "lattice": list(LATTICE), "mass": MASS, "tol": TOL, "flops_per_site": FLOPS_PER_SITE,
            "links": "random SU(3) width 0.3 (seed 1002): fat 0.9 W, long -1/24 W W W; antiperiodic t",
            "source": "Gaussian complex colour vector on even sites (seed 2200)",
            "l2": "inputs larger than L2 (FP32 links 0.6 GB + FP64 links 1.2 GB)",
            "parallelism": "replicas (one independent solve per GPU)"}


# ---------------------------------------------------------------------------
# oracle timing (CPU)
# ---------------------------------------------------------------------------
def oracle_sample(fat, lng, b, budget_s: float = 15.0):
    """Time the FP64 oracle CG on a bounded number of iterations of the same workload."""
    import oracle

    Vh = b.shape[0]
    sigma = 4 * MASS * MASS
    t0 = time.perf_counter()
    oracle.normal_op(LATTICE, fat, lng, sigma, b)
    t_a = time.perf_counter() - t0
    iters = int(max(1, min(50, budget_s / max(t_a, 1e-3) - 2)))
    t0 = time.perf_counter()
    _, it, _ = oracle.cg(LATTICE, fat, lng, sigma, b, tol=1e-300, max_iter=iters)
    dt = time.perf_counter() - t0
    apps = 2 * (iters + 2)  # initial residual + iterations + final true residual
    return {"value": FLOPS_PER_SITE * Vh * apps / dt / 1e9, "unit": UNIT, "cores": oracle.max_threads(),
            "kind": "oracle", "seconds": dt,
            "sample": f"oracle CG on the 32^4 workload, {iters} iterations + initial and final residual "
                      f"({apps} Dslash applications), OpenMP over sites"}


def cpu_info():
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True).stdout
        for ln in out.splitlines():
            if ln.startswith("Model name"):
                model = ln.split(":", 1)[1].strip()
    except Exception:
        pass
    return {"nproc": os.cpu_count(), "model": model}


def run_reference(args, ranks: Ranks):
    """The reference arm: the FP64 CPU oracle, as it stands, on the host cores."""
    if ranks.rank != 0:
        return
    import oracle
    import synth

    oracle.build()
    fat, lng = synth.fat_long_links(LATTICE, GAUGE_SEED)
    b = synth.gaussian_source(LATTICE, SOURCE_SEED)
    Vh = b.shape[0]
    sigma = 4 * MASS * MASS
    iters = 1
    apps = 2 * (iters + 2)

    def step():
        oracle.cg(LATTICE, fat, lng, sigma, b, tol=1e-300, max_iter=iters)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = (time.perf_counter() - t0) / args.steps
    value = FLOPS_PER_SITE * Vh * apps / dt / 1e9
    cores = oracle.max_threads()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(),
            "cpu_baseline": {"kind": "oracle", "cores": cores, "value": value, "unit": UNIT,
                             "sample": f"each step: oracle CG on the 32^4 workload, {iters} iteration + initial "
                                       f"and final residual ({apps} Dslash applications), OpenMP over sites"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "cpu": cpu_info()}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def time_dslash(torch, lat, sq, prec, reps):
    """Average duration of one Dslash launch (CUDA events on the launching stream)."""
    a = lat.new_spinor(prec)
    b = lat.new_spinor(prec)
    a.normal_()
    for _ in range(3):
        lat.dslash(1, a, b, prec)
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(s)
    for _ in range(reps):
        lat.dslash(1, a, b, prec)
    e1.record(s)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps / 1e3


def run_ours(args, ranks: Ranks):
    import torch

    import paper_1611_00728_gb300 as sq
    from paper_1611_00728_gb300 import build as _build
    import synth

    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    torch.cuda.set_device(ranks.local)
    _build.build()
    Vh = int(np.prod(LATTICE)) // 2
    fat, lng = synth.fat_long_links(LATTICE, GAUGE_SEED)
    b_host = synth.gaussian_source(LATTICE, SOURCE_SEED)
    lat = sq.Lattice(LATTICE)
    lat.load_links(fat, lng)
    peak, peak_kind = hbm_peak()

    if args.dslash_only:
        t = time_dslash(torch, lat, sq, sq.F32, 20)
        print(json.dumps({"dslash_f32_ms": t * 1e3}), flush=True)
        return

    b = lat.pack(b_host)
    x = lat.new_spinor()

    def solve(mode):
        x.zero_()
        return lat.cg_solve(MASS, b, x, tol=TOL, max_iter=20000, mode=mode)

    for _ in range(max(args.warmup, 0)):
        solve(sq.MODE_MIXED)
    torch.cuda.synchronize()

    uuid = None
    try:
        uuid = str(torch.cuda.get_device_properties(ranks.local).uuid)
    except Exception:
        pass
    clocks = ClockSampler(uuid)
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ranks.barrier()
    torch.cuda.synchronize()
    clocks.start()
    e0.record(s)
    infos = [solve(sq.MODE_MIXED) for _ in range(args.steps)]
    e1.record(s)
    torch.cuda.synchronize()
    ranks.barrier()
    clk = clocks.stop()
    t_step = e0.elapsed_time(e1) / 1e3 / args.steps
    apps = [2 * (i.iters + i.reliable_updates + 1) for i in infos]
    flops_step = FLOPS_PER_SITE * Vh * statistics.mean(apps)
    value, t_max = whole_job_rate(flops_step, t_step, ranks)
    res_mixed = max(i.true_rel_resid for i in infos)
    launches = sum(i.launches for i in infos)
    mixed_info = {"ms": t_step * 1e3, "iters": infos[-1].iters, "reliable_updates": infos[-1].reliable_updates,
                  "true_rel_resid": res_mixed, "dslash_applications": apps[-1]}

    # plain FP64 GPU CG to the same residual (time to solution)
    torch.cuda.synchronize()
    e0.record(s)
    info64 = solve(sq.MODE_F64)
    e1.record(s)
    torch.cuda.synchronize()
    t64 = e0.elapsed_time(e1) / 1e3
    apps64 = 2 * (info64.iters + info64.reliable_updates + 1)
    fp64_info = {"ms": t64 * 1e3, "iters": info64.iters, "true_rel_resid": info64.true_rel_resid,
                 "dslash_gflops": FLOPS_PER_SITE * Vh * apps64 / t64 / 1e9}

    # Dslash-only roofline of the dominant kernel (FP32 Dslash) and the other variants
    t32 = time_dslash(torch, lat, sq, sq.F32, 50)
    t64d = time_dslash(torch, lat, sq, sq.F64, 20)
    lat_r = sq.Lattice(LATTICE)
    lat_r.load_links(fat, lng, recon12=True)
    t32r = time_dslash(torch, lat_r, sq, sq.F32, 50)
    lat_r.close()
    ach = BYTES_PER_SITE["f32"] * Vh / t32 / 1e9
    traffic = None
    if NCU_TRAFFIC["sources_sha256"] == sources_sha256() and NCU_TRAFFIC["lattice"] == list(LATTICE):
        traffic = NCU_TRAFFIC["bytes_per_launch"]
    roofline = {"bound": "hbm", "kernel": "k_dslash<float> (FP32 Dslash, full links)", "achieved": ach,
                "peak": peak, "unit": "GB/s", "frac": ach / peak, "peak_kind": f"{peak_kind} (copy bandwidth)",
                "traffic": traffic, "algorithmic_bytes_per_launch": BYTES_PER_SITE["f32"] * Vh,
                "ms_per_launch": t32 * 1e3}
    dslash = {"f32": {"ms": t32 * 1e3, "gflops": FLOPS_PER_SITE * Vh / t32 / 1e9,
                      "gbs": ach, "frac_hbm": ach / peak},
              "f32_recon12": {"ms": t32r * 1e3, "gflops": FLOPS_PER_SITE * Vh / t32r / 1e9,
                              "gbs": BYTES_PER_SITE["f32_recon12"] * Vh / t32r / 1e9,
                              "frac_hbm": BYTES_PER_SITE["f32_recon12"] * Vh / t32r / 1e9 / peak},
              "f64": {"ms": t64d * 1e3, "gflops": FLOPS_PER_SITE * Vh / t64d / 1e9,
                      "gbs": BYTES_PER_SITE["f64"] * Vh / t64d / 1e9,
                      "frac_hbm": BYTES_PER_SITE["f64"] * Vh / t64d / 1e9 / peak}}

    # end to end through the C ABI with host buffers: H2D of b, solve, D2H of x
    b_pin = torch.from_numpy(b_host.view(np.float64)).pin_memory()
    x_pin = torch.empty_like(b_pin).pin_memory()
    b_pin_np = b_pin.numpy().view(np.complex128)
    x_pin_np = x_pin.numpy().view(np.complex128)
    torch.cuda.synchronize()
    ranks.barrier()
    t0 = time.perf_counter()
    e2e_apps = []
    for _ in range(args.steps):
        lat.pack(b_pin_np, sq.F64, out=b)
        x.zero_()
        i = lat.cg_solve(MASS, b, x, tol=TOL, max_iter=20000, mode=sq.MODE_MIXED)
        lat.unpack(x, sq.F64, out=x_pin_np)
        e2e_apps.append(2 * (i.iters + i.reliable_updates + 1))
    torch.cuda.synchronize()
    t_e2e = (time.perf_counter() - t0) / args.steps
    e2e_value, _ = whole_job_rate(FLOPS_PER_SITE * Vh * statistics.mean(e2e_apps), t_e2e, ranks)
    e2e = {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(b_host.nbytes),
           "d2h_bytes_per_step": int(b_host.nbytes), "ms_per_step": t_e2e * 1e3}

    cpu = None
    if ranks.rank == 0 and ranks.world == 1 and not args.no_cpu_baseline:
        cpu = oracle_sample(fat, lng, b_host)
    lat.close()
    if ranks.rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ranks.world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": t_max * 1e3, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": workload_config(),
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
                "clocks": clk, "cg_mixed": mixed_info, "cg_fp64": fp64_info,
                "speedup_vs_fp64_cg": t64 / t_step, "dslash": dslash, "cpu": cpu_info(),
                "notes": "dtype f32: FP32 Dslash and Krylov vectors; FP64 x, reductions, scalar recurrences and "
                         "reliable updates. Roofline: Dslash-only loop timed with CUDA events in this run."}
        print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.steps < 1:
        raise SystemExit("--steps must be >= 1")
    ranks = Ranks()
    try:
        if args.impl == "reference":
            run_reference(args, ranks)
        else:
            run_ours(args, ranks)
    finally:
        ranks.close()


if __name__ == "__main__":
    main()
