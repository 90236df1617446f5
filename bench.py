#!/usr/bin/env python
"""Benchmark of the improved-staggered CG on one GB300 (or N replicas).

Workload: the single-mass 32^4 lattice, m = 0.01, seeded random fat/long
links (fat = 0.9 SU(3), long = -1/24 times a product of three SU(3)),
antiperiodic time, one Gaussian source; the mixed-precision CG (FP32 Dslash
and vectors, float-float sums, FP64 x, scalars and true residuals) solved from x0 = 0 to
a true relative residual of 1e-8. One step = one such solve.

value: sustained Dslash GFLOP/s inside the solve, counting MILC's 1146 flops
per output site for every Dslash application the solve performs (Krylov
loop and FP64 reliable updates; from x0 = 0 the initial residual is b itself);
whole-job over all ranks.
Also reported: the plain FP64 GPU CG time to the same residual, the
Dslash-only HBM roofline of the dominant kernel (FP32 Dslash), an end-to-end
number through the C ABI with host buffers, the FP64 CPU oracle timed on
the host cores on a bounded sample of the same workload, and (one GPU) a
`forms` block: the multi-shift, rational, batched, learned and HISQ-link
forms of the solve, each against plain FP64 GPU CG at the same residual,
each with its own clock record.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""

from __future__ import annotations

import argparse
import contextlib
import datetime
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
# the paper's own figures (Sec. 4), other hardware and FP64 multi-mass CG: context, not targets
PAPER_CONTEXT = {"milc_multimass_cg_one_knl7250_gflops": 65, "qphix_speedup_one_knl": 1.5,
                 "qphix_multimass_cg_16_knl7210_gflops": 900,
                 "qphix_dslash_fraction_of_knl_read_bandwidth": 0.8, "precision": "FP64"}
# The HISQ construction runs its 3x3 products in float-float arithmetic on the FP32 pipe. A counted complex
# multiply-add (8 flops) executes as four float-float accumulations (TwoProduct and TwoSum: 10 FP32
# instructions each) plus a share of 2 for the renormalisation after every three: 42 FP32 instructions.
# The FP32 pipe issues 128 lanes per SM and clock: 152 SMs at 2.07 GHz (nominal unit counts and clock).
FF_INSTR_PER_COUNTED_CFMA = 42
HISQ_FF_ALU_PEAK_GFLOPS = 128 * 152 * 2.07e9 / FF_INSTR_PER_COUNTED_CFMA * 8 / 1e9

# DRAM bytes per launch (read + write) of the FP32 Dslash with 12-real long links
# at 32^4, measured by ncu (profiles/dslash_f32_recon12_32x32x32x32.md), with the
# hash of the kernel sources they were taken on (reported as null once those change).
NCU_TRAFFIC = {"sources_sha256": "c601c38d9faf1a218dcd10ebf5bedbfed27590c1b8a899eeb479301e9383c0bc",
               "bytes_per_launch": 525900000 + 11370000, "lattice": [32, 32, 32, 32]}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true", help="skip the oracle timing (profiling runs)")
    ap.add_argument("--dslash-only", action="store_true", help="only the Dslash roofline loop (profiling runs)")
    ap.add_argument("--links", choices=["recon12", "full", "8way", "8way-recon12", "ff", "f64"], default="recon12",
                    help="--dslash-only: the FP32 link storage to time (default: 12-real long links, as the solvers), "
                         "or the float-float (ff) or FP64 (f64) Dslash")
    ap.add_argument("--lattice", default=None,
                    help="hisq and batched workloads: extents as Lx,Ly,Lz,Lt (hisq default 32^4; batched: one "
                         "lattice with 16 sources instead of the three; for profiling)")
    ap.add_argument("--pin", default=None,
                    help="batched: pin the FP32 Dslash configuration W,WT,T,carve,warp_sites instead of tuning "
                         "(for profiling runs)")
    ap.add_argument("--save-params", default=None, help="learned: write the trained network parameters (.npy)")
    ap.add_argument("--load-params", default=None, help="learned: skip training, use these parameters (.npy)")
    ap.add_argument("--no-forms", action="store_true",
                    help="default workload: skip the forms block (multi-shift, rational, batched, learned, HISQ)")
    ap.add_argument("--no-compare", action="store_true",
                    help="batched, multishift, learned: skip the FP64 and mixed comparison solves (profiling runs)")
    ap.add_argument("--workload", choices=["single", "multishift", "rational", "batched", "learned", "hisq"], default="single",
                    help="single (default): the 32^4 single-mass solve; the others print their own line")
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
    """nvidia-smi samples every 50 ms, started before the warm-up (so that the tool is
    running when a timed region begins) and filtered to the timed regions by their
    timestamps (host clock of the same machine). Timed regions are tagged, so one
    sampler serves the main solve and each form of the `forms` block."""
    FIELDS = ("timestamp,uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    REASONS = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")

    def __init__(self, uuid: str | None):
        self.uuid = (uuid or "").replace("GPU-", "")
        self.proc = None
        self.windows = []  # (tag, t0, t1)
        self.rows = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    @contextlib.contextmanager
    def timed(self, tag: str):
        t0 = datetime.datetime.now()
        try:
            yield
        finally:
            self.windows.append((tag, t0, datetime.datetime.now()))

    @staticmethod
    def _when(ts: str):
        try:
            return datetime.datetime.strptime(ts, "%Y/%m/%d %H:%M:%S.%f")
        except ValueError:
            return None

    def stop(self):
        if not self.proc:
            self.rows = []
            return self
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        rows = [[c.strip() for c in ln.split(",")] for ln in out.strip().splitlines() if ln.count(",") >= 9]
        mine = [r for r in rows if self.uuid and self.uuid in r[1]] or rows
        self.rows = [(self._when(r[0]), r[1:]) for r in mine]
        return self

    def summary(self, prefix: str = ""):
        """Clock record of the timed regions whose tag starts with prefix (median SM clock under load,
        maximum clock, throttle reasons seen, sample count); None without samples."""
        if self.rows is None:
            self.stop()
        wins = [(a, b) for tag, a, b in self.windows if tag.startswith(prefix)]
        inside = [r for w, r in self.rows if w is not None and any(a <= w <= b for a, b in wins)]
        if not inside:
            return None
        sm = [float(r[1]) for r in inside if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in inside if r[2].replace(".", "").isdigit()]
        reasons = sorted({self.REASONS[k] for r in inside for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(inside)}


def gpu_uuid(torch, dev: int):
    try:
        return str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        return None


def hbm_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


DSLASH_SOURCES = ("dslash_core.cuh", "dslash.cu", "solver_device.cuh", "sqcg_internal.cuh")  # what k_dslash is compiled from


def sources_sha256() -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1611_00728_gb300", "csrc")
    for name in DSLASH_SOURCES:
        with open(os.path.join(csrc, name), "rb") as f:
            h.update(name.encode() + f.read())
    return h.hexdigest()


def workload_config():
    return {"workload": "32^4 single-mass CG, m=0.01, mixed FP32/FP64 with reliable updates, to true rel. residual 1e-8",
            "lattice": list(LATTICE), "mass": MASS, "tol": TOL, "flops_per_site": FLOPS_PER_SITE,
            "links": "random SU(3) width 0.3 (seed 1002): fat 0.9 W, long -1/24 W W W; antiperiodic t; "
                     "FP32 long links in 12-real form (accepted by the library's unitarity test)",
            "source": "Gaussian complex colour vector on even sites (seed 2200)",
            "l2": "inputs larger than L2 (FP32 links 0.5 GB + FP64 links 1.2 GB)",
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
                      f"({apps} Dslash applications), OpenMP over sites",
            "dslash": oracle_dslash_rates(fat, lng)}


def oracle_dslash_rates(fat32, lng32, reps: int = 3):
    """The oracle Dslash alone, single-threaded and on all host cores, at 8^4 and at 32^4 (median of reps)."""
    import oracle
    import synth

    out = {}
    for L in ((8, 8, 8, 8), LATTICE):
        if L == LATTICE:
            fat, lng = fat32, lng32
        else:
            fat, lng = synth.fat_long_links(L, 1001)
        psi = synth.gaussian_source(L, 2001)
        Vh = int(np.prod(L)) // 2
        row = {}
        for name, nt in (("single_thread", 1), ("all_cores", oracle.max_threads())):
            ts = []
            for _ in range(reps):
                t0 = time.perf_counter()
                oracle.dslash(L, fat, lng, psi, 1, nthreads=nt)
                ts.append(time.perf_counter() - t0)
            row[name + "_gflops"] = FLOPS_PER_SITE * Vh / statistics.median(ts) / 1e9
        row["cores"] = oracle.max_threads()
        out["x".join(map(str, L))] = row
    return out


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
    # the long links are s * SU(3) with one global s, so the library accepts their
    # 12-real form (it checks); the FP32 copy is stored that way, FP64 stays full
    lat.load_links(fat, lng, recon12=True)
    peak, peak_kind = hbm_peak()

    if args.dslash_only:
        if args.links in ("ff", "f64"):
            t = time_dslash(torch, lat, sq, sq.FF if args.links == "ff" else sq.F64, 20)
            print(json.dumps({f"dslash_{args.links}_ms": t * 1e3,
                              "gbs": BYTES_PER_SITE["f64"] * Vh / t / 1e9}), flush=True)
            return
        if args.links != "recon12":
            lat.close()
            lat = sq.Lattice(LATTICE)
            lat.load_links(fat, lng, recon12=args.links.endswith("recon12"), eight_way=args.links.startswith("8way"))
        t = time_dslash(torch, lat, sq, sq.F32, 20)
        print(json.dumps({f"dslash_f32_{args.links}_ms": t * 1e3}), flush=True)
        return

    b = lat.pack(b_host)
    x = lat.new_spinor()

    def solve(mode):
        x.zero_()
        return lat.cg_solve(MASS, b, x, tol=TOL, max_iter=20000, mode=mode)

    clocks = ClockSampler(gpu_uuid(torch, ranks.local)).start()
    for _ in range(max(args.warmup, 0)):
        solve(sq.MODE_MIXED)
    torch.cuda.synchronize()

    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ranks.barrier()
    torch.cuda.synchronize()
    with clocks.timed("main"):
        e0.record(s)
        infos = [solve(sq.MODE_MIXED) for _ in range(args.steps)]
        e1.record(s)
        torch.cuda.synchronize()
    ranks.barrier()
    t_step = e0.elapsed_time(e1) / 1e3 / args.steps
    # Dslash applications: 2 per iteration and 2 per FP64 reliable update (the last one is the convergence
    # check); from x0 = 0 the initial residual is b itself, with no operator application
    apps = [2 * (i.iters + i.reliable_updates) for i in infos]
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
    apps64 = 2 * (info64.iters + info64.reliable_updates)
    fp64_info = {"ms": t64 * 1e3, "iters": info64.iters, "true_rel_resid": info64.true_rel_resid,
                 "dslash_gflops": FLOPS_PER_SITE * Vh * apps64 / t64 / 1e9}

    # Dslash-only roofline of the dominant kernel (the FP32 Dslash with 12-real long
    # links, as the solve uses it) and the other variants
    t32r = time_dslash(torch, lat, sq, sq.F32, 50)
    t64d = time_dslash(torch, lat, sq, sq.F64, 20)
    tffd = time_dslash(torch, lat, sq, sq.FF, 20)
    lat_f = sq.Lattice(LATTICE)
    lat_f.load_links(fat, lng)
    t32 = time_dslash(torch, lat_f, sq, sq.F32, 50)
    lat_f.close()
    # 8-way storage of the FP32 links (backward links at the site that uses them)
    t8 = {}
    for rc in (False, True):
        lat8 = sq.Lattice(LATTICE)
        lat8.load_links(fat, lng, recon12=rc, eight_way=True)
        t8[rc] = time_dslash(torch, lat8, sq, sq.F32, 50)
        lat8.close()
    ach = BYTES_PER_SITE["f32_recon12"] * Vh / t32r / 1e9
    traffic = None
    if NCU_TRAFFIC["sources_sha256"] == sources_sha256() and NCU_TRAFFIC["lattice"] == list(LATTICE):
        traffic = NCU_TRAFFIC["bytes_per_launch"]
    roofline = {"bound": "hbm", "kernel": "k_dslash<float, float, 1, 0, 0> (FP32 Dslash, 12-real long links)",
                "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                "peak_kind": f"{peak_kind} (copy bandwidth)", "traffic": traffic,
                "algorithmic_bytes_per_launch": BYTES_PER_SITE["f32_recon12"] * Vh, "ms_per_launch": t32r * 1e3}
    dslash = {"f32": {"ms": t32 * 1e3, "gflops": FLOPS_PER_SITE * Vh / t32 / 1e9,
                      "gbs": BYTES_PER_SITE["f32"] * Vh / t32 / 1e9,
                      "frac_hbm": BYTES_PER_SITE["f32"] * Vh / t32 / 1e9 / peak},
              "f32_recon12": {"ms": t32r * 1e3, "gflops": FLOPS_PER_SITE * Vh / t32r / 1e9,
                              "gbs": BYTES_PER_SITE["f32_recon12"] * Vh / t32r / 1e9,
                              "frac_hbm": BYTES_PER_SITE["f32_recon12"] * Vh / t32r / 1e9 / peak},
              "f32_8way": {"ms": t8[False] * 1e3, "gflops": FLOPS_PER_SITE * Vh / t8[False] / 1e9,
                           "gbs": BYTES_PER_SITE["f32"] * Vh / t8[False] / 1e9,
                           "frac_hbm": BYTES_PER_SITE["f32"] * Vh / t8[False] / 1e9 / peak},
              "f32_8way_recon12": {"ms": t8[True] * 1e3, "gflops": FLOPS_PER_SITE * Vh / t8[True] / 1e9,
                                   "gbs": BYTES_PER_SITE["f32_recon12"] * Vh / t8[True] / 1e9,
                                   "frac_hbm": BYTES_PER_SITE["f32_recon12"] * Vh / t8[True] / 1e9 / peak},
              "f64": {"ms": t64d * 1e3, "gflops": FLOPS_PER_SITE * Vh / t64d / 1e9,
                      "gbs": BYTES_PER_SITE["f64"] * Vh / t64d / 1e9,
                      "frac_hbm": BYTES_PER_SITE["f64"] * Vh / t64d / 1e9 / peak},
              "ff": {"ms": tffd * 1e3, "gflops": FLOPS_PER_SITE * Vh / tffd / 1e9,
                     "gbs": BYTES_PER_SITE["f64"] * Vh / tffd / 1e9,
                     "frac_hbm": BYTES_PER_SITE["f64"] * Vh / tffd / 1e9 / peak,
                     "note": "float-float (hi + lo floats per real) Dslash of the reliable updates; FP64 bytes"}}

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
        e2e_apps.append(2 * (i.iters + i.reliable_updates))
    torch.cuda.synchronize()
    t_e2e = (time.perf_counter() - t0) / args.steps
    e2e_value, _ = whole_job_rate(FLOPS_PER_SITE * Vh * statistics.mean(e2e_apps), t_e2e, ranks)
    e2e = {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(b_host.nbytes),
           "d2h_bytes_per_step": int(b_host.nbytes), "ms_per_step": t_e2e * 1e3}

    lat.close()
    del lat, b, x, lat_f
    forms = None
    if ranks.world == 1 and not args.no_forms:
        forms = run_forms(torch, sq, clocks)
    clocks.stop()
    clk = clocks.summary("main")
    if forms:
        for name, rec in forms.items():
            if "unavailable" not in rec:
                rec["clocks"] = clocks.summary(name)
    cpu = None
    if ranks.rank == 0 and ranks.world == 1 and not args.no_cpu_baseline:
        cpu = oracle_sample(fat, lng, b_host)
    if ranks.rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ranks.world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": t_max * 1e3, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": workload_config(),
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
                "clocks": clk, "cg_mixed": mixed_info, "cg_fp64": fp64_info, "forms": forms,
                "speedup_vs_fp64_cg": t64 / t_step, "dslash": dslash, "cpu": cpu_info(),
                "dslash_gpu_vs_oracle": None if cpu is None else {
                    "gpu_f32_recon12_gflops": dslash["f32_recon12"]["gflops"], "gpu_f64_gflops": dslash["f64"]["gflops"],
                    "vs_single_thread_32^4": dslash["f32_recon12"]["gflops"]
                    / cpu["dslash"]["x".join(map(str, LATTICE))]["single_thread_gflops"],
                    "vs_all_cores_32^4": dslash["f32_recon12"]["gflops"]
                    / cpu["dslash"]["x".join(map(str, LATTICE))]["all_cores_gflops"]},
                "paper_context": PAPER_CONTEXT,
                "notes": "dtype f32: FP32 Dslash and Krylov vectors; float-float grid sums; FP64 x, scalar "
                         "recurrences and reliable-update residuals (float-float Dslash, FP64 sum). Roofline: "
                         "Dslash-only loop timed with CUDA events in this run."}
        print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# other forms of the solve, each against plain FP64 GPU CG at the same residual
# ---------------------------------------------------------------------------
def _timed(torch, fn):
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s = torch.cuda.current_stream()
    e0.record(s)
    out = fn()
    e1.record(s)
    torch.cuda.synchronize()
    return out, e0.elapsed_time(e1)


def _repeat(torch, clk, tag, fn, steps):
    """steps timed calls of fn inside one clock window; (median ms, last result)."""
    times, out = [], None
    with clk.timed(tag):
        for _ in range(steps):
            out, ms = _timed(torch, fn)
            times.append(ms)
    return statistics.median(times), out


def _solve_sigma(lat, sigma, b, x, sq, mode=None):
    """CG of (sigma - D_eo D_oe) x = b (mass = sqrt(sigma) / 2), plain FP64 unless mode says otherwise."""
    x.zero_()
    return lat.cg_solve(float(np.sqrt(sigma) / 2), b, x, tol=TOL, max_iter=20000,
                        mode=sq.MODE_F64 if mode is None else mode)


MS_SEEDS = (1003, 2300)  # gauge, source of the multi-shift workload (third configuration)
MS_SHIFTS = tuple(float(v) for v in np.logspace(-4, 0, 11))


def measure_multishift(torch, sq, clk, lat, b, steps, compare=True, tag="multishift"):
    """Mixed multi-shift (11 shifts) against the FP64 multi-shift and plain FP64 CG one shift at a time."""
    shifts = list(MS_SHIFTS)
    xs = [lat.new_spinor() for _ in shifts]
    res = {}
    modes = (("mixed", sq.MODE_MIXED),) + ((("fp64_multishift", sq.MODE_F64),) if compare else ())
    for name, mode in modes:
        def run(mode=mode):
            return lat.multishift_cg_solve(shifts, b, xs, tol=TOL, max_iter=20000, mode=mode)
        run()
        ms, infos = _repeat(torch, clk, f"{tag}.{name}", run, steps if name == "mixed" else 1)
        res[name] = {"ms": ms, "iters": [i.iters for i in infos],
                     "max_true_rel_resid": max(i.true_rel_resid for i in infos)}
        if name == "mixed":  # the batched refinement's tuned Dslash configuration (its plan stays with lat)
            res[name]["base_reliable_updates"] = len(lat.multishift_ru_record())
            res[name]["refinement_tuning"] = sq.batched_tuning_ex(lat)
    # the same mixed solve with shift-aware reliable updates: at each base update every shift still
    # iterating gets its FP64 true residual and its collinearity loss |r_s - zeta'_s r_0| / |b|; a shift
    # continues from the fitted zeta'_s only where that loss is at most tol / 2
    def run_ru():
        return lat.multishift_cg_solve(shifts, b, xs, tol=TOL, max_iter=20000, mode=sq.MODE_MIXED | sq.MS_SHIFT_RU)
    run_ru()
    ms, infos = _repeat(torch, clk, f"{tag}.mixed_shift_aware", run_ru, steps)
    rec = lat.multishift_ru_record()
    base = int(np.argmin(shifts))
    res["mixed_shift_aware"] = {
        "ms": ms, "iters": [i.iters for i in infos], "max_true_rel_resid": max(i.true_rel_resid for i in infos),
        "updates": [{"iter": it, "base_rel_resid": r0,
                     "loss_over_b": [None if np.isnan(v) else v for v in loss],
                     "shifts_continuing": sum(1 for j, v in enumerate(loss) if j != base and v <= 0.5 * TOL),
                     "shifts_iterating": sum(1 for j, v in enumerate(loss) if j != base and not np.isnan(v))}
                    for it, r0, loss in rec]}
    # the shared loop without the mixed mode's base reliable updates
    def run_no_ru():
        return lat.multishift_cg_solve(shifts, b, xs, tol=TOL, max_iter=20000, mode=sq.MODE_MIXED | sq.MS_NO_RU)
    run_no_ru()
    ms, infos = _repeat(torch, clk, f"{tag}.mixed_no_ru", run_no_ru, steps)
    res["mixed_no_ru"] = {"ms": ms, "iters": [i.iters for i in infos],
                          "max_true_rel_resid": max(i.true_rel_resid for i in infos)}
    if compare:  # plain FP64 CG, one solve per shift (the same buffers: one captured graph)
        x = lat.new_spinor()
        _solve_sigma(lat, shifts[0], b, x, sq)
        total, iters = 0.0, []
        with clk.timed(f"{tag}.fp64_cg"):
            for sg in shifts:
                info, ms = _timed(torch, lambda sg=sg: _solve_sigma(lat, sg, b, x, sq))
                total += ms
                iters.append(info.iters)
        res["fp64_cg_one_per_shift"] = {"ms": total, "iters": iters}
        res["speedup_vs_fp64_cg_one_per_shift"] = total / res["mixed"]["ms"]
        res["speedup_vs_fp64_multishift"] = res["fp64_multishift"]["ms"] / res["mixed"]["ms"]
    return res


def measure_rational(torch, sq, clk, lat, b, steps, tag="rational"):
    """12-pole rational approximation of (4m^2 - D_eo D_oe)^(-1/2) applied to b (m = 0.01), mixed vs FP64."""
    m = 0.01
    a0, a, beta = synth_rational(m)
    shifts = 4 * m * m + beta
    out = lat.new_spinor()
    res = {"shifts": [float(v) for v in shifts]}
    for name, mode in (("mixed", sq.MODE_MIXED), ("fp64", sq.MODE_F64)):
        def run(mode=mode):
            return lat.rational_apply(shifts, a, a0, b, out, tol=TOL, max_iter=20000, mode=mode)
        run()
        ms, infos = _repeat(torch, clk, f"{tag}.{name}", run, steps if name == "mixed" else 1)
        res[name] = {"ms": ms, "iters": max(i.iters for i in infos),
                     "max_true_rel_resid": max(i.true_rel_resid for i in infos)}
    res["speedup_vs_fp64"] = res["fp64"]["ms"] / res["mixed"]["ms"]
    return res


def synth_rational(m):
    import synth

    return synth.inverse_sqrt_rational(12, 4 * m * m, 16.0)


BATCHED_SPECS = ((16, 16, 16, 16), (24, 24, 24, 24), (32, 32, 32, 64))


def make_batched(sq, torch, specs, nr=16):
    import synth

    lats, bs, xs = [], [], []
    for n, L in enumerate(specs):
        fat, lng = synth.fat_long_links(L, 1004 + n)
        lat = sq.Lattice(L)
        lat.load_links(fat, lng, recon12=True)
        src = synth.gaussian_source(L, 2400 + 10 * n, nrhs=nr)
        b = torch.stack([lat.pack(v) for v in src]).contiguous()
        lats.append(lat); bs.append(b); xs.append(torch.zeros_like(b))
    return lats, bs, xs


def measure_batched(torch, sq, clk, lats, bs, xs, steps, compare=True, fp64_per_lattice=None, tag="batched"):
    """All RHS of all lattices in one batched solve (m = 0.02), against mixed CG and plain FP64 CG one source
    at a time. fp64_per_lattice: time plain FP64 CG on only the first sources of each lattice and scale the
    sum by nrhs / that count (None: every source)."""
    m = 0.02
    specs = [lat.dims for lat in lats]

    def solve():
        for x in xs:
            x.zero_()
        return sq.cg_solve_batched(lats, [m] * len(lats), bs, xs, tol=TOL, max_iter=20000)

    solve()  # tunes the batched Dslash on the first call
    t_batched, infos = _repeat(torch, clk, f"{tag}.batched", solve, steps)
    cfg = sq.batched_tuning_ex(lats[0])
    nr = int(bs[0].shape[0])
    res = {"ms": t_batched, "tuned": cfg, "nrhs_per_lattice": nr, "lattices": ["x".join(map(str, L)) for L in specs],
           "max_iters": max(i.iters for lst in infos for i in lst),
           "max_true_rel_resid": max(i.true_rel_resid for lst in infos for i in lst)}
    apps = sum(2 * (i.iters + i.reliable_updates) * int(np.prod(L)) // 2 for L, lst in zip(specs, infos) for i in lst)
    res["dslash_gflops_in_solve"] = FLOPS_PER_SITE * apps / (t_batched / 1e3) / 1e9
    if compare:
        t64, tmix, n64 = 0.0, 0.0, 0
        k64 = nr if fp64_per_lattice is None else min(nr, fp64_per_lattice)
        for lat, b in zip(lats, bs):
            x = lat.new_spinor()
            for mode in (sq.MODE_MIXED, sq.MODE_F64):  # capture each mode's graph once
                x.zero_()
                lat.cg_solve(m, b[0], x, tol=TOL, max_iter=20000, mode=mode)
            with clk.timed(f"{tag}.sequential"):
                for j in range(nr):
                    def run(mode, j=j):
                        x.zero_()
                        return lat.cg_solve(m, b[j], x, tol=TOL, max_iter=20000, mode=mode)

                    tmix += _timed(torch, lambda: run(sq.MODE_MIXED))[1]
                    if j < k64:
                        t64 += _timed(torch, lambda: run(sq.MODE_F64))[1]
                        n64 += 1
        scale = len(lats) * nr / n64
        res.update({"mixed_cg_one_per_source_ms": tmix, "fp64_cg_one_per_source_ms": t64 * scale,
                    "fp64_cg_sources_timed": n64, "fp64_cg_scaled_by": scale,
                    "speedup_vs_fp64_cg": t64 * scale / t_batched, "speedup_vs_mixed_cg_sequential": tmix / t_batched})
    return res


LEARNED_MASS = 0.005
LEARNED_HELD_OUT = (9000, 9100)  # gauge, source of the held-out evaluation
PARAMS_DIR = os.path.join(ROOT, "paper_1611_00728_gb300", "trained")
PARAMS_FILE = os.path.join(PARAMS_DIR, "fcg_network_16x16x16x16.npy")


def measure_learned(torch, sq, clk, L, params, steps, compare=True, tag="learned"):
    """Flexible CG with the network on the held-out gauge field, against plain FP64 and mixed CG at 1e-8."""
    import synth

    m = LEARNED_MASS
    fat, lng = synth.fat_long_links(L, LEARNED_HELD_OUT[0])
    lat = sq.Lattice(L)
    lat.load_links(fat, lng, recon12=True)
    net = sq.Network(lat)
    net.set_params(params)
    b = lat.pack(synth.gaussian_source(L, LEARNED_HELD_OUT[1]))
    x = lat.new_spinor()
    out = {}
    def fcg(mix):
        net.set_mixing(mix)
        return net.fcg_solve(m, b, x, tol=TOL, max_iter=50000)

    # the network's inference 8 -> 8 mixing in FP32 on the CUDA cores (default), and in BF16 on the tensor cores
    solvers = [("fcg_nn", lambda: fcg(sq.NN_MIX_FP32)), ("fcg_nn_bf16_mixing", lambda: fcg(sq.NN_MIX_BF16))]
    if compare:
        solvers += [("mixed_cg", lambda: lat.cg_solve(m, b, x, tol=TOL, max_iter=50000, mode=sq.MODE_MIXED)),
                    ("fp64_cg", lambda: lat.cg_solve(m, b, x, tol=TOL, max_iter=50000, mode=sq.MODE_F64))]
    for name, fn in solvers:
        def run(fn=fn):
            x.zero_()
            return fn()
        run()
        ms, info = _repeat(torch, clk, f"{tag}.{name}", run, steps if name != "fp64_cg" else 1)
        out[name] = {"ms": ms, "iters": info.iters, "true_rel_resid": info.true_rel_resid,
                     "fallback": getattr(info, "fallback", 0)}
    if compare:
        out["speedup_vs_fp64_cg"] = out["fp64_cg"]["ms"] / out["fcg_nn"]["ms"]
        out["speedup_vs_mixed_cg"] = out["mixed_cg"]["ms"] / out["fcg_nn"]["ms"]
        out["bf16_mixing_speedup_vs_mixed_cg"] = out["mixed_cg"]["ms"] / out["fcg_nn_bf16_mixing"]["ms"]
        out["bf16_mixing_speedup_vs_fp64_cg"] = out["fp64_cg"]["ms"] / out["fcg_nn_bf16_mixing"]["ms"]
    net.close()
    lat.close()
    return out


def measure_hisq(torch, sq, clk, lattice, steps, tag="hisq"):
    """HISQ link construction (device entry point), then mixed and FP64 CG on the HISQ links."""
    import synth

    V = int(np.prod(lattice))
    thin = synth.thin_links(lattice, GAUGE_SEED)
    d_thin = torch.from_numpy(thin.view(np.float64).reshape(-1)).cuda()
    d_fat, d_lng = torch.empty_like(d_thin), torch.empty_like(d_thin)
    ws = torch.empty(sq.hisq_workspace_bytes(lattice), dtype=torch.uint8, device="cuda")
    sq.hisq_smear(lattice, d_thin, d_fat, d_lng, ws)
    t_ms, _ = _repeat(torch, clk, f"{tag}.smear", lambda: sq.hisq_smear(lattice, d_thin, d_fat, d_lng, ws), steps)
    del d_fat, d_lng, ws
    gflops = V * 4 * sq.HISQ_FLOPS_PER_LINK / (t_ms / 1e3) / 1e9
    lat = sq.Lattice(lattice)
    lat.hisq_load_links(thin)
    b = lat.pack(synth.gaussian_source(lattice, SOURCE_SEED))
    x = lat.new_spinor()
    cg = {}
    for name, mode in (("mixed", sq.MODE_MIXED), ("fp64", sq.MODE_F64)):
        def solve(mode=mode):
            x.zero_()
            return lat.cg_solve(MASS, b, x, tol=TOL, max_iter=20000, mode=mode)
        solve()
        ms, info = _repeat(torch, clk, f"{tag}.cg_{name}", solve, steps if name == "mixed" else 1)
        cg[name] = {"ms": ms, "iters": info.iters, "true_rel_resid": info.true_rel_resid}
    lat.close()
    return {"smear_ms": t_ms, "smear_gflops": gflops, "smear_frac_of_ff_alu_peak": gflops / HISQ_FF_ALU_PEAK_GFLOPS,
            "cg_on_hisq_links": cg, "cg_speedup_mixed_vs_fp64": cg["fp64"]["ms"] / cg["mixed"]["ms"]}


def load_trained_params():
    """The committed network parameters and their training record (None, reason when absent)."""
    if not os.path.exists(PARAMS_FILE):
        return None, f"no trained parameters at {os.path.relpath(PARAMS_FILE, ROOT)}"
    rec = None
    side = PARAMS_FILE[:-4] + ".json"
    if os.path.exists(side):
        with open(side) as f:
            rec = json.load(f)
    return np.load(PARAMS_FILE).astype(np.float32), rec


def run_forms(torch, sq, clk):
    """The other forms of the solve, each against plain FP64 GPU CG at the same true residual 1e-8, in the
    default line (one GPU): mixed multi-shift, rational application, the batched 48-source solve, the learned
    flexible CG (committed parameters) and the CG on GPU-built HISQ links."""
    import synth

    forms = {}
    fat, lng = synth.fat_long_links(LATTICE, MS_SEEDS[0])
    lat = sq.Lattice(LATTICE)
    lat.load_links(fat, lng, recon12=True)
    b = lat.pack(synth.gaussian_source(LATTICE, MS_SEEDS[1]))
    del fat, lng
    forms["multishift"] = measure_multishift(torch, sq, clk, lat, b, 3)
    forms["multishift"]["config"] = "32^4, 11 shifts logspace(-4,0), seeds 1003/2300"
    forms["rational"] = measure_rational(torch, sq, clk, lat, b, 3)
    forms["rational"]["config"] = "32^4, m=0.01, 12 poles of x^(-1/2) on [4m^2, 16], seeds 1003/2300"
    lat.close()
    lats, bs, xs = make_batched(sq, torch, BATCHED_SPECS)
    forms["batched"] = measure_batched(torch, sq, clk, lats, bs, xs, 2, fp64_per_lattice=4)
    forms["batched"]["config"] = "16 sources each on 16^4, 24^4, 32^3x64, m=0.02 (gauge seeds 1004-1006)"
    for lat_ in lats:
        lat_.close()
    del lats, bs, xs
    params, rec = load_trained_params()
    if params is None:
        forms["learned"] = {"unavailable": rec}
    else:
        forms["learned"] = measure_learned(torch, sq, clk, LATTICE, params, 3)
        forms["learned"]["config"] = ("32^4, m=0.005, held-out gauge seed 9000, source 9100; network parameters "
                                      f"from {os.path.relpath(PARAMS_FILE, ROOT)}")
        if rec:
            forms["learned"]["training"] = {k: rec.get(k) for k in ("pairs", "schedule", "seconds_data",
                                                                     "seconds_train", "command")}
    forms["hisq"] = measure_hisq(torch, sq, clk, LATTICE, 3)
    forms["hisq"]["config"] = "32^4 thin links seed 1002 -> HISQ fat/long (FP64); CG m=0.01 on the result"
    torch.cuda.synchronize()
    return forms


def _workload_line(metric, value, args, config, clk, extra, dtype="f32", unit="ms", hib=False):
    line = {"metric": metric, "unit": unit, "value": value, "higher_is_better": hib, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "data": "synthetic", "dtype": dtype, "config": config,
            "clocks": clk.summary("")}
    line.update(extra)
    print(json.dumps(line), flush=True)


def run_multishift(args):
    """32^4, 11 shifts logspace(-4, 0), one Gaussian source, per-shift tol 1e-8."""
    import torch

    import paper_1611_00728_gb300 as sq
    import synth

    sq.build_if_needed()
    fat, lng = synth.fat_long_links(LATTICE, MS_SEEDS[0])
    lat = sq.Lattice(LATTICE)
    lat.load_links(fat, lng, recon12=True)
    b = lat.pack(synth.gaussian_source(LATTICE, MS_SEEDS[1]))
    clk = ClockSampler(gpu_uuid(torch, 0)).start()
    res = measure_multishift(torch, sq, clk, lat, b, args.steps, compare=not args.no_compare)
    clk.stop()
    res["clocks"] = clk.summary("multishift")
    lat.close()
    _workload_line("multi-shift CG time to per-shift true residual 1e-8 vs plain FP64 CG", res["mixed"]["ms"], args,
                   {"workload": "32^4 multi-shift CG, 11 shifts logspace(-4,0), 1 source (seeds 1003/2300)",
                    "vh": int(np.prod(LATTICE)) // 2, "shifts": list(MS_SHIFTS)}, clk, {"multishift": res})


def run_rational(args):
    """32^4, m=0.01: one application of a 12-pole rational approximation of (4m^2 - D_eo D_oe)^(-1/2)
    to a Gaussian source (the RHMC use of the multi-shift solver), per-pole tol 1e-8."""
    import torch

    import paper_1611_00728_gb300 as sq
    import synth

    sq.build_if_needed()
    fat, lng = synth.fat_long_links(LATTICE, MS_SEEDS[0])
    lat = sq.Lattice(LATTICE)
    lat.load_links(fat, lng, recon12=True)
    b = lat.pack(synth.gaussian_source(LATTICE, MS_SEEDS[1]))
    clk = ClockSampler(gpu_uuid(torch, 0)).start()
    res = measure_rational(torch, sq, clk, lat, b, args.steps)
    clk.stop()
    lat.close()
    _workload_line("rational-function application r(A) b (12 poles) time, every pole to true residual 1e-8",
                   res["mixed"]["ms"], args,
                   {"workload": "32^4, m=0.01, 12-pole Gauss-Legendre approximation of x^(-1/2) on [4m^2, 16], "
                                "1 source (seeds 1003/2300)", "vh": int(np.prod(LATTICE)) // 2}, clk,
                   {"rational": res})


def run_batched(args):
    """16 sources each on 16^4, 24^4, 32^3x64, m = 0.02, one batched solve vs FP64 CG per source."""
    import torch

    import paper_1611_00728_gb300 as sq

    sq.build_if_needed()
    specs = BATCHED_SPECS
    if args.lattice:
        specs = (tuple(int(v) for v in args.lattice.split(",")),)
    if args.pin:
        sq.pin_batched_tuning(*[int(v) for v in args.pin.split(",")])
    lats, bs, xs = make_batched(sq, torch, specs)
    clk = ClockSampler(gpu_uuid(torch, 0)).start()
    res = measure_batched(torch, sq, clk, lats, bs, xs, args.steps, compare=not args.no_compare)
    clk.stop()
    res["clocks"] = clk.summary("batched")
    for lat in lats:
        lat.close()
    n = int(bs[0].shape[0]) * len(specs)
    _workload_line(f"batched CG time to true residual 1e-8 ({n} sources, {len(specs)} lattices) vs plain FP64 CG",
                   res["ms"], args, {"workload": "16 Gaussian sources each on " + ", ".join("x".join(map(str, L))
                                                                                        for L in specs)
                                     + ", m=0.02 (gauge seeds from 1004)",
                                     "site_rhs": sum(16 * int(np.prod(L)) // 2 for L in specs)}, clk,
                   {"batched": res})


def run_hisq(args):
    """HISQ link construction at 32^4 (thin -> fat7 -> U(3) projection -> Lepage/Naik level), device entry
    point timed with CUDA events; then mixed and FP64 CG on the HISQ links (m = 0.01, true residual 1e-8)."""
    import torch

    import paper_1611_00728_gb300 as sq
    import synth

    sq.build_if_needed()
    lattice = tuple(int(v) for v in args.lattice.split(",")) if args.lattice else LATTICE
    V = int(np.prod(lattice))
    clk = ClockSampler(gpu_uuid(torch, 0)).start()
    res = measure_hisq(torch, sq, clk, lattice, args.steps)
    clk.stop()
    cpu = None
    if not args.no_cpu_baseline:
        import oracle.hisq as oh

        Ls = (8, 8, 8, 8)
        th = synth.thin_links(Ls, GAUGE_SEED)
        t0 = time.perf_counter()
        oh.hisq_links(Ls, th)
        dt = time.perf_counter() - t0
        Vs = int(np.prod(Ls))
        cpu = {"value": Vs * 4 * sq.HISQ_FLOPS_PER_LINK / dt / 1e9, "unit": "GFLOP/s", "cores": 1, "kind": "oracle",
               "seconds": dt, "sample": "oracle (numpy path sums, FP64) HISQ links of an 8^4 lattice, same counted "
                                        "flops per link"}
    gflops = res["smear_gflops"]
    _workload_line("HISQ link construction time (thin -> fat, long; float-float products, FP64 links) and CG time "
                   "on the HISQ links",
                   res["smear_ms"], args,
                   {"workload": "x".join(map(str, lattice)) + " HISQ smearing of random SU(3) thin links (width 0.3, "
                                "seed 1002); CG m=0.01 to true rel. residual 1e-8 on the result", "sites": V,
                    "l2": f"thin links {V * 576 / 1e9:.2f} GB, workspace {V * 56 * 144 / 1e9:.2f} GB (L2 129 MB)"},
                   clk, {"roofline": {"bound": "alu", "kernel": "sqcg_hisq_smear (8 kernels, float-float 3x3 products)",
                                      "achieved": gflops, "peak": HISQ_FF_ALU_PEAK_GFLOPS, "unit": "GFLOP/s",
                                      "frac": gflops / HISQ_FF_ALU_PEAK_GFLOPS,
                                      "peak_kind": "FP32 pipe (128 lanes x 152 SMs x 2.07 GHz, nominal) at 42 FP32 "
                                                   "instructions per counted float-float complex multiply-add",
                                      "counted_flops_per_link": sq.HISQ_FLOPS_PER_LINK, "traffic": None},
                         "cpu_baseline": cpu, "hisq": res}, dtype="ff")


# The learned preconditioner's training set: (residual, error) pairs from plain FP64 CG on seeded 16^4 gauge
# fields (seeds 0..TRAIN_FIELDS-1), TRAIN_SOURCES Gaussian sources each, at the CG iterates TRAIN_KS.
TRAIN_FIELDS = 32
TRAIN_SOURCES = 8
TRAIN_KS = tuple(range(0, 24)) + tuple(range(24, 64, 3)) + (64, 70, 76, 82, 90)
TRAIN_LRS = (1e-2, 1e-2, 5e-3, 2.5e-3, 1.25e-3, 6e-4)
TRAIN_STEPS_PER_FIELD = 60


def train_network(torch, sq, log=None):
    """Train the network at 16^4 on about 10^4 CG pairs: CG iterates well before convergence, each against
    an FP64 x* solved to 1e-13, with the A^2-norm loss. Returns (params, record)."""
    import synth

    m, sigma = LEARNED_MASS, 4 * LEARNED_MASS ** 2
    Ltr = (16, 16, 16, 16)
    t0 = time.perf_counter()
    per = len(TRAIN_KS) * TRAIN_SOURCES
    fields = []
    for gseed in range(TRAIN_FIELDS):
        fat, lng = synth.fat_long_links(Ltr, gseed)
        lat = sq.Lattice(Ltr)
        lat.load_links(fat, lng, recon12=True)
        net = sq.Network(lat)
        net.set_loss(2)
        R = lat.new_spinor(sq.F32, count=per)
        E = lat.new_spinor(sq.F32, count=per)
        xs, xk = lat.new_spinor(), lat.new_spinor()
        n = 0
        for src in range(TRAIN_SOURCES):
            b = lat.pack(synth.gaussian_source(Ltr, 5000 + 100 * gseed + src))
            xs.zero_()
            lat.cg_solve(m, b, xs, tol=1e-13, max_iter=50000, mode=sq.MODE_F64)
            for k in TRAIN_KS:
                xk.zero_()
                if k > 0:  # CG from 0 truncated at k iterations: exactly the k-th iterate of the long run
                    lat.cg_solve(m, b, xk, tol=1e-30, max_iter=k, mode=sq.MODE_F64, raise_on_error=False)
                net.make_pair(sigma, b, xk, xs, R[n], E[n])
                n += 1
        fields.append((lat, net, R, E))
        if log:
            log(f"pairs: field {gseed + 1}/{TRAIN_FIELDS} ({time.perf_counter() - t0:.0f} s)")
    torch.cuda.synchronize()
    t_data = time.perf_counter() - t0
    rng = np.random.default_rng(0)
    params = None
    losses = []
    t0 = time.perf_counter()
    for epoch, lr in enumerate(TRAIN_LRS):
        for g in rng.permutation(TRAIN_FIELDS):
            lat, net, R, E = fields[g]
            net.set_params(params if params is not None else init_net_params(sq))
            first, last = net.train(sigma, R, E, steps=TRAIN_STEPS_PER_FIELD, batch=8, lr=lr,
                                    seed=int(g) + 1 + 100 * epoch)
            losses.append((first, last))
            params = net.get_params()
        if log:
            log(f"epoch {epoch + 1}/{len(TRAIN_LRS)}: last batch loss {losses[-1][1]:.4f}")
    t_train = time.perf_counter() - t0
    for lat, net, R, E in fields:
        net.close()
        lat.close()
    rec = {"pairs": TRAIN_FIELDS * per, "lattice": list(Ltr), "mass": m,
           "schedule": f"{len(TRAIN_LRS)} epochs x {TRAIN_FIELDS} gauge fields x {TRAIN_STEPS_PER_FIELD} Adam steps "
                       f"(batch 8), step size {list(TRAIN_LRS)}, A^2-norm loss",
           "data": f"gauge seeds 0-{TRAIN_FIELDS - 1}, {TRAIN_SOURCES} sources each (seeds 5000 + 100 field + "
                   f"source), CG iterates k in {list(TRAIN_KS)}",
           "train_loss_first_last": [losses[0][0], losses[-1][1]], "seconds_data": t_data, "seconds_train": t_train}
    return params, rec


def run_learned(args):
    """Learned preconditioner: train at 16^4 on ~10^4 CG pairs (or load parameters), flexible CG on the held-out
    gauge field at 16^4 and 32^4 against plain FP64 and mixed CG."""
    import torch

    import paper_1611_00728_gb300 as sq

    sq.build_if_needed()
    if args.load_params:
        params, rec = np.load(args.load_params).astype(np.float32), None
    else:
        params, rec = train_network(torch, sq, log=lambda msg: print(msg, file=sys.stderr, flush=True))
        rec["command"] = "python bench.py --workload learned --save-params " + (args.save_params or "<path>")
    clk = ClockSampler(gpu_uuid(torch, 0)).start()
    results = {}
    for L in ((16, 16, 16, 16), LATTICE):
        results["x".join(map(str, L))] = measure_learned(torch, sq, clk, L, params, args.steps,
                                                         compare=not args.no_compare, tag="learned" + str(L[0]))
    clk.stop()
    if rec is not None:
        rec["held_out"] = {k: {n: v for n, v in r.items() if isinstance(v, dict)} for k, r in results.items()}
    if args.save_params:
        np.save(args.save_params, np.asarray(params, dtype=np.float32))
        if rec is not None:
            with open(args.save_params[:-4] + ".json" if args.save_params.endswith(".npy")
                      else args.save_params + ".json", "w") as f:
                json.dump(rec, f, indent=1)
    _workload_line("learned-preconditioned flexible CG time to true residual 1e-8 vs plain FP64 CG",
                   results["32x32x32x32"]["fcg_nn"]["ms"], args,
                   {"workload": "held-out gauge seed 9000 (source 9100) at 16^4 and 32^4, m=0.005; network "
                                + (f"parameters from {args.load_params}" if args.load_params else
                                   "trained in this run at 16^4")}, clk,
                   {"results": results, "training": rec}, dtype="f32/bf16")


def init_net_params(sq):
    """Small seeded initial weights (numpy; the binding's parameter layout)."""
    rng = np.random.default_rng(12345)
    p = np.zeros(sq.NN_NPARAMS, dtype=np.float32)
    for sl, shape in sq.NN_LAYERS:
        p[sl] = rng.standard_normal(sl.stop - sl.start) * 0.3 / np.sqrt(9 * shape[2])
    for ga, gb in sq.NN_GATES:
        p[ga], p[gb] = -0.5, 1.0
    return p


def main():
    args = parse()
    if args.steps < 1:
        raise SystemExit("--steps must be >= 1")
    if args.workload != "single":
        {"multishift": run_multishift, "rational": run_rational, "batched": run_batched, "learned": run_learned,
         "hisq": run_hisq}[args.workload](args)
        return
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
