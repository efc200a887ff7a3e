"""Benchmark: global SPAI iterations (MR, LOMR, CG) plus PCG assessment on one GB300.

Workload (one step): the 3-D 7-point variable-coefficient diffusion operator
on a 64^3 grid (n = 262,144; kappa = exp(g), g Gaussian, sigma 1.5,
correlation length 8 cells, harmonic-mean faces, seed 0); FP32 values with
FP64 reductions; per-column cap 3 nnz(A[:,j]); from M_0 = diag(A)^{-1}:
50 MR iterations, then PCG, 50 LOMR iterations, then PCG, 50 CG iterations,
then PCG (b ~ U(-1,1) seed 0, rtol 1e-8, symmetric part of M as
preconditioner; FP64 products, vectors and scalars: FP32-values products
take 6 % more iterations with MR's M, past the 2 % the mixed path is held
to).  Metric:
SPAI iterations per second over the whole step (150 iterations / step time,
PCG and set-up included).  The FP64 path (FP64 values, FP64 PCG) is timed
on the same workload and reported beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
  python bench.py --workload batch64     # batched SPAIs + block PCG (below)
  python bench.py --workload aniso1024   # rotated anisotropic 9-point, 1024^2
  python bench.py --workload fpmr        # gradient through 10 fixed-pattern MR steps

--workload batch64: 64 variable-coefficient operators (alternating 2-D
5-point and 3-D 7-point, n log-uniform in [1e3, 6.4e4], field seed 1000+k,
953,176 rows in all) in one batched handle; one step = 30 LOMR iterations of
every matrix (mixed, cap 3 nnz(A[:,j])) from M_0 = diag(A)^{-1}, then block
PCG with 32 right-hand sides per matrix (U(-1,1), seed 2000+k), symmetric
part of M, rtol 1e-8, FP64 products (FP32-values products leave some of
the ill-conditioned 2-D systems unconverged at 1000 iterations).  Metric: matrix-iterations per second (64 x 30 / step
time); the PCG share and iteration counts are reported beside it.

--impl reference times the CPU oracle (the plain single-threaded C
implementation used by the tests) on a bounded sample of the same workload.
N > 1 runs N independent replicas (one per GPU, weak scaling): the method
shards by columns, but this build has no multi-GPU data path.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

ITERS = 50
CAP = 3.0
PCG_PREC = "fp64"  # the timed PCG's products (see accuracy_report)
PCG_MAXIT = 1000
METHODS = ("mr", "lomr", "cg")
WORKLOAD = "varcoef3d_64"


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x, dist, device="cuda"):
    """The largest value of x over all ranks (x itself without a process group)."""
    if not dist:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world, units_per_rank, seconds):
    """Whole-job throughput of independent replicas: every rank processes
    units_per_rank in the slowest rank's time."""
    return world * units_per_rank / seconds


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """Samples nvidia-smi SM clocks and throttle reasons in the background."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 7:
                continue
            try:
                sm.append(float(p[0]))
                smax = float(p[1])
            except ValueError:
                continue
            for nm, v in zip(names, p[3:7]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def run_ours(args):
    import numpy as np
    import torch

    from paper_2511_09753_gb300 import inputs as I
    from paper_2511_09753_gb300.spai import PREC_SPAI_SYM, Spai

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    n, rp, ci, v = I.varcoef_3d_7pt(64, sigma=1.5, ell=8.0, seed=0)
    b = I.rhs_uniform(n, 0)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    # device-resident inputs: A copied once, handle created outside the timed region
    g = Spai(n, rp, ci, v, prec="mixed", cap_factor=CAP)
    g.set_pcg_prec(PCG_PREC)
    tuned = {m: g.autotune(m, 10) for m in METHODS}  # launch shapes (results unchanged)
    b_dev = torch.tensor(b, dtype=torch.float64, device="cuda")
    x_dev = torch.empty_like(b_dev)

    def step(h):
        out = {}
        for m in METHODS:
            h.reset()
            r = h.run(m, ITERS)
            p = h.pcg(b_dev, x_dev, rtol=1e-8, maxit=PCG_MAXIT, precond=PREC_SPAI_SYM)
            out[m] = (r, p)
        return out

    for _ in range(args.warmup):
        step(g)
    torch.cuda.synchronize()
    g.set_timing(True)
    s0 = g.stats()
    clocks = Clocks(local)
    clocks.start()
    times = []
    last = None
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    for _ in range(args.steps):
        flush.fill_(1.0)  # evict L2 between steps (outside the events)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        torch.cuda.nvtx.range_push("step")  # lets an ncu launch list select the timed steps
        last = step(g)
        torch.cuda.nvtx.range_pop()
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    clk = clocks.stop()
    s1 = g.stats()
    g.set_timing(False)
    ms_step = max_over_ranks(sum(times) / len(times), dist)
    total_iters = ITERS * len(METHODS)
    value = job_throughput(ws, total_iters, ms_step * 1e-3)

    # dominant kernel: the column pass (timed per launch inside the library).
    # Algorithmic bytes: the iterate slabs each pass reads and writes, their
    # lengths and A once per pass (the library's device counter), without
    # the R lists CG's pass A stores for pass B (a layout choice of this
    # library, not traffic the method needs); the full counter is reported
    # beside them.
    launches = s1["colpass_launches"] - s0["colpass_launches"]
    cp_ms = s1["colpass_ms"] - s0["colpass_ms"]
    cp_bytes = s1["colpass_bytes"] - s0["colpass_bytes"]
    r_bytes = s1["colpass_r_bytes"] - s0["colpass_r_bytes"]
    peak, peak_kind = _peaks()
    per_launch_bytes = (cp_bytes - r_bytes) / max(launches, 1)
    per_launch_ms = cp_ms / max(launches, 1)
    achieved = per_launch_bytes / (per_launch_ms * 1e-3) / 1e9 if per_launch_ms > 0 else 0.0
    gpu_launches = ((s1["colpass_launches"] - s0["colpass_launches"])
                    + (s1["pcg_launches"] - s0["pcg_launches"])
                    + (s1["other_launches"] - s0["other_launches"]))

    # end to end through the C ABI with host buffers in pinned memory: create
    # (H2D of A), run, PCG with host b and x, export M (D2H) -- every step
    def pinned(a):
        t = torch.empty(a.shape, dtype=getattr(torch, a.dtype.name), pin_memory=True).numpy()
        t[...] = a
        return t

    rp_h, ci_h, v_h, b_h = pinned(rp), pinned(ci), pinned(v), pinned(b)
    x_h = pinned(np.zeros(n))
    slots = int(np.sum(np.clip(np.floor(CAP * np.diff(rp)), 1, n)))  # M's capacity
    m_out = (pinned(np.zeros(n + 1, np.int32)), pinned(np.zeros(slots, np.int32)),
             pinned(np.zeros(slots)))

    def e2e_step():
        h = Spai(n, rp_h, ci_h, v_h, prec="mixed", cap_factor=CAP)
        h.set_pcg_prec(PCG_PREC)
        h2d = rp_h.nbytes + ci_h.nbytes + v_h.nbytes
        d2h = 0
        for m in METHODS:
            h.reset()
            h.run(m, ITERS)
            p = h.pcg(b_h, x_h, rtol=1e-8, maxit=PCG_MAXIT, precond=PREC_SPAI_SYM)
            h2d += b_h.nbytes
            d2h += x_h.nbytes
            cp, ri, va = h.get_M(out=m_out)
            nz = int(cp[n])
            d2h += cp.nbytes + 4 * nz + 8 * nz
        h.close()
        return h2d, d2h

    e2e_steps = max(1, min(args.steps, 3))
    e2e_step()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        h2d, d2h = e2e_step()
    torch.cuda.synchronize()
    e2e_s = max_over_ranks((time.perf_counter() - t0) / e2e_steps, dist)

    # FP64 path, same workload, one step (reported beside the mixed path)
    g64 = Spai(n, rp, ci, v, prec="fp64", cap_factor=CAP)
    step(g64)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    r64 = step(g64)
    e1.record(stream)
    e1.synchronize()
    fp64_ms = e0.elapsed_time(e1)

    results = accuracy_report(g, g64, last, r64, b_dev, x_dev)

    cpu = cpu_baseline() if (rank == 0 and ws == 1 and not args.no_cpu) else None
    if rank == 0:
        line = {
            "metric": "SPAI iterations/s (MR+LOMR+CG, 50 each, with PCG assessment)",
            "value": value,
            "unit": "SPAI iterations/s",
            "n_gpus": ws,
            "steps": args.steps,
            "warmup": args.warmup,
            "ms_per_step": ms_step,
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": "f32 values / f64 reductions",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "n": n, "nnz": int(len(v)), "cap_factor": CAP,
                       "iters_per_method": ITERS, "methods": list(METHODS),
                       "pcg": "symmetric part of M, rtol 1e-8, maxit 1000, FP64 products",
                       "l2": "flushed between steps (256 MB write)", "parallelism": "replicas",
                       "autotuned_ms_per_iter": tuned},
            "e2e": {"value": ws * total_iters / e2e_s, "unit": "SPAI iterations/s",
                    "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
            "roofline": {"bound": "hbm", "kernel": "colpass_kernel", "achieved": achieved,
                         "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "peak_source": peak_kind, "traffic": colpass_traffic(),
                         "algorithmic_bytes_per_launch": per_launch_bytes,
                         "counter_bytes_per_launch": cp_bytes / max(launches, 1),
                         "launch_ms": per_launch_ms, "launches": launches},
            "cpu_baseline": cpu,
            "gpu_launches": int(gpu_launches),
            "clocks": clk,
            "fp64_path": {"ms_per_step": fp64_ms,
                          "value": total_iters / (fp64_ms * 1e-3), "unit": "SPAI iterations/s"},
            "results": results,
            "wall_s": wall,
        }
        print(json.dumps(line))
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def accuracy_report(g, g64, last, r64, b_dev, x_dev):
    """Per method: the mixed path against the FP64 path on the same workload
    (||I - A M||_F within 1e-5 relative and PCG iterations within 2 % are the
    targets).  residual_fp64 is ||I - A M||_F computed in FP64 from the mixed
    M; pcg_iters is the timed PCG (mixed M, FP64 products), fp64_pcg_iters
    the FP64 path's.  pcg_iters_fp32_products shows the same solve with
    FP32-values products (not timed: it misses the 2 % target with MR's M).
    Runs after the timed region."""
    from paper_2511_09753_gb300.spai import PREC_SPAI_SYM
    out = {}
    for m in METHODS:
        rm, pm = last[m]
        g.reset()
        g.run(m, ITERS)
        res_mixed = g.residual_norm()
        g.set_pcg_prec("mixed")
        p32 = g.pcg(b_dev, x_dev, rtol=1e-8, maxit=PCG_MAXIT, precond=PREC_SPAI_SYM)
        g.set_pcg_prec(PCG_PREC)
        g64.reset()
        g64.run(m, ITERS)
        res64 = g64.residual_norm()
        it, it32, it64 = int(pm["iters"]), int(p32["iters"]), int(r64[m][1]["iters"])
        out[m] = {
            "history_resnorm": float(rm["resnorm"][-1]),
            "residual_fp64": res_mixed,
            "fp64_path_residual": res64,
            "residual_rel_err": abs(res_mixed - res64) / res64,
            "pcg_iters": it,
            "pcg_status": int(pm["status"]),
            "pcg_relres": float(pm["relres"]),
            "fp64_pcg_iters": it64,
            "fp64_pcg_status": int(r64[m][1]["status"]),
            "pcg_iters_rel_diff": abs(it - it64) / max(1, it64),
            "pcg_iters_fp32_products": it32,
            "pcg_iters_fp32_products_rel_diff": abs(it32 - it64) / max(1, it64),
        }
    return out


TRAFFIC_SUMMARY = os.path.join(ROOT, "profiles", "colpass_traffic_varcoef3d64.md")
COLPASS_SOURCES = ("colpass.cuh", "warp_ops.cuh", "common.cuh", "colpass_launch.cuh",
                   "colpass_f32.cu", "colpass_hot.cu", "colpass_shape.cuh")


def colpass_sources_sha16():
    import hashlib
    h = hashlib.sha256()
    for f in COLPASS_SOURCES:
        with open(os.path.join(ROOT, "paper_2511_09753_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def colpass_traffic():
    """DRAM bytes (read + write) per column-pass launch of the bench step, from
    the ncu summary under profiles/ (its line "traffic_bytes_per_launch: B
    sources_sha16: H"), or None when the column-pass sources have changed
    since those counters were taken."""
    try:
        with open(TRAFFIC_SUMMARY) as f:
            for line in f:
                if line.startswith("traffic_bytes_per_launch:"):
                    parts = line.split()
                    if parts[3] == colpass_sources_sha16():
                        return float(parts[1])
    except (OSError, IndexError, ValueError):
        pass
    return None

BATCH_ITERS = 30
BATCH_RHS = 32


def run_batch(args):
    import numpy as np
    import torch

    from paper_2511_09753_gb300 import inputs as I
    from paper_2511_09753_gb300.spai import PREC_SPAI_SYM, SpaiBatch

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    mats = I.batch_uneven(count=64)
    ns = [m[0] for m in mats]
    B = [np.random.default_rng(2000 + k).uniform(-1.0, 1.0, size=(BATCH_RHS, n))
         for k, n in enumerate(ns)]
    flatB = np.concatenate([b.ravel() for b in B])
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    g = SpaiBatch(mats, prec="mixed", cap_factor=CAP)
    g.autotune("lomr", 5)
    b_dev = torch.tensor(flatB, dtype=torch.float64, device="cuda")
    x_dev = torch.empty_like(b_dev)
    pcg_ms = []

    def step(h, record=False):
        h.reset()
        r = h.run("lomr", BATCH_ITERS)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        p = h.pcg_block(b_dev, rtol=1e-8, maxit=PCG_MAXIT, precond=PREC_SPAI_SYM,
                        nrhs=BATCH_RHS, x=x_dev)
        e1.record(stream)
        e1.synchronize()
        if record:
            pcg_ms.append(e0.elapsed_time(e1))
        return r, p

    for _ in range(args.warmup):
        step(g)
    torch.cuda.synchronize()
    g.set_timing(True)
    s0 = g.stats()
    clocks = Clocks(local)
    clocks.start()
    times = []
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    for _ in range(args.steps):
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        last = step(g, record=True)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    torch.cuda.synchronize()
    clk = clocks.stop()
    s1 = g.stats()
    g.set_timing(False)
    ms_step = max_over_ranks(sum(times) / len(times), dist)
    units = len(mats) * BATCH_ITERS
    value = job_throughput(ws, units, ms_step * 1e-3)
    launches = s1["colpass_launches"] - s0["colpass_launches"]
    cp_ms = s1["colpass_ms"] - s0["colpass_ms"]
    cp_bytes = s1["colpass_bytes"] - s0["colpass_bytes"]
    peak, peak_kind = _peaks()
    per_launch_bytes = cp_bytes / max(launches, 1)
    per_launch_ms = cp_ms / max(launches, 1)
    achieved = per_launch_bytes / (per_launch_ms * 1e-3) / 1e9 if per_launch_ms > 0 else 0.0
    gpu_launches = ((s1["colpass_launches"] - s0["colpass_launches"])
                    + (s1["pcg_launches"] - s0["pcg_launches"])
                    + (s1["other_launches"] - s0["other_launches"]))

    def e2e_step():
        h = SpaiBatch(mats, prec="mixed", cap_factor=CAP)
        h2d = sum(m[1].nbytes + m[2].nbytes + m[3].nbytes for m in mats) + flatB.nbytes
        h.run("lomr", BATCH_ITERS)
        p = h.pcg_block(B, rtol=1e-8, maxit=PCG_MAXIT, precond=PREC_SPAI_SYM)
        d2h = sum(x.nbytes for x in p["x"])
        h.close()
        return h2d, d2h

    e2e_step()
    torch.cuda.synchronize()
    e2e_steps = max(1, min(args.steps, 3))
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        h2d, d2h = e2e_step()
    torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / e2e_steps

    r, p = last
    it = p["iters"]
    if rank == 0:
        line = {
            "metric": "batched SPAI matrix-iterations/s (64 matrices x 30 LOMR, then block PCG)",
            "value": value,
            "unit": "matrix SPAI iterations/s",
            "n_gpus": ws,
            "steps": args.steps,
            "warmup": args.warmup,
            "ms_per_step": ms_step,
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": "f32 values / f64 reductions",
            "data": "synthetic",
            "config": {"workload": "batch64_uneven", "nmat": len(mats), "n_total": int(sum(ns)),
                       "n_min": int(min(ns)), "n_max": int(max(ns)), "cap_factor": CAP,
                       "lomr_iters": BATCH_ITERS, "rhs_per_matrix": BATCH_RHS,
                       "pcg": "symmetric part of M, rtol 1e-8, maxit 1000, FP64 products",
                       "l2": "flushed between steps (256 MB write)", "parallelism": "replicas"},
            "e2e": {"value": ws * units / e2e_s, "unit": "matrix SPAI iterations/s",
                    "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
            "roofline": {"bound": "hbm", "kernel": "colpass_kernel", "achieved": achieved,
                         "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "peak_source": peak_kind, "traffic": None,
                         "algorithmic_bytes_per_launch": per_launch_bytes,
                         "launch_ms": per_launch_ms, "launches": launches},
            "cpu_baseline": None,
            "gpu_launches": int(gpu_launches),
            "clocks": clk,
            "pcg_block": {"ms_per_step": sum(pcg_ms) / len(pcg_ms),
                          "iters_min": int(it.min()), "iters_median": float(np.median(it)),
                          "iters_max": int(it.max()), "status": int(p["status"]),
                          "relres_max": float(p["relres"].max())},
            "lomr_resnorm_max": float(np.nanmax(r["resnorm_each"][:, -1])),
        }
        print(json.dumps(line))
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def profile_case(method, prec):
    """Small launch sequence for ncu captures: one handle on the workload,
    10 iterations of `method` from M_0 (11 column passes for MR/LOMR, 20 for
    CG); the later passes see columns filled to their caps as in the bench."""
    import torch

    from paper_2511_09753_gb300 import inputs as I
    from paper_2511_09753_gb300.spai import Spai
    n, rp, ci, v = I.varcoef_3d_7pt(64, sigma=1.5, ell=8.0, seed=0)
    g = Spai(n, rp, ci, v, prec=prec, cap_factor=CAP)
    r = g.run(method, 10)
    torch.cuda.synchronize()
    print(json.dumps({"profile": method, "prec": prec, "resnorm": float(r["resnorm"][-1])}))


PHASES = ("load", "union", "select", "store", "spgemm", "to_list+clear", "fixsum")
KIND_NAMES = {0: "mr", 1: "lomr", 2: "cg_a", 3: "cg_b"}


def run_phase_clocks(args):
    """Per-phase cycle budget of the FP32 column pass on the bench workload:
    builds libspai_phase.so (the same sources with SPAI_PHASE_CLOCKS), runs
    args.warmup untimed steps and one counted step of the bench (50 MR, 50
    LOMR, 50 CG iterations; no PCG), and prints, per pass kind, the clock64()
    cycles per column of each phase, summed over warps and divided by the
    columns processed.  Timings of this build are not bench values."""
    import ctypes as C

    import torch

    from paper_2511_09753_gb300 import build as B
    from paper_2511_09753_gb300 import inputs as I
    from paper_2511_09753_gb300 import spai as S
    S.use_library(B.build(variant="phase"))
    lib = S.load()
    lib.spai_phase_clocks.restype = C.c_int
    lib.spai_phase_clocks.argtypes = [C.c_void_p, C.c_int]
    n, rp, ci, v = I.varcoef_3d_7pt(64, sigma=1.5, ell=8.0, seed=0)
    g = S.Spai(n, rp, ci, v, prec="mixed", cap_factor=CAP)
    for m in METHODS:
        g.autotune(m, 10)
    buf = (C.c_ulonglong * 128)()

    def step():
        for m in METHODS:
            g.reset()
            g.run(m, ITERS)
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        step()
    assert lib.spai_phase_clocks(buf, 1) == 0
    step()
    assert lib.spai_phase_clocks(buf, 1) == 0
    out = {}
    for k, name in KIND_NAMES.items():
        row = [buf[k * 16 + q] for q in range(16)]
        cols = row[8]
        if cols == 0:
            continue
        ph = {PHASES[q]: row[q] / cols for q in range(len(PHASES))}
        ph["sum_of_phases"] = sum(row[q] for q in range(7)) / cols
        ph["warp_cycles_per_column"] = row[9] / cols
        ph["cta_tail_cycles_per_column"] = row[7] / cols
        ph["columns"] = cols
        out[name] = ph
    print(json.dumps({"phase_clocks": out, "workload": WORKLOAD, "prec": "mixed",
                      "unit": "clock64 cycles per column (warp view)"}))


def run_aniso(args):
    """Rotated anisotropic 9-point operator, 1024^2 (eps 1e-3, theta pi/6):
    LOMR and CG, 100 iterations each at caps 2, 4 and 8 nnz(A[:,j]) (mixed),
    each followed by the Lanczos extremes of sym(M); then the best
    approximate inverses on supp(A^k), k = 1..4 (FP64), with theirs.  The
    metric is SPAI iterations/s over the six runs."""
    import numpy as np
    import torch

    from paper_2511_09753_gb300 import inputs as I
    from paper_2511_09753_gb300.spai import Spai

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    n, rp, ci, v = I.aniso_2d_9pt(1024)
    v0 = np.random.default_rng(0).standard_normal(n)
    stream = torch.cuda.current_stream()
    iters = int(os.environ.get("ANISO_ITERS", "100"))
    runs, tot_ms, tot_it = [], 0.0, 0
    for capf in (2.0, 4.0, 8.0):
        h = Spai(n, rp, ci, v, prec="mixed", cap_factor=capf)
        for m in ("lomr", "cg"):
            h.reset()
            h.run(m, 2)
            h.reset()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            r = h.run(m, iters)
            e1.record(stream)
            e1.synchronize()
            ms = e0.elapsed_time(e1)
            tot_ms += ms
            tot_it += iters
            sp = h.sym_spectrum(steps=300, v0=v0)
            runs.append({"method": m, "cap_factor": capf, "ms": ms,
                         "resnorm_first_last": [float(r["resnorm"][0]), float(r["resnorm"][-1])],
                         "sym_lmin": sp["lmin"], "sym_lmax": sp["lmax"]})
        h.close()
    fixed = []
    for k in (1, 2, 3, 4):
        h = Spai(n, rp, ci, v, prec="fp64", cap_factor=10.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h.fixed_pattern(k)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        sp = h.sym_spectrum(steps=300, v0=v0)
        fixed.append({"k": k, "s": dt, "residual_fro": h.residual_norm(), "sym_lmin": sp["lmin"],
                      "sym_lmax": sp["lmax"], "nnz": h.nnz_M()})
        h.close()
    if rank == 0:
        print(json.dumps({
            "metric": "SPAI iterations/s (LOMR and CG, 100 each at caps 2/4/8)",
            "value": ws * tot_it / (tot_ms * 1e-3), "unit": "SPAI iterations/s", "n_gpus": ws,
            "higher_is_better": True, "dtype": "f32 values / f64 reductions", "data": "synthetic",
            "config": {"workload": "aniso9_1024", "n": n, "nnz": int(len(v)), "eps": 1e-3,
                       "theta": "pi/6", "iters": iters, "lanczos_steps": 300},
            "runs": runs, "fixed_pattern": fixed}))


def run_fpmr(args):
    """Gradient of ||I - A M_K||_F^2 through K = 10 fixed-pattern MR steps with
    respect to A's values: the 32^3 and 128^3 variable-coefficient operators
    (seed 0), FP64, one checkpoint of M per step; then the same through 10
    fixed-pattern LOMR steps (checkpoints of M and P per step).  Metric:
    gradients per second at 128^3 (MR, forward + backward, inputs resident)."""
    import numpy as np
    import torch

    from paper_2511_09753_gb300 import inputs as I
    from paper_2511_09753_gb300.spai import FixedPatternMR

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    out = {}
    for N, prec, method in ((32, "fp64", "mr"), (128, "fp64", "mr"), (128, "mixed", "mr"),
                            (32, "fp64", "lomr"), (128, "fp64", "lomr"), (128, "mixed", "lomr")):
        n, rp, ci, v = I.varcoef_3d_7pt(N, sigma=1.5, ell=8.0, seed=0)
        t0 = time.perf_counter()
        f = FixedPatternMR(n, rp, ci, 10, prec=prec, method=method)
        setup = time.perf_counter() - t0
        vd = torch.tensor(v, dtype=torch.float64, device="cuda")
        gd = torch.empty_like(vd)
        for _ in range(max(1, args.warmup)):
            f.forward(vd)
            f.backward(1.0, gd)
        torch.cuda.synchronize()
        times = []
        for _ in range(max(1, args.steps)):
            t0 = time.perf_counter()
            loss = f.forward(vd)
            f.backward(1.0, gd)
            torch.cuda.synchronize()
            times.append(time.perf_counter() - t0)
        info = f.info()
        out[f"{method}_{N}_{prec}"] = {"n": n, "nnz": int(len(v)), "setup_s": setup, "s_per_gradient": min(times),
                  "median_s": statistics.median(times), "loss": loss,
                  "grad_norm": float(torch.linalg.vector_norm(gd).item()), **info}
        f.close()
    if rank == 0:
        print(json.dumps({
            "metric": "gradients/s of ||I - A M_10||_F^2 w.r.t. A's values (128^3)",
            "value": ws / out["mr_128_fp64"]["median_s"], "unit": "gradients/s", "n_gpus": ws,
            "higher_is_better": True, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "fpmr_varcoef3d", "K": 10, "checkpoints": "M per step"},
            "cases": out}))


def profile_bpcg(prec):
    """Launch sequence for ncu captures of the block PCG kernels: the 64-matrix
    batch, 30 LOMR iterations, one block solve (products in `prec`)."""
    import numpy as np
    import torch

    from paper_2511_09753_gb300 import inputs as I
    from paper_2511_09753_gb300.spai import PREC_SPAI_SYM, SpaiBatch
    mats = I.batch_uneven(count=64)
    B = [np.random.default_rng(2000 + k).uniform(-1.0, 1.0, size=(BATCH_RHS, m[0]))
         for k, m in enumerate(mats)]
    g = SpaiBatch(mats, prec="mixed", cap_factor=CAP)
    g.set_pcg_prec(prec)
    g.run("lomr", BATCH_ITERS)
    p = g.pcg_block(B, rtol=1e-8, maxit=PCG_MAXIT, precond=PREC_SPAI_SYM)
    torch.cuda.synchronize()
    print(json.dumps({"profile": "bpcg", "prec": prec, "iters_max": int(p["iters"].max())}))


def profile_pcg(prec):
    """Launch sequence for ncu captures of the one-vector PCG kernels: the
    bench workload, 50 MR iterations (mixed values), then 64 PCG iterations
    with the symmetric part of M (products in `prec`), as in the bench step."""
    import torch

    from paper_2511_09753_gb300 import inputs as I
    from paper_2511_09753_gb300.spai import PREC_SPAI_SYM, Spai
    n, rp, ci, v = I.varcoef_3d_7pt(64, sigma=1.5, ell=8.0, seed=0)
    g = Spai(n, rp, ci, v, prec="mixed", cap_factor=CAP)
    g.set_pcg_prec(prec)
    g.run("mr", ITERS)
    p = g.pcg(I.rhs_uniform(n, 0), rtol=1e-8, maxit=64, precond=PREC_SPAI_SYM)
    torch.cuda.synchronize()
    print(json.dumps({"profile": "pcg", "prec": prec, "iters": int(p["iters"])}))


def profile_fpmr(prec):
    """Launch sequence for ncu captures of the differentiation kernels: the
    64^3 variable-coefficient operator, K = 10 fixed-pattern MR steps, one
    forward and one backward pass (values in `prec`)."""
    import torch

    from paper_2511_09753_gb300 import inputs as I
    from paper_2511_09753_gb300.spai import FixedPatternMR
    n, rp, ci, v = I.varcoef_3d_7pt(64, sigma=1.5, ell=8.0, seed=0)
    f = FixedPatternMR(n, rp, ci, 10, prec=prec)
    vd = torch.tensor(v, dtype=torch.float64, device="cuda")
    gd = torch.empty_like(vd)
    loss = f.forward(vd)
    f.backward(1.0, gd)
    torch.cuda.synchronize()
    print(json.dumps({"profile": "fpmr", "prec": prec, "loss": float(loss), **f.info()}))
    f.close()


def profile_fixed_pattern():
    """Launch sequence for ncu captures of the definiteness diagnostics: the
    rotated anisotropic 9-point operator on a 256^2 grid, the best SPAI on
    supp(A^2) (FP64), then 100 Lanczos steps on its symmetric part."""
    import numpy as np
    import torch

    from paper_2511_09753_gb300 import inputs as I
    from paper_2511_09753_gb300.spai import Spai
    n, rp, ci, v = I.aniso_2d_9pt(256)
    h = Spai(n, rp, ci, v, prec="fp64", cap_factor=10.0)
    h.fixed_pattern(2)
    sp = h.sym_spectrum(steps=100, v0=np.random.default_rng(0).standard_normal(n))
    torch.cuda.synchronize()
    print(json.dumps({"profile": "fixed_pattern", "nnz": h.nnz_M(), "lmin": sp["lmin"],
                      "lmax": sp["lmax"]}))
    h.close()


# PCG iterations of the step's three solves (FP64 products, rtol 1e-8, maxit
# 1000, symmetric part of M after 50 iterations of MR, LOMR, CG): the same on
# the oracle and on the GPU, which the 50-iteration full-size parity test
# checks bit for bit.  The CPU estimates below count this PCG work.
STEP_PCG_ITERS = {"mr": 227, "lomr": 166, "cg": 1000}


class CpuStep:
    """The oracle on the bench workload, for the CPU baseline: one handle per
    method, filled by `fill` iterations from M_0 (columns at their caps, as in
    the step), then sampled: `sample(k, q)` times k more iterations of each
    method and q PCG iterations with each method's M (symmetric part, FP64
    products), and extrapolates the step (50 iterations of each method plus
    the step's PCG iterations) from those per-iteration times."""

    def __init__(self, omp=True, fill=3):
        import oracle as O
        from paper_2511_09753_gb300 import inputs as I
        self.O = O
        self.omp = omp
        n, rp, ci, v = I.varcoef_3d_7pt(64, sigma=1.5, ell=8.0, seed=0)
        self.A = (n, rp, ci, v)
        self.b = I.rhs_uniform(n, 0)
        self.orc = {}
        for m in METHODS:
            o = O.Oracle(n, rp, ci, v, mixed=True, cap_factor=CAP, omp=omp)
            o.run(m, fill)
            self.orc[m] = o
        self.threads = self._threads()

    def _threads(self):
        if not self.omp:
            return 1
        import ctypes
        try:
            lib = ctypes.CDLL("libgomp.so.1")
            return int(lib.omp_get_max_threads())
        except OSError:
            return os.cpu_count() or 1

    def sample(self, k=1, q=5):
        n, rp, ci, v = self.A
        t_it, t_pcg = {}, {}
        for m in METHODS:
            o = self.orc[m]
            t0 = time.perf_counter()
            o.run(m, k)
            t_it[m] = (time.perf_counter() - t0) / k
            M = o.get_M()
            t0 = time.perf_counter()
            self.O.pcg(n, rp, ci, v, self.b, rtol=0.0, maxit=q, precond=3, M=M, mixed=False,
                       omp=self.omp)
            t_pcg[m] = (time.perf_counter() - t0) / q
        step = sum(ITERS * t_it[m] + STEP_PCG_ITERS[m] * t_pcg[m] for m in METHODS)
        wall = sum(k * t_it[m] + q * t_pcg[m] for m in METHODS)
        return {"step_s": step, "sample_s": wall, "s_per_iter": t_it, "s_per_pcg_iter": t_pcg}

    def describe(self, k, q):
        kind = f"OpenMP build, {self.threads} threads" if self.omp else "serial build, 1 thread"
        return (f"{k} iteration(s) of each of MR, LOMR, CG (columns already at their caps) and "
                f"{q} PCG iterations with each M on the full n={self.A[0]} operator, mixed "
                f"arithmetic (FP64 PCG products), {kind}; step time extrapolated to 50 iterations of each method plus "
                f"the step's PCG iterations {STEP_PCG_ITERS}")


def cpu_baseline(k=2, q=10):
    """The oracle on a bounded sample of the bench step, on all host cores."""
    st = CpuStep(omp=True)
    r = st.sample(k, q)
    value = ITERS * len(METHODS) / r["step_s"]
    return {"value": value, "unit": "SPAI iterations/s", "cores": st.threads, "kind": "oracle",
            "sample": st.describe(k, q), "sample_seconds": r["sample_s"],
            "s_per_iter": r["s_per_iter"], "s_per_pcg_iter": r["s_per_pcg_iter"]}


def run_reference(args):
    """The oracle as it stands on the host cores: each step is a bounded sample
    (one iteration of each method, five PCG iterations with each M) from
    which the bench step's time is extrapolated."""
    ws, rank, _ = _dist()
    if rank != 0:
        return
    k = max(1, args.steps)
    st = CpuStep(omp=True)
    for _ in range(args.warmup):
        st.sample(1, 5)
    steps = [st.sample(1, 5) for _ in range(k)]
    secs = sum(r["step_s"] for r in steps) / k
    sample_secs = sum(r["sample_s"] for r in steps) / k
    value = ITERS * len(METHODS) / secs
    line = {
        "impl": "reference",
        "metric": "SPAI iterations/s (MR+LOMR+CG, 50 each, with PCG assessment)",
        "value": value,
        "unit": "SPAI iterations/s",
        "n_gpus": ws,
        "steps": k,
        "warmup": args.warmup,
        "ms_per_step": secs * 1e3,
        "sample_ms_per_step": sample_secs * 1e3,
        "note": "ms_per_step is the full step extrapolated from each step's timed sample "
                "(sample_ms_per_step of wall time)",
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32 values / f64 reductions",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "cap_factor": CAP,
                   "parallelism": f"cpu, {st.threads} OpenMP threads"},
        "cpu_baseline": {"value": value, "unit": "SPAI iterations/s", "cores": st.threads,
                         "kind": "oracle", "sample": st.describe(1, 5)},
        "e2e": {"value": value, "unit": "SPAI iterations/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-baseline sample")
    ap.add_argument("--profile", choices=list(METHODS) + ["pcg", "bpcg", "fpmr", "fixed_pattern"],
                    default=None,
                    help="profiling case for ncu: 10 iterations of one method on the workload, "
                         "(pcg) 64 iterations of its vector PCG, (bpcg) one block PCG "
                         "solve of the 64-matrix batch, (fpmr) one gradient at 64^3, or "
                         "(fixed_pattern) the SPAI on supp(A^2) and Lanczos at 256^2")
    ap.add_argument("--phase-clocks", action="store_true",
                    help="per-phase cycles per column of the FP32 column pass (profiling build)")
    ap.add_argument("--prec", choices=["mixed", "fp64"], default="mixed")
    ap.add_argument("--workload", choices=[WORKLOAD, "batch64", "aniso1024", "fpmr"],
                    default=WORKLOAD)
    args = ap.parse_args()
    if args.phase_clocks:
        run_phase_clocks(args)
    elif args.profile == "bpcg":
        profile_bpcg(args.prec)
    elif args.profile == "pcg":
        profile_pcg(args.prec)
    elif args.profile == "fpmr":
        profile_fpmr(args.prec)
    elif args.profile == "fixed_pattern":
        profile_fixed_pattern()
    elif args.profile:
        profile_case(args.profile, args.prec)
    elif args.workload == "batch64" and args.impl == "ours":
        run_batch(args)
    elif args.workload == "aniso1024" and args.impl == "ours":
        run_aniso(args)
    elif args.workload == "fpmr" and args.impl == "ours":
        run_fpmr(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
