#!/usr/bin/env python
"""Benchmark: LS matvecs/s and time to a 1e-10 solve, FP64 vs mixed, on one GB300.

Workload (config 2): kite x = cos t + 0.65 cos 2t - 0.65, y = 1.5 sin t,
n^2 = 1.5 + 0.5 exp(-|x|^2 / 0.1) inside, kappa = 20, ~274k Nystrom nodes,
1024 x 1024 padded lattice FFT, synthetic seeded data.

A step is one application of the whole hot path (equivalent-source projection,
lattice FFT convolution, local expansion, near-field correction, assembly) to
one right-hand side already resident in HBM.  ``value`` is FP64 matvecs/s over
all ranks (replicas: one independent plan per GPU, no collectives).  ``e2e``
times the same through the public API with the input copied from pinned host
memory and the result read back every step.  The mixed (complex64) apply and
the time to a 1e-10 solve with each path are reported beside it.

``--impl reference`` times the CPU oracle (direct O(N^2) Nystrom sum, plain
FP64 numpy) on a bounded sample of rows of the same operator.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "LS matvecs/s and time to 1e-10 solve at N, mixed vs FP64 path, 1 GB300"
FALLBACK_HBM_GBS = 6800.0
FALLBACK_BF16_TFLOPS = 1900.0
KERNELS_PER_APPLY = 6    # projection, source rows (fill + row FFT), columns (FFT, product, inverse),
#                          inverse rows, local coefficients, near field + assembly
# DRAM bytes (read + write) per launch of the near-field kernels on the full-size kite
# (358 205 610 near-field entries), from the ncu capture of the half-resolution kite
# summarised in profiles/near_field_kite_dram.md, scaled to the full launch by the
# ratio of algorithmic bytes (DRAM / algorithmic there: FP64 1.017, complex64 1.005,
# tensor cores 1.030).  Keyed by the plan's near-field entry count and by kernel:
# another workload, or a kernel changed since the capture (remove its entry then),
# reports null.
NEAR_TRAFFIC = {358205610: {"fp64": 8.892e9, "mixed": 2.955e9, "tc16": 3.106e9}}


def apply_bytes(info, cb, wb=None):
    """Algorithmic HBM bytes of one single-RHS 2-D apply of a plan (cb bytes per
    complex, wb per near-field weight): the near field (weights once, u, Phi,
    gamma, metadata, out), the projection's input and staged forms, and the
    lattice passes (source rows, quarter spectra, kept rows; each read and
    written once)."""
    N, nnz, nfb2, nocc = info["N"], info["nnz_near"], 2 * info["n_fb"] + 1, info["n_cells_occupied"]
    M, n_lat = info["fft_M"], info["L"] * info["N_eq"] + 1
    near = nnz * (wb or cb) + N * cb + N * nfb2 * cb + N * 12 + nocc * nfb2 * cb + N * cb
    lattice = 2 * (info["L"] + 1) * M * cb * 2 + 2 * (M // 2 + 1) ** 2 * cb + 2 * n_lat * M * cb * 2
    return near + N * cb * 4 + lattice


def hbm_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            d = json.load(open(p))
            for k in ("hbm_gbs", "hbm_GBs", "hbm_copy_gbs"):
                if k in d:
                    return float(d[k]), "measured"
        except Exception:
            pass
    return FALLBACK_HBM_GBS, "fallback"


def fp16_peak():
    """Dense FP16/BF16 tensor peak (kind::f16 runs FP16 at the BF16 rate): the
    measured burst figure of MEASURED_PEAKS.json, else the recipe's fallback."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            d = json.load(open(p))
            if "bf16_tflops" in d:
                return float(d["bf16_tflops"]), "measured (bf16 cuBLAS burst, the FP16 dense rate)"
        except Exception:
            pass
    return FALLBACK_BF16_TFLOPS, "fallback"


class Clocks:
    """nvidia-smi sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
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
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            self.proc.wait()

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) < 9:
                    continue
                try:
                    sm.append(float(f[1]))
                    smax.append(float(f[2]))
                except ValueError:
                    continue
                for n, v in zip(names, f[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(n)
        except Exception:
            pass
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_info():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def replica_rate(local_ms: float, local_units: int, device="cpu"):
    """Whole-job throughput of independent replicas: the units processed by all
    ranks over the slowest rank's time.  Returns (units / s, max ms, total units).
    Single process when torch.distributed is not initialised."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return local_units / (local_ms * 1e-3), local_ms, local_units
    t = torch.tensor([float(local_ms)], dtype=torch.float64, device=device)
    n = torch.tensor([float(local_units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(n, op=dist.ReduceOp.SUM)
    ms, units = float(t.item()), float(n.item())
    return units / (ms * 1e-3), ms, units


_ORACLE = {}


def _oracle_worker_init(wl):
    """Spawned worker: build the oracle's direct operator of the workload once."""
    import workloads as W
    from oracle.geometry import Discretisation
    from oracle.operator import DirectOperator
    dz = Discretisation(wl)
    _ORACLE["op"] = DirectOperator(dz, dense_limit=0)
    _ORACLE["u"] = W.random_density(dz.N)[0]


def _oracle_worker_rows(rows):
    """Direct O(N^2) apply on these rows (64 at a time); returns (rows done, seconds)."""
    t0 = time.perf_counter()
    for s in range(0, len(rows), 64):
        _ORACLE["op"].apply(_ORACLE["u"], rows=rows[s:s + 64])
    return len(rows), time.perf_counter() - t0


class OraclePool:
    """The CPU oracle on the host's cores: one spawned process per core (each
    single-threaded), every process holding the workload's direct operator.
    A step splits its rows evenly over the processes; its time is the wall time
    of the whole split, so rows/s counts every core."""

    def __init__(self, wl, procs: int | None = None):
        import multiprocessing as mp
        self.procs = procs or os.cpu_count() or 1
        for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            os.environ[k] = "1"      # the spawned workers read these at start: one core each
        self.pool = mp.get_context("spawn").Pool(self.procs, initializer=_oracle_worker_init, initargs=(wl,))
        import workloads as W
        self.N = None
        self.W = W

    def run(self, rows):
        import numpy as np
        parts = [p for p in np.array_split(np.asarray(rows), self.procs) if len(p)]
        t0 = time.perf_counter()
        done = sum(r for r, _ in self.pool.map(_oracle_worker_rows, parts, chunksize=1))
        return done, time.perf_counter() - t0

    def close(self):
        self.pool.close()
        self.pool.join()


def cpu_oracle_rate(wl, n_rows: int, procs: int | None = None):
    """The oracle's direct O(N^2) apply on n_rows seeded rows, split over all
    host cores: returns (matvecs/s extrapolated from rows/s, rows, seconds, N,
    processes)."""
    import workloads as W
    from oracle.geometry import Discretisation
    N = Discretisation(wl).N
    pool = OraclePool(wl, procs)
    try:
        pool.run(W.random_rows(N, pool.procs, seed=W.SEED + 2))   # every worker built and warm
        done, dt = pool.run(W.random_rows(N, n_rows))
    finally:
        pool.close()
    return (done / dt) / N, done, dt, N, pool.procs


def run_reference(args):
    rank, world, _ = dist_info()
    if rank != 0:
        return 0
    import workloads as W
    from oracle.geometry import Discretisation
    wl = W.cfg2()
    N = Discretisation(wl).N
    pool = OraclePool(wl)
    rows_per_step = args.ref_rows * pool.procs
    rows_all = W.random_rows(N, rows_per_step * (args.steps + args.warmup))
    try:
        for s in range(args.warmup):
            pool.run(rows_all[s * rows_per_step:(s + 1) * rows_per_step])
        dt = 0.0
        for s in range(args.warmup, args.warmup + args.steps):
            dt += pool.run(rows_all[s * rows_per_step:(s + 1) * rows_per_step])[1]
    finally:
        pool.close()
    rate = (args.steps * rows_per_step / dt) / N
    sample = (f"{rows_per_step} seeded rows x all N sources per step ({args.ref_rows} per process, "
              f"{pool.procs} single-threaded processes), extrapolated to N rows")
    line = {
        "impl": "reference", "metric": METRIC, "value": rate, "unit": "matvecs/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"cfg2 kite kappa=20 N={N}", "N": N, "sample": sample},
        "cpu_baseline": {"value": rate, "unit": "matvecs/s", "cores": pool.procs, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": rate, "unit": "matvecs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_batch(n_inst, dev, barrier, timed):
    """Reduced config 3: n_inst seeded discs / kites (scale in [0.5, 1], kappa in
    [5, 20], N log-uniform in [2e4, 1.2e5]) with autotuned layouts, as one
    multi-instance batch: apply throughput (instance-matvecs/s) and the mixed
    lock-step solve to 1e-10, against the instances' own applies and solves."""
    import numpy as np
    import torch
    import workloads as W
    from paper_1509_05063_gb300 import LS_FP64, LS_MIXED, Batch, Plan, autotune
    insts = W.cfg3_instances(n_inst, N_lo=2e4, N_hi=1.2e5, scale_range=(0.5, 1.0), kappa_range=(5.0, 20.0))
    t0 = time.perf_counter()
    plans = []
    for wl in insts:
        tw, _ = autotune.tune(wl, W.n2_of(wl), target_eps=1e-9)
        plans.append(Plan(tw, W.n2_of(tw)))
    t_plan = time.perf_counter() - t0
    b = Batch(plans)
    out = {"instances": n_inst, "N_total": b.N, "N_each": [p.N for p in plans],
           "kappa_each": [round(wl.kappa, 3) for wl in insts], "shape_each": [wl.shape for wl in insts],
           "plan_s_total": t_plan, "plan_s_each": [round(p.info["plan_seconds"], 3) for p in plans],
           "plan_stage_s_total": {k: round(sum(p.info["stage_seconds"][k] for p in plans), 3)
                                  for k in ("nodes", "near", "accel", "device")}}
    steps = 20
    for prec, dt, key in [(LS_FP64, torch.complex128, "fp64"), (LS_MIXED, torch.complex64, "mixed")]:
        u = torch.from_numpy(W.random_density(b.N)[0]).to(dev, dt)
        o = torch.empty_like(u)
        for _ in range(3):
            b.apply(u, o, prec=prec)
        ms_b = timed(lambda: b.apply(u, o, prec=prec), steps)
        pu = [x.contiguous() for x in b.split(u)]
        po = [torch.empty_like(x) for x in pu]

        def seq():
            for p, x, y in zip(plans, pu, po):
                p.apply(x, y, prec=prec)
        for _ in range(3):
            seq()
        ms_s = timed(seq, steps)
        out[key] = {"batch_apply_ms": ms_b / steps, "instance_matvecs_per_s": n_inst * steps / (ms_b * 1e-3),
                    "separate_applies_ms": ms_s / steps}
        if key == "mixed":
            peak, _ = hbm_peak()
            nbytes = sum(apply_bytes(p.info, 8) for p in plans)
            out[key]["apply_hbm_frac"] = (nbytes / (ms_b / steps * 1e-3) / 1e9) / peak
    parts = []
    for wl, p in zip(insts, plans):
        xy, _ = p.nodes()
        parts.append(W.plane_wave(wl.kappa, wl.inc_dir, xy))
    ui = torch.from_numpy(np.concatenate(parts)).to(dev)
    b.solve(ui, tol=1e-3, prec=LS_MIXED, max_iter=3)
    barrier()
    t0 = time.perf_counter()
    _, info = b.solve(ui, tol=1e-10, prec=LS_MIXED, max_iter=4000, restart=100)
    barrier()
    t_b = time.perf_counter() - t0
    t0 = time.perf_counter()
    for p, x in zip(plans, b.split(ui)):
        p.solve(x.contiguous(), tol=1e-10, prec=LS_MIXED, max_iter=4000, restart=100)
    barrier()
    t_s = time.perf_counter() - t0
    out["solve_mixed"] = {"tol": 1e-10, "restart": 100, "makespan_s": t_b, "separate_solves_s": t_s,
                          "converged": info["converged"], "residual": info["residual"],
                          "iterations_each": [r["iterations"] for r in info["per_instance"]]}
    b.close()
    for p in plans:
        p.close()
    return out


def run_sphere(spec, dev, barrier, timed, steps):
    """Reduced config 4: the penetrable sphere of Section 5 (radius 1, n^2 = 1.5
    inside, kappa = 8, plane wave exp(i kappa x_3)) on a coarser ball than the
    config's ~2M nodes; spec = (n_f, n_s, h, L, N_eq): shell face points, depth
    lines, interior spacing, cells per axis of the box [-1.13, 1.13]^3, lattice
    intervals per cell.  Device apply rates (FP64, complex64) and the time to a
    1e-10 FP64 residual with the FP64 solve and with mixed precision, plus the
    solution's error against the Mie series."""
    import numpy as np
    import torch
    from oracle import exact
    from paper_1509_05063_gb300 import LS_FP64, LS_MIXED, LS_MIXED32, Plan3
    n_f, n_s, h, L, Ne = spec
    kappa, n2, half = 8.0, 1.5, 1.13
    t0 = time.perf_counter()
    plan = Plan3(lambda x: np.full(len(x), n2), kappa, [-half] * 3, 2 * half / L, L, Ne,
                 ball=dict(n_f=n_f, n_s=n_s, h=h), rules=dict(rc=3.0, rs=3.0))
    t_plan = time.perf_counter() - t0
    xyz, _ = plan.nodes()
    N = plan.N
    u = torch.from_numpy(__import__("workloads").random_density(N)[0]).to(dev)
    u32 = u.to(torch.complex64)
    o, o32 = torch.empty_like(u), torch.empty_like(u32)
    for _ in range(3):
        plan.apply(u, o, prec=LS_FP64)
        plan.apply(u32, o32, prec=LS_MIXED)
    ms64 = timed(lambda: plan.apply(u, o, prec=LS_FP64), steps)
    ms32 = timed(lambda: plan.apply(u32, o32, prec=LS_MIXED), steps)
    ui = torch.from_numpy(np.exp(1j * kappa * xyz[:, 2])).to(dev)
    plan.solve(ui, tol=1e-3, prec=LS_FP64, max_iter=3)
    plan.solve(ui, tol=1e-3, prec=LS_MIXED, max_iter=3)
    out = {"workload": f"sphere a=1 n^2={n2} kappa={kappa} N={N} (n_f={n_f}, n_s={n_s}, h={h}), "
                       f"L={L} cells/axis, N_eq={Ne}, lattice M={plan.info['fft_M']}",
           "N": N, "nnz_near": plan.info["nnz_near"], "plan_s": t_plan, "plan_stage_s": plan.info["stage_seconds"],
           "fp64_matvecs_per_s": steps / (ms64 * 1e-3), "mixed_matvecs_per_s": steps / (ms32 * 1e-3)}
    ue = exact.sphere_total_field(kappa, n2, 1.0, xyz)
    sols = {}
    for name, prec, restart in (("fp64", LS_FP64, 100), ("mixed", LS_MIXED, 30), ("mixed32", LS_MIXED32, 30)):
        barrier()
        t0 = time.perf_counter()
        sol, info = plan.solve(ui, tol=1e-10, prec=prec, max_iter=2000, restart=restart)
        barrier()
        sols[name] = sol
        out[name] = {"time_to_1e-10_s": time.perf_counter() - t0, "iterations": info["iterations"],
                     "refinements": info["refinements"], "residual": info["residual"],
                     "converged": info["converged"], "restart": restart}
    s64 = sols["fp64"].cpu().numpy()
    out["mixed_vs_fp64_solution_rel"] = float(np.linalg.norm(sols["mixed"].cpu().numpy() - s64) / np.linalg.norm(s64))
    out["fp64_vs_mie_rel_l2"] = float(np.linalg.norm(s64 - ue) / np.linalg.norm(ue))
    out["mixed_speedup_time_to_tol"] = out["fp64"]["time_to_1e-10_s"] / out["mixed"]["time_to_1e-10_s"]
    plan.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-solve", action="store_true")
    ap.add_argument("--cpu-rows", type=int, default=4096)
    ap.add_argument("--ref-rows", type=int, default=24, help="oracle rows per process and step")
    ap.add_argument("--autotune", action="store_true",
                    help="pick the cell layout with the autotuner (model + GPU timing of the best 3)")
    ap.add_argument("--directions", type=int, default=16,
                    help="incident directions of the lock-step mixed solve (theta_j = 2 pi j / D)")
    ap.add_argument("--batch", type=int, default=12,
                    help="also time a multi-instance batch of this many seeded scatterers (reduced config 3)")
    ap.add_argument("--sphere", default="49,17,0.05,14,4",
                    help="reduced config 4 (penetrable sphere, kappa = 8): n_f,n_s,h,L,N_eq; 'none' to skip")
    ap.add_argument("--scale", type=int, default=1,
                    help="coarsen config 2 by this factor (h, cells) for profiling captures")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)

    import numpy as np
    import torch
    import workloads as W
    from paper_1509_05063_gb300 import LS_FP64, LS_MIXED, LS_MIXED32, Plan
    from paper_1509_05063_gb300.ls import measure_peaks

    rank, world, local = dist_info()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    sc = args.scale
    wl = W.cfg2(h=0.0045 * sc, n1=3200 // sc)
    if sc > 1:
        wl = wl.replace(L=0)          # the plan places the box around the coarser node set
    if args.autotune:
        from paper_1509_05063_gb300 import autotune
        wl, _ = autotune.tune(wl, W.n2_of(wl), target_eps=1e-9, measure_top=3)
    plan = Plan(wl, W.n2_of(wl))
    # kernel variants of this plan (lattice column-pass width, complex64 RHS
    # group and near-field unit) timed on this GPU; the fastest is kept
    kernel_tune = plan.autotune(16)
    info = plan.info
    N = plan.N
    u = torch.from_numpy(W.random_density(N, seed=W.SEED + rank)[0]).to(dev)
    u32 = u.to(torch.complex64)
    out = torch.empty_like(u)
    out32 = torch.empty_like(u32)

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    def timed(fn, steps):
        """max over ranks of the CUDA-event time of `steps` calls (ms)."""
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            fn()
        e1.record()
        barrier()
        return replica_rate(e0.elapsed_time(e1), steps, device=dev)[1]

    f64 = lambda: plan.apply(u, out, prec=LS_FP64)
    f32 = lambda: plan.apply(u32, out32, prec=LS_MIXED)
    # batched right-hand sides: one pass over the near-field weights serves all of them
    NB32, NB64 = 16, 4      # complex64: 16 RHS take the tensor-core near field
    ub32 = torch.from_numpy(W.random_density(N, nrhs=NB32, seed=W.SEED + 3 + rank)).to(dev, torch.complex64)
    ob32 = torch.empty_like(ub32)
    ub64 = torch.from_numpy(W.random_density(N, nrhs=NB64, seed=W.SEED + 5 + rank)).to(dev)
    ob64 = torch.empty_like(ub64)
    fb32 = lambda: plan.apply(ub32, ob32, prec=LS_MIXED)
    fb64 = lambda: plan.apply(ub64, ob64, prec=LS_FP64)
    for _ in range(args.warmup):
        f64()
        f32()
        fb32()
        fb64()
    peaks = measure_peaks()          # FP64 FMA and TF32 tensor-core probes (outside the timed region)
    with Clocks(local) as clk:
        ms64 = timed(f64, args.steps)
        ms32 = timed(f32, args.steps)
        msb32 = timed(fb32, max(args.steps // 4, 3))
        msb64 = timed(fb64, max(args.steps // 4, 3))
    clocks = clk.summary()
    nb_steps = max(args.steps // 4, 3)

    # per-stage CUDA-event timing on the launch stream (roofline of the dominant kernel)
    plan.set_stage_timing(True)
    for _ in range(args.steps):
        f64()
    st64, c64 = plan.stage_times(LS_FP64)
    for _ in range(args.steps):
        f32()
    st32, c32 = plan.stage_times(LS_MIXED)
    plan.set_stage_timing(True)
    for _ in range(nb_steps):
        fb32()
    stb, cb = plan.stage_times(LS_MIXED)
    plan.set_stage_timing(False)

    # end to end through the public API: pinned host input in, result out, every step
    h_u = torch.from_numpy(W.random_density(N, seed=W.SEED + 7 + rank)[0]).pin_memory()
    h_out = torch.empty_like(h_u).pin_memory()
    d_u = torch.empty_like(u)

    def e2e_step():
        d_u.copy_(h_u, non_blocking=True)
        plan.apply(d_u, out, prec=LS_FP64)
        h_out.copy_(out, non_blocking=True)

    for _ in range(args.warmup):
        e2e_step()
    ms_e2e = timed(e2e_step, args.steps)

    # time to tolerance
    solve = None
    if not args.no_solve:
        xy, _ = plan.nodes()
        ui = torch.from_numpy(W.plane_wave(wl.kappa, wl.inc_dir, xy)).to(dev)
        plan.solve(ui, tol=1e-4, prec=LS_FP64, max_iter=5)      # allocate work space
        barrier()
        t0 = time.perf_counter()
        s64, i64 = plan.solve(ui, tol=1e-10, prec=LS_FP64, max_iter=800, restart=200)
        barrier()
        t64 = time.perf_counter() - t0
        t0 = time.perf_counter()
        s32, i32 = plan.solve(ui, tol=1e-10, prec=LS_MIXED, max_iter=800, restart=30)
        barrier()
        t32 = time.perf_counter() - t0
        diff = float(torch.linalg.vector_norm(s32 - s64) / torch.linalg.vector_norm(s64))
        # block right-hand sides: D incident directions theta_j = 2 pi j / D in lock-step (batches of 8)
        D = args.directions
        th = [2 * math.pi * j / D for j in range(D)]
        UI = torch.from_numpy(np.stack([W.plane_wave(wl.kappa, (math.cos(t), math.sin(t)), xy) for t in th])).to(dev)
        barrier()
        t0 = time.perf_counter()
        sb32, ib32 = plan.solve(UI, tol=1e-10, prec=LS_MIXED, max_iter=800, restart=30)
        barrier()
        tb32 = time.perf_counter() - t0
        # LS_MIXED32: complex64 Arnoldi vectors in the correction solves as well
        t0 = time.perf_counter()
        s3, i3 = plan.solve(ui, tol=1e-10, prec=LS_MIXED32, max_iter=800, restart=30)
        barrier()
        t3 = time.perf_counter() - t0
        t0 = time.perf_counter()
        sb3, ib3 = plan.solve(UI, tol=1e-10, prec=LS_MIXED32, max_iter=800, restart=30)
        barrier()
        tb3 = time.perf_counter() - t0
        solve = {"tol": 1e-10, "restart_fp64": 200, "restart_mixed": 30, "fp64_s": t64, "fp64_iterations": i64["iterations"],
                 "fp64_residual": i64["residual"], "fp64_converged": i64["converged"],
                 "mixed_s": t32, "mixed_inner_iterations": i32["iterations"],
                 "mixed_refinements": i32["refinements"], "mixed_residual": i32["residual"],
                 "mixed_converged": i32["converged"], "mixed_vs_fp64_solution_rel": diff,
                 "directions": D, "mixed_block_s": tb32, "mixed_block_per_rhs_s": tb32 / D,
                 "mixed_block_converged": ib32["converged"], "mixed_block_residual": ib32["residual"],
                 "mixed_block_inner_iterations": ib32["iterations"],
                 "mixed32_s": t3, "mixed32_inner_iterations": i3["iterations"], "mixed32_residual": i3["residual"],
                 "mixed32_converged": i3["converged"], "mixed32_block_s": tb3,
                 "mixed32_block_converged": ib3["converged"], "mixed32_block_residual": ib3["residual"]}

    batch = run_batch(args.batch, dev, barrier, timed) if args.batch > 0 else None
    sphere = None
    if args.sphere != "none":
        f = args.sphere.split(",")
        sphere = run_sphere((int(f[0]), int(f[1]), float(f[2]), int(f[3]), int(f[4])), dev, barrier, timed,
                            max(args.steps // 2, 3))

    # roofline of the dominant kernel (near field + local evaluation + assembly)
    nnz = info["nnz_near"]
    nfb2 = 2 * info["n_fb"] + 1
    nocc = info["n_cells_occupied"]

    def near_bytes(cb, wb=None):   # algorithmic bytes of one k_near_eval launch, cb = bytes per complex,
        # wb = bytes per block weight (complex128 also reads Re + Im of each weight: 24 B):
        # dense per-cell weight blocks (+ the tiny CSR remainder, counted as blocks), u, Phi, gamma, out
        return nnz * (wb or cb) + N * cb + N * nfb2 * cb + N * 12 + nocc * nfb2 * cb + N * cb

    peak, peak_src = hbm_peak()
    traffic = NEAR_TRAFFIC.get(nnz, {})
    fp64_peak = peaks["fp64"]
    # FP16 work the tensor-core near field issues per launch (kind::f16, split
    # operands): per complex weight (2 real K entries) an MMA of N = 4R
    # (A_hi against B_hi | B_lo) and one of N = 2R (A_lo against B_hi), 2 flops each
    nchunk_cols = nnz              # close to the padded count (rows padded to 8 add < 3 %)
    G32 = min(NB32, kernel_tune["group32"])       # RHS per near-field launch (autotuned)
    tc_used = kernel_tune["near_cuda32"] == 0 and G32 >= 8
    tc_flops = nchunk_cols * 2 * 2 * (4 * G32 + 2 * G32)
    f16_peak, f16_src = fp16_peak()
    # FP64 flops of one launch: 3 FMAs per block weight (three-multiplication
    # complex product), 4 per Phi-gamma term
    near_flops = nnz * 6 + N * nfb2 * 8
    t_near64 = st64[4] / max(c64, 1) * 1e-3
    t_near32 = st32[4] / max(c32, 1) * 1e-3
    ach64 = near_bytes(16, 24) / t_near64 / 1e9
    ach32 = near_bytes(8) / t_near32 / 1e9
    M = info["fft_M"]
    n_lat = info["L"] * info["N_eq"] + 1
    # whole-apply byte model: u in, out, weights, projections, Phi, lattice passes, quarter spectra
    lat_bytes = lambda cb: (2 * (info["L"] + 1) * M * cb * 2 + 2 * (M // 2 + 1) ** 2 * cb
                            + 2 * n_lat * M * cb * 2)
    apply_bytes64 = apply_bytes(info, 16, 24)
    apply_bytes32 = apply_bytes(info, 8)
    # batched complex64 (tensor-core near field): weights once, per-RHS vectors, Phi once
    near_bytes_b = nnz * 8 + N * nfb2 * 8 + N * 12 + G32 * (2 * N * 8 + nocc * nfb2 * 8)
    t_near_b = stb[4] / max(cb, 1) * 1e-3
    ach_b = near_bytes_b / t_near_b / 1e9
    # whole batched apply: near field + per-RHS projection input, lattice passes and spectra
    apply_bytes_b = near_bytes_b * (NB32 // G32) + NB32 * (N * 8 + lat_bytes(8))
    stage_names = ["es_project", "lattice_fill(fused)", "lattice_fft_conv", "local_coeffs", "near_eval"]

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, nrows, dt, n, procs = cpu_oracle_rate(wl, args.cpu_rows)
        cpu = {"value": rate, "unit": "matvecs/s", "cores": procs, "kind": "oracle",
               "sample": f"{nrows} seeded rows of the direct O(N^2) FP64 apply split over {procs} "
                         f"single-threaded processes ({dt:.1f} s), extrapolated to all {n} rows"}

    value = world * args.steps / (ms64 * 1e-3)
    line = {
        "metric": METRIC, "value": value, "unit": "matvecs/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms64 / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"cfg2 kite kappa=20 N={N}",
                   "N": N, "nnz_near": nnz, "fft_M": M, "L": info["L"], "N_eq": info["N_eq"],
                   "n_fb": info["n_fb"], "parallelism": f"replicas x{world}",
                   "l2": "inputs larger than L2 (FP64 near-field weights %.1f GB)" % (nnz * 24 / 1e9),
                   "plan_seconds": info["plan_seconds"], "plan_stage_seconds": info["stage_seconds"],
                   "device_bytes": info["device_bytes"]},
        "e2e": {"value": world * args.steps / (ms_e2e * 1e-3), "unit": "matvecs/s",
                "h2d_bytes_per_step": N * 16, "d2h_bytes_per_step": N * 16},
        "roofline": {"bound": "alu", "kernel": "k_near_eval5<double2,1>",
                     "achieved": near_flops / t_near64 / 1e12, "peak": fp64_peak, "unit": "TFLOP/s",
                     "frac": near_flops / t_near64 / 1e12 / fp64_peak, "traffic": traffic.get("fp64"),
                     "peak_source": "measured: ls_measure_peaks FP64 FMA probe (best of 8, 16 and 32 "
                                    "independent chains per thread, every SM, CUDA events), this run",
                     "flops_per_launch": near_flops, "bytes_per_launch": near_bytes(16, 24),
                     "hbm_GBs": ach64, "hbm_frac": ach64 / peak, "hbm_peak": peak, "hbm_peak_source": peak_src,
                     "launch_ms": t_near64 * 1e3},
        "gpu_launches": KERNELS_PER_APPLY * args.steps,
        "peaks_measured": {"fp64_tflops": peaks["fp64"], "tf32_tflops": peaks["tf32"],
                           "hbm_gbs": peak, "hbm_source": peak_src},
        "clocks": clocks,
        "mixed": {"value": world * args.steps / (ms32 * 1e-3), "unit": "matvecs/s", "dtype": "f32",
                  "ms_per_step": ms32 / args.steps,
                  "apply_hbm_frac": (apply_bytes32 / (ms32 / args.steps * 1e-3) / 1e9) / peak,
                  "roofline": {"bound": "hbm", "kernel": "k_near_eval<float2,1>", "achieved": ach32,
                               "peak": peak, "unit": "GB/s", "frac": ach32 / peak, "peak_source": peak_src,
                               "bytes_per_launch": near_bytes(8), "traffic": traffic.get("mixed"),
                               "launch_ms": t_near32 * 1e3}},
        "batched": {"unit": "RHS-matvecs/s",
                    "mixed": {"nrhs": NB32, "value": world * nb_steps * NB32 / (msb32 * 1e-3), "dtype": "f32",
                              "ms_per_apply": msb32 / nb_steps,
                              "roofline": dict({"bound": "hbm",
                                                "kernel": (f"k_near_tc<{G32}> (tcgen05 kind::f16, split FP16 operands)"
                                                           if tc_used else f"k_near_eval4<float2,{G32}> (CUDA cores)"),
                                                "achieved": ach_b, "peak": peak, "unit": "GB/s", "frac": ach_b / peak,
                                                "peak_source": peak_src, "bytes_per_launch": near_bytes_b,
                                                "traffic": traffic.get("tc16") if tc_used and G32 == 16 else None,
                                                "launch_ms": t_near_b * 1e3},
                                               **({"tensor_tflops": tc_flops / t_near_b / 1e12,
                                                   "tensor_peak": f16_peak,
                                                   "tensor_frac": tc_flops / t_near_b / 1e12 / f16_peak,
                                                   "tensor_peak_source": f16_src} if tc_used else {})),
                              "apply_hbm_frac": (apply_bytes_b / (msb32 / nb_steps * 1e-3) / 1e9) / peak,
                              "stages_ms": dict(zip(stage_names, [float(x) / max(cb, 1) for x in stb]))},
                    "fp64": {"nrhs": NB64, "value": world * nb_steps * NB64 / (msb64 * 1e-3), "dtype": "f64"}},
        "stages_ms": {"fp64": dict(zip(stage_names, [float(x) / max(c64, 1) for x in st64])),
                      "mixed": dict(zip(stage_names, [float(x) / max(c32, 1) for x in st32]))},
        "apply_hbm_frac_fp64": (apply_bytes64 / (ms64 / args.steps * 1e-3) / 1e9) / peak,
        "time_to_tol": solve,
        "kernel_autotune": kernel_tune,
    }
    if batch is not None:
        line["batch"] = batch
    if sphere is not None:
        line["sphere_3d"] = sphere
    if cpu is not None:
        line["cpu_baseline"] = cpu
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    plan.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
