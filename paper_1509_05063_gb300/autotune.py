"""Autotuner for the accelerator layout: cell side H = m h, box and N_eq.

For a workload (geometry, kappa, quadrature radii) and a target accuracy of
the accelerated far part it
  1. picks N_eq (equivalent-source lattice intervals per cell side) from the
     accuracy target (measured equivalent-source / local-fit error ~1e-9 at
     N_eq = 8, ~1e-11 at 12 for kappa H ~ 1);
  2. scans cell multiples m, letting the library choose the box (L = 0) and
     check, natively and without building the quadratures, that every node's
     cut-off support stays inside its 3 x 3 cell block, kappa H is admissible
     and the lattice FFT fits (ls_check_cells);
  3. ranks the valid layouts by a GB300 cost model of one complex64 apply:
     near-field block entries streamed from HBM plus the lattice passes, the
     per-cell equivalent-source / local-expansion work and a launch floor;
  4. optionally measures the best few layouts with real plans on the GPU and
     keeps the fastest.
"""
from __future__ import annotations

import math

from .ls import LS_MIXED, Plan, check_cells

HBM_BYTES_PER_S = 6.0e12      # sustained complex64 near-field stream (measured ~6.1 TB/s)
LAUNCH_FLOOR_S = 40e-6


def neq_for(target_eps: float) -> int:
    if target_eps >= 1e-7:
        return 6
    if target_eps >= 1e-9:
        return 8
    if target_eps >= 1e-11:
        return 12
    return 16


def model_seconds(stats: dict, N_eq: int) -> float:
    """Estimated seconds of one complex64 apply for a checked layout."""
    M, L, cells = stats["M"], stats["L"], stats["cells"]
    n_lat = L * N_eq + 1
    near = stats["block_entries"] * 8 + stats["N"] * 8 * (2 * (2 * N_eq - 1) + 4)
    lattice = 8 * (4 * (L + 1) * M + 2 * (M // 2 + 1) ** 2 + 4 * n_lat * M)
    per_cell = cells * (4 * (N_eq + 1)) * 8 * 64
    return (near + lattice + per_cell) / HBM_BYTES_PER_S + LAUNCH_FLOOR_S


def tune(wl, n2, target_eps: float = 1e-9, m_values=range(4, 41), measure_top: int = 0, verbose: bool = False):
    """Return (workload with the chosen layout, report list)."""
    N_eq = neq_for(target_eps)
    report = []
    for m in m_values:
        H = m * wl.h
        if wl.kappa * H / math.sqrt(2.0) >= 2.4:
            break
        cand = wl.replace(H=H, L=0, N_eq=N_eq, n_fb=2 * N_eq - 1)
        st = check_cells(cand, n2)
        if not st["ok"]:
            report.append({"m": m, "ok": False, "error": st["error"]})
            continue
        cand = cand.replace(L=st["L"], box_x0=st["box_x0"], box_y0=st["box_y0"])
        est = model_seconds(st, N_eq)
        report.append({"m": m, "ok": True, "H": H, "L": st["L"], "M": st["M"], "block_entries": st["block_entries"],
                       "model_ms": est * 1e3, "wl": cand})
        if verbose:
            print(f"m={m} H={H:.4f} L={st['L']} M={st['M']} entries={st['block_entries']:.3e} "
                  f"model={est * 1e3:.3f} ms")
    ok = sorted([r for r in report if r["ok"]], key=lambda r: r["model_ms"])
    if not ok:
        raise ValueError("no admissible cell layout: " + "; ".join(r.get("error", "") for r in report[:3]))
    best = ok[0]
    if measure_top > 0:
        import torch
        import numpy as np
        for r in ok[:measure_top]:
            plan = Plan(r["wl"], n2)
            u = torch.ones(plan.N, dtype=torch.complex64, device="cuda")
            out = torch.empty_like(u)
            for _ in range(3):
                plan.apply(u, out, prec=LS_MIXED)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(10):
                plan.apply(u, out, prec=LS_MIXED)
            e1.record()
            torch.cuda.synchronize()
            r["measured_ms"] = e0.elapsed_time(e1) / 10
            plan.close()
        best = min(ok[:measure_top], key=lambda r: r["measured_ms"])
    return best["wl"], report
