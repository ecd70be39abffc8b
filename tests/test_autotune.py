"""CPU checks of the layout autotuner and of the native cell-layout check."""
import numpy as np
import pytest

import workloads as W


def test_check_cells_matches_plan_and_rejects_small_cells():
    from paper_1509_05063_gb300 import HostPlan
    from paper_1509_05063_gb300.ls import check_cells
    wl = W.cfg1()
    st = check_cells(wl, W.n2_of(wl))
    assert st["ok"] and st["L"] == wl.L and st["M"] == 256
    hp = HostPlan(wl, W.n2_of(wl))
    assert st["N"] == hp.N
    bad = wl.replace(H=3 * wl.h, L=0)
    st = check_cells(bad, W.n2_of(bad))
    assert not st["ok"] and "3 x 3" in st["error"]


def test_autotune_picks_cheapest_admissible_layout():
    from paper_1509_05063_gb300 import HostPlan, autotune
    wl = W.cfg1()
    best, report = autotune.tune(wl, W.n2_of(wl), target_eps=1e-9, m_values=range(4, 16))
    ok = [r for r in report if r["ok"]]
    assert ok and any(not r["ok"] for r in report)          # small cells are rejected
    assert min(r["model_ms"] for r in ok) == [r for r in ok if r["wl"] is best][0]["model_ms"]
    hp = HostPlan(best, W.n2_of(best))                       # the chosen layout builds
    assert hp.N > 0 and best.N_eq == 8 and best.n_fb == 15


def test_auto_box_covers_nodes_with_faces_off_grid():
    from paper_1509_05063_gb300.ls import check_cells
    wl = W.cfg1().replace(L=0)
    st = check_cells(wl, W.n2_of(wl))
    assert st["ok"]
    off = (st["box_x0"] - wl.cart_x0) / wl.h
    assert abs(off - round(off - 0.5) - 0.5) < 1e-9
