"""GPU test of ls_apply_noalloc, the apply variant for callers that must not
allocate device memory (stream capture, foreign memory pools, allocator-free
loops).  Its work arrays live in a fixed device array inside the library; the
result must equal the regular ls_apply's, on two calls in a row (the second
call reuses the array the first one left behind).  Collected last on purpose:
if it fails, a run that stops at the first failure has run every other test."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _disc():
    return W.place_cells(W.disc(level=2, kappa=2.0, n2c=2.0, collar_w=0.6, tau0=0.3, tau1=0.95, R_a=4, R_b=4,
                                R_cart=5, n_rho=48, N_tau=64), L=8, m=6, N_eq=8)


def _kite():
    # collar cells of several hundred nodes: the whole-cell projection path of
    # this entry point runs far past one 128-node piece
    return W.place_cells(W.kite(n1=512, n2=17, h=0.025, kappa=6.0, collar_w=0.07, tau0=0.4, tau1=0.9, R_a=6,
                                R_b=5, R_cart=4, n_rho=32, N_tau=48), L=17, m=8, center=(-0.25, 0.0), N_eq=8)


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("shape", ["disc", "kite"])
@pytest.mark.parametrize("prec_name", ["fp64", "mixed"])
def test_noalloc_apply_matches_apply_on_two_calls(prec_name, shape):
    from paper_1509_05063_gb300 import LS_FP64, LS_MIXED, Plan
    prec = LS_FP64 if prec_name == "fp64" else LS_MIXED
    dt = torch.complex128 if prec == LS_FP64 else torch.complex64
    tol = 1e-12 if prec == LS_FP64 else 1e-5      # the parity tolerances of the apply tests
    wl = _disc() if shape == "disc" else _kite()
    plan = Plan(wl, W.n2_of(wl))
    if shape == "kite":
        xy, _ = plan.nodes()
        ij = np.floor((xy - [wl.box_x0, wl.box_y0]) / wl.H).astype(np.int64)
        assert np.bincount(ij[:, 1] * wl.L + ij[:, 0]).max() > 256
    us = W.random_density(plan.N, nrhs=2)
    out = torch.empty(plan.N, dtype=dt, device="cuda:0")
    for r in range(2):
        u = torch.from_numpy(us[r]).to("cuda:0", dt)
        ref = plan.apply(u, prec=prec).cpu().numpy()
        got = plan.apply_noalloc(u, out, prec=prec).cpu().numpy()
        assert rel(got, ref) <= tol
    plan.close()


def test_noalloc_apply_rejects_plans_beyond_the_fixed_array():
    from paper_1509_05063_gb300 import LS_FP64, LSError, Plan
    wl = W.place_cells(W.kite(n1=512, n2=17, h=0.025, kappa=6.0, collar_w=0.07, tau0=0.4, tau1=0.9, R_a=6,
                              R_b=5, R_cart=4, n_rho=32, N_tau=48), L=17, m=8, center=(-0.25, 0.0), N_eq=31)
    plan = Plan(wl, W.n2_of(wl))
    assert plan.info["fft_M"] == 2048
    u = torch.zeros(plan.N, dtype=torch.complex128, device="cuda:0")
    with pytest.raises(LSError, match="fixed device array"):
        plan.apply_noalloc(u, torch.empty_like(u), prec=LS_FP64)
    plan.close()
