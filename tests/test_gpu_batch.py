"""Multi-instance batches (ls_batch_*) on the GPU.

* The batched apply runs the same per-cell arithmetic as each plan's own apply
  (shared kernel bodies, one right-hand side per instance), so it must equal the
  instances' single applies bit for bit, FP64 and complex64.
* The lock-step batch solve must reproduce each instance's own solve (same
  Arnoldi per instance; only the mixed refinement's inner tolerance, taken over
  all instances, differs): 1e-9 relative at tol 1e-11.
* One instance is small enough for the CPU oracle: the batch solution of that
  instance matches the oracle's GMRES on its accelerated operator to 1e-9.
"""
import numpy as np
import pytest

import workloads as W
from oracle.accel import AcceleratedOperator
from oracle.geometry import Discretisation
from oracle.gmres import gmres

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _instances():
    disc = W.place_cells(W.disc(level=2, kappa=2.0, n2c=2.0, collar_w=0.6, tau0=0.3, tau1=0.95, R_a=4, R_b=4,
                                R_cart=5, n_rho=48, N_tau=64), L=8, m=6, N_eq=8)
    kite = W.place_cells(W.kite(n1=512, n2=17, h=0.025, kappa=6.0, collar_w=0.07, tau0=0.4, tau1=0.9, R_a=6,
                                R_b=5, R_cart=4, n_rho=32, N_tau=48), L=17, m=8, center=(-0.25, 0.0), N_eq=8)
    small = W.scatterer("kite", 0.6, 9.0, 6000)
    return [disc, kite, small]


@pytest.fixture(scope="module")
def batch():
    from paper_1509_05063_gb300 import Batch, Plan
    wls = _instances()
    plans = [Plan(wl, W.n2_of(wl)) for wl in wls]
    b = Batch(plans)
    yield wls, plans, b
    b.close()


def test_offsets_concatenate_the_instances(batch):
    _, plans, b = batch
    assert b.offsets[0] == 0
    assert list(np.diff(b.offsets)) == [p.N for p in plans]


@pytest.mark.parametrize("prec_name", ["fp64", "mixed"])
def test_batch_apply_equals_single_applies(batch, prec_name):
    from paper_1509_05063_gb300 import LS_FP64, LS_MIXED
    _, plans, b = batch
    prec = LS_FP64 if prec_name == "fp64" else LS_MIXED
    dt = torch.complex128 if prec == LS_FP64 else torch.complex64
    u = torch.from_numpy(W.random_density(b.N, seed=W.SEED + 21)[0]).to("cuda:0", dt)
    for _ in range(3):                         # direct, captured, replayed
        got = b.apply(u, prec=prec)
        parts = b.split(got)
        for p, ui, gi in zip(plans, b.split(u), parts):
            ref = p.apply(ui.contiguous(), prec=prec)
            assert torch.equal(gi, ref)


@pytest.mark.parametrize("prec_name", ["fp64", "mixed", "mixed32"])
def test_batch_solve_matches_single_solves(batch, prec_name):
    from paper_1509_05063_gb300 import LS_FP64, LS_MIXED, LS_MIXED32
    wls, plans, b = batch
    prec = {"fp64": LS_FP64, "mixed": LS_MIXED, "mixed32": LS_MIXED32}[prec_name]
    parts = []
    for wl, p in zip(wls, plans):
        xy, _ = p.nodes()
        parts.append(W.plane_wave(wl.kappa, (1.0, 0.0), xy))
    uinc = torch.from_numpy(np.concatenate(parts)).to("cuda:0")
    sol, info = b.solve(uinc, tol=1e-11, prec=prec)
    assert info["converged"] and info["residual"] <= 1e-11
    assert all(r["residual"] <= 1e-11 for r in info["per_instance"])
    for p, ui, si in zip(plans, b.split(uinc), b.split(sol)):
        ref, rinfo = p.solve(ui.contiguous(), tol=1e-11, prec=prec)
        assert rinfo["converged"]
        err = torch.linalg.vector_norm(si - ref) / torch.linalg.vector_norm(ref)
        assert float(err) < 1e-9


def test_batch_solution_matches_oracle(batch):
    from paper_1509_05063_gb300 import LS_MIXED
    wls, plans, b = batch
    parts = []
    for wl, p in zip(wls, plans):
        xy, _ = p.nodes()
        parts.append(W.plane_wave(wl.kappa, (0.6, 0.8), xy))
    sol, info = b.solve(torch.from_numpy(np.concatenate(parts)).to("cuda:0"), tol=1e-12, prec=LS_MIXED)
    assert info["converged"]
    dz = Discretisation(wls[0])
    op = AcceleratedOperator(dz)
    ui = W.plane_wave(wls[0].kappa, (0.6, 0.8), dz.x)
    ref, _, _ = gmres(op.apply, ui, tol=1e-13, restart=200)
    _, canon = plans[0].nodes()
    got = b.split(sol)[0].cpu().numpy()
    assert np.linalg.norm(got - ref[canon]) / np.linalg.norm(ref) < 1e-9
