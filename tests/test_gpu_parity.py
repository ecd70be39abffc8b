"""GPU parity of the CUDA path (through the C ABI) against the CPU oracle.

Tolerances (written here, derived from the arithmetic):
* FP64 apply vs the oracle's accelerated operator (same algorithm, Section 3.2
  steps): 1e-12 relative (2-norm over all nodes).  Both sides are FP64; the
  differences are rounding in the lattice FFT / contractions and the two
  independent SVD factorisations of the equivalent-source fit (~1e-13).
* FP64 apply vs the oracle's direct operator (far part summed exactly): the
  acceleration error, ~1e-9 at N_eq = 8 (Tables accel1/accel2 magnitude);
  tested at 1e-8.
* complex64 apply vs FP64 oracle: 1e-5 relative (the mixed-precision bound).
* solves: FP64 GMRES to 1e-12 vs the oracle's GMRES on the same operator:
  1e-9 relative; mixed refinement must reach the FP64 residual 1e-10.
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import exact
from oracle.accel import AcceleratedOperator, Accelerator, Cells, near_matrix
from oracle.farfield import far_field
from oracle.geometry import Discretisation
from oracle.gmres import gmres
from oracle.operator import DirectOperator

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _small_disc():
    return W.place_cells(W.disc(level=2, kappa=2.0, n2c=2.0, collar_w=0.6, tau0=0.3, tau1=0.95, R_a=4, R_b=4,
                                R_cart=5, n_rho=48, N_tau=64), L=8, m=6, N_eq=8)


def _small_kite():
    return W.place_cells(W.kite(n1=512, n2=17, h=0.025, kappa=6.0, collar_w=0.07, tau0=0.4, tau1=0.9, R_a=6,
                                R_b=5, R_cart=4, n_rho=32, N_tau=48), L=17, m=8, center=(-0.25, 0.0), N_eq=8)


class Case:
    def __init__(self, wl):
        from paper_1509_05063_gb300 import Plan
        self.wl = wl
        self.plan = Plan(wl, W.n2_of(wl))
        self.xy, self.canon = self.plan.nodes()
        self.dz = Discretisation(wl)
        self.op = AcceleratedOperator(self.dz)
        self.u = W.random_density(self.dz.N, nrhs=3)

    def to_plan(self, v):
        return np.ascontiguousarray(v[..., self.canon])

    def dev(self, v, dtype=torch.complex128):
        return torch.from_numpy(self.to_plan(v)).to("cuda:0", dtype)


@pytest.fixture(scope="module")
def disc():
    return Case(_small_disc())


@pytest.fixture(scope="module")
def kite():
    return Case(_small_kite())


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def check_mixed(got, ref, tol=1e-5):
    """The complex64 bound, normwise AND element by element (a few bad rows,
    such as one broken tile, cannot hide under the 2-norm): max |got - ref|
    over max |ref| <= tol as well."""
    got = np.asarray(got).astype(np.complex128)
    assert rel(got, ref) < tol
    assert np.max(np.abs(got - ref)) <= tol * np.max(np.abs(ref))


@pytest.mark.parametrize("name", ["disc", "kite"])
def test_fp64_apply_matches_oracle_accelerated_operator(name, request):
    c = request.getfixturevalue(name)
    from paper_1509_05063_gb300 import LS_FP64
    ref = c.to_plan(c.op.apply(c.u[0]))
    got = c.plan.apply(c.dev(c.u[0]), prec=LS_FP64).cpu().numpy()
    assert rel(got, ref) < 1e-12
    assert np.max(np.abs(got - ref)) < 1e-11 * np.max(np.abs(ref))


def test_fp64_apply_matches_direct_operator(disc):
    from paper_1509_05063_gb300 import LS_FP64
    direct = DirectOperator(disc.dz)
    ref = disc.to_plan(direct.apply(disc.u[1]))
    got = disc.plan.apply(disc.dev(disc.u[1]), prec=LS_FP64).cpu().numpy()
    assert rel(got, ref) < 1e-8


def test_multi_rhs_apply_equals_single(disc):
    from paper_1509_05063_gb300 import LS_FP64
    U = disc.dev(disc.u)
    many = disc.plan.apply(U, prec=LS_FP64).cpu().numpy()
    for r in range(3):
        one = disc.plan.apply(disc.dev(disc.u[r]), prec=LS_FP64).cpu().numpy()
        assert np.array_equal(many[r], one)


def test_batched_complex64_apply_equals_single(kite):
    """Four right-hand sides in one pass over the weights (CUDA cores, four
    rows per warp) give exactly the single-RHS results (same summation order
    per RHS)."""
    from paper_1509_05063_gb300 import LS_MIXED
    U = W.random_density(kite.dz.N, nrhs=4, seed=W.SEED + 11)
    Ud = kite.dev(U, torch.complex64)
    many = kite.plan.apply(Ud, prec=LS_MIXED).cpu().numpy()
    for r in (0, 3):
        one = kite.plan.apply(kite.dev(U[r], torch.complex64), prec=LS_MIXED).cpu().numpy()
        assert np.array_equal(many[r], one)


@pytest.mark.parametrize("nrhs", [8, 16])
@pytest.mark.parametrize("name", ["disc", "kite"])
def test_tensor_core_near_field(name, nrhs, request):
    """8 and 16 complex64 right-hand sides take the tcgen05 near field (split FP16):
    every RHS agrees with its single (CUDA-core, FP32) apply to FP32 rounding
    and with the FP64 oracle within the mixed-precision bound."""
    from paper_1509_05063_gb300 import LS_MIXED
    c = request.getfixturevalue(name)
    U = W.random_density(c.dz.N, nrhs=nrhs, seed=W.SEED + 12)
    many = c.plan.apply(c.dev(U, torch.complex64), prec=LS_MIXED).cpu().numpy()
    for r in (0, nrhs // 2, nrhs - 1):
        one = c.plan.apply(c.dev(U[r], torch.complex64), prec=LS_MIXED).cpu().numpy()
        assert rel(many[r].astype(np.complex128), one.astype(np.complex128)) < 2e-6
    for r in range(nrhs):
        check_mixed(many[r], c.to_plan(c.op.apply(U[r])))


@pytest.mark.parametrize("nrhs", [8, 16])
def test_every_complex64_unit_variant(kite, nrhs):
    """Pinned by ls_plan_set_variants, each tensor-core / CUDA-core choice for
    the projection (3xTF32), local coefficients (3xTF32) and near field (split
    FP16) reproduces the FP64 oracle within the mixed bound, element by
    element, and the eight variants agree with one another to FP32 rounding;
    two of them take the radix-4 lattice transforms."""
    from paper_1509_05063_gb300 import LS_MIXED
    U = W.random_density(kite.dz.N, nrhs=nrhs, seed=W.SEED + 13)
    refs = [kite.to_plan(kite.op.apply(U[r])) for r in range(nrhs)]
    Ud = kite.dev(U, torch.complex64)
    outs = []
    try:
        for var in range(8):
            kite.plan.set_variants(conv_cols32=1 + (var % 2), group32=nrhs, near_cuda32=var & 1,
                                   local_cuda32=(var >> 1) & 1, proj_cuda32=var >> 2,
                                   fft_radix32=4 if var in (3, 4) else 16)
            got = kite.plan.apply(Ud, prec=LS_MIXED).cpu().numpy()
            for r in range(nrhs):
                check_mixed(got[r], refs[r])
            outs.append(got.astype(np.complex128))
        for got in outs[1:]:
            assert rel(got, outs[0]) < 2e-6
        kite.plan.device_status()
    finally:
        kite.plan.set_variants()                # the plan's defaults: tensor cores, groups of 16
    from paper_1509_05063_gb300 import LSError
    with pytest.raises(LSError):
        kite.plan.set_variants(group32=5)
    with pytest.raises(LSError):
        kite.plan.set_variants(proj_cuda32=2)
    with pytest.raises(LSError):
        kite.plan.set_variants(fft_radix32=8)


@pytest.mark.parametrize("name", ["disc", "kite"])
def test_mixed_apply_within_bound(name, request):
    c = request.getfixturevalue(name)
    from paper_1509_05063_gb300 import LS_MIXED
    ref = c.to_plan(c.op.apply(c.u[2]))
    got = c.plan.apply(c.dev(c.u[2], torch.complex64), prec=LS_MIXED).cpu().numpy()
    check_mixed(got, ref)


def test_identity_when_contrast_vanishes():
    from paper_1509_05063_gb300 import LS_FP64, Plan
    wl = _small_disc().replace(n2_params=(1.0,))
    plan = Plan(wl, W.n2_of(wl))
    u = W.random_density(plan.N)[0]
    got = plan.apply(torch.from_numpy(u).to("cuda:0"), prec=LS_FP64).cpu().numpy()
    assert np.array_equal(got, u)


def test_fp64_solve_matches_oracle_gmres(disc):
    from paper_1509_05063_gb300 import LS_FP64
    ui = W.plane_wave(disc.wl.kappa, (1, 0), disc.dz.x)
    ref, it, _ = gmres(disc.op.apply, ui, tol=1e-12, restart=100)
    sol, info = disc.plan.solve(disc.dev(ui), tol=1e-12, prec=LS_FP64)
    assert info["converged"] and info["residual"] <= 1e-12
    assert rel(sol.cpu().numpy(), disc.to_plan(ref)) < 1e-9
    assert abs(info["iterations"] - it) <= 2


def test_mixed_solve_reaches_fp64_tolerance(disc):
    from paper_1509_05063_gb300 import LS_FP64, LS_MIXED
    ui = disc.dev(W.plane_wave(disc.wl.kappa, (0.6, 0.8), disc.dz.x))
    s64, i64 = disc.plan.solve(ui, tol=1e-10, prec=LS_FP64)
    s32, i32 = disc.plan.solve(ui, tol=1e-10, prec=LS_MIXED)
    assert i32["converged"] and i32["residual"] <= 1e-10 and i32["refinements"] >= 1
    assert rel(s32.cpu().numpy(), s64.cpu().numpy()) < 1e-8


@pytest.mark.parametrize("prec_name", ["fp64", "mixed", "mixed32"])
def test_lockstep_multi_rhs_solve_equals_single_solves(disc, prec_name):
    """Three incident directions solved together (one batched apply per
    iteration, Arnoldi per RHS) give the single-RHS solutions."""
    from paper_1509_05063_gb300 import LS_FP64, LS_MIXED, LS_MIXED32
    prec = {"fp64": LS_FP64, "mixed": LS_MIXED, "mixed32": LS_MIXED32}[prec_name]
    dirs = [(1.0, 0.0), (0.6, 0.8), (-0.28, 0.96)]
    U = np.stack([W.plane_wave(disc.wl.kappa, d, disc.dz.x) for d in dirs])
    sol, info = disc.plan.solve(disc.dev(U), tol=1e-10, prec=prec)
    assert info["converged"] and info["residual"] <= 1e-10
    for r in range(3):
        one, _ = disc.plan.solve(disc.dev(U[r]), tol=1e-10, prec=prec)
        assert rel(sol[r].cpu().numpy(), one.cpu().numpy()) < 1e-12


def test_far_field_matches_oracle(disc):
    from paper_1509_05063_gb300 import LS_FP64
    ui = W.plane_wave(disc.wl.kappa, (1, 0), disc.dz.x)
    sol, _ = disc.plan.solve(disc.dev(ui), tol=1e-12, prec=LS_FP64)
    th = np.linspace(0, 2 * math.pi, 24, endpoint=False)
    dirs = np.stack([np.cos(th), np.sin(th)], -1)
    got = disc.plan.farfield(sol, dirs).cpu().numpy()[0]
    u_canon = np.empty(disc.dz.N, complex)
    u_canon[disc.canon] = sol.cpu().numpy()
    ref = far_field(disc.dz, u_canon, th)
    assert rel(got, ref) < 1e-12
    series = exact.disc_far_field(disc.wl.kappa, 2.0, 1.0, th)
    assert np.max(np.abs(got - series)) < 2e-3 * np.max(np.abs(series))


def test_mixed_solution_and_far_field_within_1e10_of_fp64_oracle(disc):
    """Mixed precision (complex64 apply, FP64 refinement) against the FP64
    oracle's solution of the same operator: solution and far field <= 1e-10."""
    from paper_1509_05063_gb300 import LS_MIXED
    ui = W.plane_wave(disc.wl.kappa, (0.6, 0.8), disc.dz.x)
    ref, _, _ = gmres(disc.op.apply, ui, tol=1e-14, restart=200)
    sol, info = disc.plan.solve(disc.dev(ui), tol=1e-12, prec=LS_MIXED)
    assert info["converged"] and info["refinements"] >= 2
    got = sol.cpu().numpy()
    assert rel(got, disc.to_plan(ref)) < 1e-10
    th = np.linspace(0, 2 * math.pi, 32, endpoint=False)
    ff = disc.plan.farfield(sol, np.stack([np.cos(th), np.sin(th)], -1)).cpu().numpy()[0]
    assert rel(ff, far_field(disc.dz, ref, th)) < 1e-10


def test_mixed32_solution_within_1e10_of_fp64_oracle(disc):
    """LS_MIXED32 (complex64 apply and complex64 Arnoldi vectors in the
    correction solves, FP64 refinement) against the FP64 oracle's solution:
    the outer FP64 residual decides, so the solution meets the same 1e-10."""
    from paper_1509_05063_gb300 import LS_MIXED32, LSError
    ui = W.plane_wave(disc.wl.kappa, (0.6, 0.8), disc.dz.x)
    ref, _, _ = gmres(disc.op.apply, ui, tol=1e-14, restart=200)
    sol, info = disc.plan.solve(disc.dev(ui), tol=1e-12, prec=LS_MIXED32)
    assert info["converged"] and info["refinements"] >= 2 and info["residual"] <= 1e-12
    assert rel(sol.cpu().numpy(), disc.to_plan(ref)) < 1e-10
    with pytest.raises(LSError):      # solve-only precision
        disc.plan.apply(torch.zeros(disc.plan.N, dtype=torch.complex64, device="cuda:0"), prec=LS_MIXED32)


def test_cfg1_solution_against_bessel_series():
    """Config 1 (disc, n^2 = 2, kappa = 2, ~4.6k nodes): GPU FP64 solve vs the series."""
    from paper_1509_05063_gb300 import LS_FP64, Plan
    wl = W.cfg1()
    plan = Plan(wl, W.n2_of(wl))
    xy, _ = plan.nodes()
    ui = torch.from_numpy(W.plane_wave(wl.kappa, (1, 0), xy)).to("cuda:0")
    sol, info = plan.solve(ui, tol=1e-10, prec=LS_FP64)
    ue = exact.disc_total_field(wl.kappa, 2.0, 1.0, xy)
    assert info["converged"]
    assert rel(sol.cpu().numpy(), ue) < 2e-4


def test_apply_rejects_wrong_dtype(disc):
    from paper_1509_05063_gb300 import LS_FP64, LSError
    with pytest.raises(LSError):
        disc.plan.apply(torch.zeros(disc.plan.N, dtype=torch.complex64, device="cuda:0"), prec=LS_FP64)


def test_cfg2_full_size_sampled_rows():
    """Config 2 at full size (kite, kappa = 20, ~274k nodes, 1024^2 lattice) in
    every launch configuration the bench times: one FP64 right-hand side, four
    FP64 right-hand sides in one pass, one complex64 right-hand side and 16
    complex64 right-hand sides on the tensor cores (every 128-row tile of every
    cell, collar cells up to several hundred rows).  Oracle rows computed one
    by one (near rows + the oracle accelerator's far part) for four of the
    right-hand sides; element-wise bounds besides the 2-norm."""
    from paper_1509_05063_gb300 import LS_FP64, LS_MIXED, Plan
    wl = W.cfg2()
    plan = Plan(wl, W.n2_of(wl))
    xy, canon = plan.nodes()
    dz = Discretisation(wl)
    rows = W.random_rows(dz.N, 96)
    U = W.random_density(dz.N, nrhs=16, seed=W.SEED + 21)
    cells = Cells(dz)
    nm = near_matrix(dz, cells, rows=rows, chunk=16)
    acc = Accelerator(dz, cells)
    checked = (0, 3, 9, 15)
    ref = {r: U[r][rows] + wl.kappa ** 2 * (nm @ U[r] + acc.apply_far(U[r])[rows]) for r in checked}
    inv = np.argsort(canon)
    sel = inv[rows]
    Ud = torch.from_numpy(np.ascontiguousarray(U[:, canon])).to("cuda:0")
    got = plan.apply(Ud[0].contiguous(), prec=LS_FP64).cpu().numpy()[sel]
    assert rel(got, ref[0]) < 1e-12
    assert np.max(np.abs(got - ref[0])) < 1e-11 * np.max(np.abs(ref[0]))
    got4 = plan.apply(Ud[:4].contiguous(), prec=LS_FP64).cpu().numpy()[:, sel]
    for r in (0, 3):
        assert rel(got4[r], ref[r]) < 1e-12
        assert np.max(np.abs(got4[r] - ref[r])) < 1e-11 * np.max(np.abs(ref[r]))
    got32 = plan.apply(Ud[0].to(torch.complex64), prec=LS_MIXED).cpu().numpy()[sel]
    check_mixed(got32, ref[0])
    got16 = plan.apply(Ud.to(torch.complex64), prec=LS_MIXED).cpu().numpy()[:, sel]
    for r in checked:
        check_mixed(got16[r], ref[r])
    plan.close()


def test_largest_lattice_sampled_rows():
    """A 65 x 65 cell layout (N_eq = 8: n_lat = 521) takes the largest lattice,
    M = 2048, where the complex64 transform ends with its radix-8 pass: FP64,
    one complex64 and 16 complex64 right-hand sides against oracle rows
    computed one by one (near rows + the oracle accelerator's far part)."""
    from paper_1509_05063_gb300 import LS_FP64, LS_MIXED, Plan
    wl = W.place_cells(W.disc(level=3, kappa=2.0, n2c=2.0, collar_w=0.6, tau0=0.3, tau1=0.95, R_a=3, R_b=2,
                              R_cart=2, n_rho=48, N_tau=64), L=65, m=3, N_eq=8)
    plan = Plan(wl, W.n2_of(wl))
    assert plan.info["fft_M"] == 2048
    xy, canon = plan.nodes()
    dz = Discretisation(wl)
    rows = W.random_rows(dz.N, 48)
    U = W.random_density(dz.N, nrhs=16, seed=W.SEED + 22)
    cells = Cells(dz)
    nm = near_matrix(dz, cells, rows=rows, chunk=16)
    acc = Accelerator(dz, cells)
    checked = (0, 7, 15)
    ref = {r: U[r][rows] + wl.kappa ** 2 * (nm @ U[r] + acc.apply_far(U[r])[rows]) for r in checked}
    sel = np.argsort(canon)[rows]
    Ud = torch.from_numpy(np.ascontiguousarray(U[:, canon])).to("cuda:0")
    got = plan.apply(Ud[0].contiguous(), prec=LS_FP64).cpu().numpy()[sel]
    assert rel(got, ref[0]) < 1e-12
    got32 = plan.apply(Ud[0].to(torch.complex64), prec=LS_MIXED).cpu().numpy()[sel]
    check_mixed(got32, ref[0])
    got16 = plan.apply(Ud.to(torch.complex64), prec=LS_MIXED).cpu().numpy()[:, sel]
    for r in checked:
        check_mixed(got16[r], ref[r])
    plan.set_variants(fft_radix32=4)            # the radix-4 transform at M = 2048 too
    got32 = plan.apply(Ud[0].to(torch.complex64), prec=LS_MIXED).cpu().numpy()[sel]
    check_mixed(got32, ref[0])
    plan.close()


def test_many_directions_seeded_from_earlier_solutions(disc):
    """More directions than one lock-step batch: later batches start from the
    least-squares combination of the earlier solutions (A x_j = b_j), which
    must not change the solutions and must save iterations."""
    from paper_1509_05063_gb300 import LS_FP64
    th = 2 * math.pi * np.arange(24) / 24
    U = np.stack([W.plane_wave(disc.wl.kappa, (math.cos(t), math.sin(t)), disc.dz.x) for t in th])
    sol, info = disc.plan.solve(disc.dev(U), tol=1e-10, prec=LS_FP64)
    assert info["converged"] and info["residual"] <= 1e-10
    separate = 0
    for r in (0, 7, 23):
        one, i1 = disc.plan.solve(disc.dev(U[r]), tol=1e-10, prec=LS_FP64)
        assert rel(sol[r].cpu().numpy(), one.cpu().numpy()) < 1e-8
    for r in range(24):
        _, i1 = disc.plan.solve(disc.dev(U[r]), tol=1e-10, prec=LS_FP64)
        separate += i1["iterations"]
    assert info["iterations"] < separate


def test_fp64_apply_on_a_fourier_star_matches_oracle():
    """A third scatterer shape through the same device path: the cosine Fourier
    star r = 1 + 0.1 cos 5s (n^2 = 2), FP64 apply against the oracle's
    accelerated operator."""
    from paper_1509_05063_gb300 import LS_FP64
    wl = W.place_cells(W.star(level=1, kappa=2.0, n2c=2.0, tau0=0.3, tau1=0.95, R_a=4, R_b=2, R_cart=3, p=7,
                              n_rho=48, N_tau=64), L=7, m=4, N_eq=8)
    c = Case(wl)
    ref = c.to_plan(c.op.apply(c.u[0]))
    got = c.plan.apply(c.dev(c.u[0]), prec=LS_FP64).cpu().numpy()
    assert rel(got, ref) < 1e-11
    c.plan.close()
