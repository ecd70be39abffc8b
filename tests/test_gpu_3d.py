"""GPU parity of the 3-D device path (Section 5: the penetrable ball) against the
CPU oracle, through the C ABI (ls_plan_create3, ls_apply, ls_solve).

The oracle's accelerated 3-D operator on the same nodes: the adjacent part of
each sampled row is the oracle's whole row (every singular rule plus the
regular sums, oracle/quadrature3d.k_row) less its exact non-adjacent entries,
and the far part is the oracle's equivalent-source accelerator
(oracle/accel3d.Accelerator3) with the same cells, N_eq and local degree.

Tolerances (derived from the arithmetic):
* FP64 apply: 1e-11 relative, normwise and element-wise.  Both sides are FP64
  and follow the same steps; they differ by the rounding of the FFTs and
  contractions and by the two independent truncated SVD fits (rcond 1e-13),
  whose far parts agree to ~6e-11 of the far part (measured on the CPU with
  the library's host matrices), itself ~0.5 % of the apply here.
* complex64 apply: 1e-5 relative, normwise and element-wise (the mixed bound).
* mixed solve: the FP64 residual 1e-10 and the FP64 solution to 1e-8.
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import exact

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

KAPPA, N2 = 2.0, 2.0
BALL = dict(n_f=17, n_s=5, h=0.15)
RULES = dict(rc=3.0, rs=3.0)
L, HALF, NE = 5, 1.13, 4


def n2_const(x):
    return np.full(len(x), N2)


def n2_varying(x):
    """Config 5's medium, n^2 = 1.2 + 0.6 sin(pi x1) cos(pi x2), on the ball."""
    return 1.2 + 0.6 * np.sin(np.pi * x[:, 0]) * np.cos(np.pi * x[:, 1])


class Case3:
    def __init__(self, n2=n2_const):
        from oracle.accel3d import Accelerator3
        from oracle.geometry3d import Ball3, Discretisation3
        from paper_1509_05063_gb300 import Plan3
        H = 2 * HALF / L
        self.plan = Plan3(n2, KAPPA, [-HALF] * 3, H, L, NE, ball=BALL, rules=RULES)
        self.xyz, self.canon = self.plan.nodes()
        self.dz = Discretisation3(Ball3(**BALL))
        self.m = 1.0 - n2(self.dz.x)
        wfac = self.dz.w * self.dz.omega * self.m
        self.acc = Accelerator3(self.dz.x, wfac, KAPPA, -HALF, H, L, NE)

    def to_plan(self, v):
        return np.ascontiguousarray(v[..., self.canon])

    def dev(self, v, dtype=torch.complex128):
        return torch.from_numpy(self.to_plan(v)).to("cuda:0", dtype)

    def oracle_rows(self, u, rows):
        """(A u)[rows] of the oracle's accelerated 3-D operator (ball order): the
        whole row less its exact non-adjacent sum (w omega m G over the nodes
        outside the 3 x 3 x 3 cell block; singular-rule stencil entries that
        reach past the block stay), plus the accelerator's far part."""
        from oracle.quadrature3d import Rules3, k_row
        ru = Rules3(**RULES)
        far = self.acc.apply_far(u)
        exact_far = self.acc.direct_far(u, rows=rows)
        out = np.empty(len(rows), complex)
        for i, q in enumerate(rows):
            near = k_row(self.dz, KAPPA, int(q), ru) @ (self.m * u) - exact_far[i]
            out[i] = u[q] + KAPPA ** 2 * (near + far[q])
        return out


@pytest.fixture(scope="module")
def ball():
    c = Case3()
    yield c
    c.plan.close()


def sample_rows(dz, k=24, seed=17):
    rng = np.random.default_rng(seed)
    return np.concatenate([rng.choice(dz.n_shell, k, replace=False), dz.n_shell + rng.choice(dz.n_cart, k, replace=False)])


def test_plan_matches_oracle_nodes(ball):
    assert ball.plan.N == ball.dz.N
    assert np.array_equal(np.sort(ball.canon), np.arange(ball.dz.N))
    assert np.max(np.abs(ball.xyz - ball.dz.x[ball.canon])) < 1e-14


def test_fp64_apply_matches_oracle_accelerated_operator(ball):
    from paper_1509_05063_gb300 import LS_FP64
    u = W.random_density(ball.dz.N)[0]
    rows = sample_rows(ball.dz)
    ref = ball.oracle_rows(u, rows)
    got = ball.plan.apply(ball.dev(u), prec=LS_FP64).cpu().numpy()
    inv = np.argsort(ball.canon)
    g = got[inv[rows]]
    assert np.linalg.norm(g - ref) / np.linalg.norm(ref) < 1e-11
    assert np.max(np.abs(g - ref)) < 1e-11 * np.max(np.abs(ref))


def test_mixed_apply_within_bound(ball):
    from paper_1509_05063_gb300 import LS_MIXED
    u = W.random_density(ball.dz.N, seed=W.SEED + 41)[0]
    rows = sample_rows(ball.dz, seed=18)
    ref = ball.oracle_rows(u, rows)
    got = ball.plan.apply(ball.dev(u, torch.complex64), prec=LS_MIXED).cpu().numpy().astype(np.complex128)
    g = got[np.argsort(ball.canon)[rows]]
    assert np.linalg.norm(g - ref) / np.linalg.norm(ref) < 1e-5
    assert np.max(np.abs(g - ref)) < 1e-5 * np.max(np.abs(ref))


def test_varying_medium_apply_matches_oracle():
    """n^2 varying inside the ball (config 5's sin . cos medium): the contrast is
    folded into every stored entry and projection per source node, so both
    precisions must still meet their bounds against the oracle built with the
    same m(x)."""
    from paper_1509_05063_gb300 import LS_FP64, LS_MIXED
    c = Case3(n2_varying)
    assert np.ptp(c.m) > 0.5
    u = W.random_density(c.dz.N, seed=W.SEED + 43)[0]
    rows = sample_rows(c.dz, seed=19)
    ref = c.oracle_rows(u, rows)
    inv = np.argsort(c.canon)
    g = c.plan.apply(c.dev(u), prec=LS_FP64).cpu().numpy()[inv[rows]]
    assert np.linalg.norm(g - ref) / np.linalg.norm(ref) < 1e-11
    assert np.max(np.abs(g - ref)) < 1e-11 * np.max(np.abs(ref))
    g32 = c.plan.apply(c.dev(u, torch.complex64), prec=LS_MIXED).cpu().numpy().astype(np.complex128)[inv[rows]]
    assert np.max(np.abs(g32 - ref)) < 1e-5 * np.max(np.abs(ref))
    c.plan.close()


def test_multi_rhs_apply_equals_single(ball):
    from paper_1509_05063_gb300 import LS_FP64
    U = W.random_density(ball.dz.N, nrhs=3, seed=W.SEED + 42)
    many = ball.plan.apply(ball.dev(U), prec=LS_FP64).cpu().numpy()
    for r in range(3):
        one = ball.plan.apply(ball.dev(U[r]), prec=LS_FP64).cpu().numpy()
        assert np.array_equal(many[r], one)


def test_solves_against_mie_series_and_mixed_reaches_fp64(ball):
    """The penetrable sphere (n^2 = 2, kappa = 2, plane wave exp(i kappa z)):
    the FP64 solve of the accelerated operator against the Mie series, and
    the mixed solve (complex64 apply, FP64 refinement) to the same FP64
    residual and solution."""
    from paper_1509_05063_gb300 import LS_FP64, LS_MIXED
    ui = np.exp(1j * KAPPA * ball.xyz[:, 2])
    uid = torch.from_numpy(ui).to("cuda:0")
    s64, i64 = ball.plan.solve(uid, tol=1e-10, prec=LS_FP64, restart=60)
    assert i64["converged"] and i64["residual"] <= 1e-10
    ue = exact.sphere_total_field(KAPPA, N2, 1.0, ball.xyz)
    err = np.linalg.norm(s64.cpu().numpy() - ue) / np.linalg.norm(ue)
    assert err < 3e-2
    s32, i32 = ball.plan.solve(uid, tol=1e-10, prec=LS_MIXED, restart=30)
    assert i32["converged"] and i32["residual"] <= 1e-10 and i32["refinements"] >= 1
    assert np.linalg.norm((s32 - s64).cpu().numpy()) / np.linalg.norm(s64.cpu().numpy()) < 1e-8


def test_far_field_against_mie_series(ball):
    from paper_1509_05063_gb300 import LS_FP64
    ui = torch.from_numpy(np.exp(1j * KAPPA * ball.xyz[:, 2])).to("cuda:0")
    sol, _ = ball.plan.solve(ui, tol=1e-10, prec=LS_FP64, restart=60)
    th = np.linspace(0.1, math.pi - 0.1, 9)
    dirs = np.stack([np.sin(th), np.zeros_like(th), np.cos(th)], -1)
    got = ball.plan.farfield(sol, dirs).cpu().numpy()[0]
    ref = exact.sphere_far_field(KAPPA, N2, 1.0, th)
    assert np.max(np.abs(got - ref)) < 5e-2 * np.max(np.abs(ref))


def test_3d_plan_rejects_unsupported_calls(ball):
    from paper_1509_05063_gb300 import LS_FP64, Batch, LSError
    u = torch.zeros(ball.plan.N, dtype=torch.complex128, device="cuda:0")
    with pytest.raises(LSError) as e:
        ball.plan.apply_noalloc(u, torch.empty_like(u), prec=LS_FP64)
    assert e.value.status == 6
    with pytest.raises(LSError):
        Batch([ball.plan])
