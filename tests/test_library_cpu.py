"""CPU checks of the C-ABI library (no GPU): it loads, exports every symbol
declared in include/ls.h, rejects bad input with status codes, and its
independent host plan construction reproduces the oracle's discretisation
(nodes, weights, near-field matrix, accelerator matrices)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import workloads as W
from oracle.accel import Accelerator, Cells, near_matrix
from oracle.geometry import Discretisation

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    import paper_1509_05063_gb300 as pkg
    if not os.path.exists(pkg.lib_path()):
        pkg.build_library()
    return pkg.load_library()


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "ls.h")).read()
    return sorted(set(re.findall(r"^\s*(?:ls_status|const char\*)\s+(ls_\w+)\s*\(", src, re.M)))


def test_library_exports_every_declared_symbol(lib):
    import paper_1509_05063_gb300.ls as b
    names = declared_symbols()
    assert len(names) >= 14
    for n in names:
        assert hasattr(lib, n), n
        assert n in b.EXPORTED, n


def test_invalid_arguments_return_status(lib):
    import paper_1509_05063_gb300.ls as b
    wl = W.cfg1()
    g = b.geometry_from(wl)
    o = b.options_from(wl)
    h = C.c_void_p()
    cb = b._n2_callback(W.n2_of(wl))
    g.dim = 3
    assert lib.ls_host_plan_create(C.byref(g), cb, None, wl.kappa, C.byref(o), C.byref(h)) == 6
    g.dim = 2
    assert lib.ls_host_plan_create(C.byref(g), cb, None, -1.0, C.byref(o), C.byref(h)) == 1
    gs = b.geometry_from(wl)
    gs.shape = 2                                  # Fourier star with r(s) < 0 somewhere
    gs.params[0], gs.params[7] = 0.5, 0.6
    assert lib.ls_host_plan_create(C.byref(gs), cb, None, wl.kappa, C.byref(o), C.byref(h)) == 1
    o.L = 2            # cells too large for the box -> nodes outside
    assert lib.ls_host_plan_create(C.byref(g), cb, None, wl.kappa, C.byref(o), C.byref(h)) == 1
    assert b"outside" in lib.ls_last_error(None)
    o = b.options_from(wl)
    o.H, o.L = 0.12, 20   # cells too small for the cut-off support -> eta leaves N(x)
    o.box_x0 = o.box_y0 = -1.2
    assert lib.ls_host_plan_create(C.byref(g), cb, None, wl.kappa, C.byref(o), C.byref(h)) == 1
    assert b"3 x 3" in lib.ls_last_error(None)
    bad = b.N2FN(lambda n, xy, out, ctx: 1)
    o = b.options_from(wl)
    assert lib.ls_host_plan_create(C.byref(g), bad, None, wl.kappa, C.byref(o), C.byref(h)) == 1
    assert lib.ls_apply(None, None, None, 1, 0, None) == 1
    assert lib.ls_plan_destroy(None) == 0
    assert lib.ls_status_string(4) == b"no convergence"
    hb = C.c_void_p()
    assert lib.ls_batch_create(None, 0, C.byref(hb)) == 1
    assert b"no plans" in lib.ls_batch_last_error(None)
    same = (C.c_void_p * 2)(0x1000, 0x1000)       # rejected before either handle is used
    assert lib.ls_batch_create(same, 2, C.byref(hb)) == 1
    assert b"appears twice" in lib.ls_batch_last_error(None)
    assert lib.ls_batch_apply(None, None, None, 0, None) == 1
    assert lib.ls_batch_solve(None, None, None, 1e-10, 10, 10, 0, None, None, None) == 1
    assert lib.ls_batch_destroy(None) == 0
    assert lib.ls_plan_device_status(None) == 1
    assert lib.ls_set_wait_limit(None, 0) == 1
    assert lib.ls_plan_autotune(None, 16, None) == 1
    assert lib.ls_plan_set_variants(None, None) == 1


def _small_disc():
    return W.place_cells(W.disc(level=1, kappa=2.0, n2c=2.0, collar_w=0.6, tau0=0.3, tau1=0.95, R_a=4, R_b=2,
                                R_cart=3, p=7, n_rho=48, N_tau=64), L=8, m=3, N_eq=8)


def _small_kite():
    return W.place_cells(W.kite(n1=512, n2=17, h=0.025, kappa=6.0, collar_w=0.07, tau0=0.4, tau1=0.9, R_a=6,
                                R_b=5, R_cart=4, n_rho=32, N_tau=48), L=17, m=8, center=(-0.25, 0.0), N_eq=8)


def _small_star():
    return W.place_cells(W.star(level=1, kappa=2.0, n2c=2.0, tau0=0.3, tau1=0.95, R_a=4, R_b=2, R_cart=3, p=7,
                                n_rho=48, N_tau=64), L=7, m=4, N_eq=8)


@pytest.mark.parametrize("make", [_small_disc, _small_kite, _small_star])
def test_host_plan_matches_oracle_discretisation(lib, make):
    from paper_1509_05063_gb300 import HostPlan
    wl = make()
    hp = HostPlan(wl, W.n2_of(wl))
    xy, canon, wfac = hp.nodes()
    dz = Discretisation(wl)
    assert hp.N == dz.N
    assert np.array_equal(np.sort(canon), np.arange(dz.N))
    assert np.max(np.abs(xy - dz.x[canon])) < 1e-13
    assert np.max(np.abs(wfac - dz.wfac[canon])) < 1e-15
    cells = Cells(dz)
    rows = np.arange(dz.N) if dz.N < 2000 else W.random_rows(dz.N, 300)
    ref = near_matrix(dz, cells, rows=rows)[:, canon].toarray()
    inv = np.argsort(canon)
    near = hp.near()
    got = near[inv[rows]].toarray()
    assert np.max(np.abs(got - ref)) <= 1e-13 * np.max(np.abs(ref))
    # every row's columns strictly increase (sorted, each column once)
    for r in range(0, hp.N, max(1, hp.N // 500)):
        assert np.all(np.diff(near.indices[near.indptr[r]:near.indptr[r + 1]]) > 0)


@pytest.mark.parametrize("make", [_small_disc, _small_kite, _small_star])
def test_host_accelerator_matrices_reproduce_oracle_far_field(lib, make):
    """Run the accelerator's steps in numpy with the library's matrices (P_c,
    B^+, B^+ T_o, Phi, kernel tables) and compare with the oracle's far part."""
    from paper_1509_05063_gb300 import HostPlan
    wl = make()
    hp = HostPlan(wl, W.n2_of(wl))
    xy, canon, _ = hp.nodes()
    dz = Discretisation(wl)
    acc = Accelerator(dz)
    u = W.random_density(dz.N)[0]
    ref = acc.apply_far(u)[canon]
    A = hp.accel()
    up = u[canon]
    L, Ne, n_es, M = wl.L, wl.N_eq, hp.n_es, hp.M
    cell = (np.floor((xy[:, 0] - wl.box_x0) / wl.H).astype(int)
            + L * np.floor((xy[:, 1] - wl.box_y0) / wl.H).astype(int))
    sig = {}
    for k, c in enumerate(A["occ"]):
        mem = np.nonzero(cell == c)[0]
        sig[c] = A["P"][A["P_off"][k]:A["P_off"][k + 1]].reshape(n_es, len(mem)) @ up[mem]
    Sm = np.zeros((M, M), complex)
    Sd = np.zeros((M, M), complex)
    for c, s in sig.items():
        ci, cj = c % L, c // L
        for f in range(4):
            for kk in range(Ne + 1):
                (Sm if f < 2 else Sd)[(ci + f % 2) * Ne, cj * Ne + kk] += s[f * (Ne + 1) + kk]
    V = np.fft.ifft2(np.fft.fft2(Sm) * np.fft.fft2(A["Gtab"]) + np.fft.fft2(Sd) * np.fft.fft2(A["Dtab"]))
    got = np.zeros(hp.N, complex)
    for c in sig:
        ci, cj = c % L, c // L
        g = A["Bpinv"] @ np.array([V[ci * Ne + a, cj * Ne + b] for a in range(Ne + 1) for b in range(Ne + 1)])
        for oi in (-1, 0, 1):
            for oj in (-1, 0, 1):
                nb = (cj + oj) * L + (ci + oi)
                if 0 <= ci + oi < L and 0 <= cj + oj < L and nb in sig:
                    g = g - A["BT"][(oi + 1) * 3 + (oj + 1)] @ sig[nb]
        mem = np.nonzero(cell == c)[0]
        got[mem] = A["Phi"][mem] @ g
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-11


def _apply_far3(A, u, L, Ne, n_es, M):
    """The 3-D accelerator's steps in numpy with the library's matrices."""
    nf = (Ne + 1) ** 2
    members, sig, pos = {}, {}, 0
    for k, c in enumerate(A["occ"]):
        n_c = (A["P_off"][k + 1] - A["P_off"][k]) // n_es
        members[c] = A["order"][pos:pos + n_c]
        pos += n_c
        sig[c] = A["P"][A["P_off"][k]:A["P_off"][k + 1]].reshape(n_es, n_c) @ u[members[c]]
    Sm = np.zeros((M,) * 3, complex)
    Sd = np.zeros((M,) * 3, complex)
    bb, cc = np.meshgrid(np.arange(Ne + 1), np.arange(Ne + 1), indexing="ij")
    bb, cc = bb.ravel(), cc.ravel()
    for c, s in sig.items():
        i, j, k = c % L, (c // L) % L, c // (L * L)
        for f in range(4):
            np.add.at(Sm if f < 2 else Sd, (np.full(nf, (i + f % 2) * Ne), j * Ne + bb, k * Ne + cc),
                      s[f * nf:(f + 1) * nf])
    V = np.fft.ifftn(np.fft.fftn(Sm) * np.fft.fftn(A["Gtab"]) + np.fft.fftn(Sd) * np.fft.fftn(A["Dtab"]))
    g = np.arange(Ne + 1)
    la = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    out = np.zeros(len(u), complex)
    for c in sig:
        ijk = np.array([c % L, (c // L) % L, c // (L * L)])
        p = ijk * Ne + la
        gam = A["Bpinv"] @ V[p[:, 0], p[:, 1], p[:, 2]]
        for o in range(27):
            nb = ijk + np.array([o // 9, (o // 3) % 3, o % 3]) - 1
            if np.all((nb >= 0) & (nb < L)):
                nc = int((nb[2] * L + nb[1]) * L + nb[0])
                if nc in sig:
                    gam = gam - A["BT"][o] @ sig[nc]
        out[members[c]] = A["Phi"][members[c]] @ gam
    return out


def test_host_accel3_reproduces_oracle_far_field(lib):
    """The library's 3-D accelerator setup (equivalent-source fits by a
    QR-preconditioned Jacobi SVD, spherical-wave local expansion, 27 neighbour
    tables, 3-D kernel lattice tables) run through the accelerator's steps in
    numpy: equal to the oracle's 3-D far part up to the fits' truncation, and
    to the exact non-adjacent sum within the equivalent-source error."""
    from paper_1509_05063_gb300 import HostAccel3, LSError
    from oracle.accel3d import Accelerator3
    from oracle.geometry3d import Ball3, Discretisation3
    dz = Discretisation3(Ball3(n_f=9, n_s=5, h=0.2))
    wfac = dz.w * dz.omega * (1 - dz.b.n2c)
    u = W.random_density(dz.N)[0]
    L, Ne = 6, 6
    ha = HostAccel3(dz.x, wfac, 2.0, [-1.13] * 3, 2.26 / L, L, Ne)
    assert (ha.n_es, ha.nb, ha.n_loc, ha.M) == (4 * 49, 14 * 14, 343, 128)
    got = _apply_far3(ha.get(), u, L, Ne, ha.n_es, ha.M)
    acc = Accelerator3(dz.x, wfac, 2.0, -1.13, 2.26 / L, L, Ne)
    ref = acc.apply_far(u)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-8
    direct = acc.direct_far(u)
    assert np.linalg.norm(got - direct) / np.linalg.norm(direct) < 1e-5
    with pytest.raises(LSError, match="outside"):
        HostAccel3(dz.x, wfac, 2.0, [-0.5] * 3, 2.26 / L, L, Ne)
    with pytest.raises(LSError, match="more terms"):
        HostAccel3(dz.x, wfac, 2.0, [-1.13] * 3, 2.26 / L, L, 2, p=5)


def test_host_ball3_matches_oracle_discretisation(lib):
    """The library's 3-D ball discretisation (six blended cubed-sphere shell
    faces, interior grid) node for node against the oracle's: positions,
    weights, partitions of unity, faces and grid indices."""
    from paper_1509_05063_gb300 import HostBall3, LSError
    from oracle.geometry3d import Ball3, Discretisation3
    for nf, ns, h in ((9, 5, 0.2), (25, 9, 0.1)):
        dz = Discretisation3(Ball3(n_f=nf, n_s=ns, h=h))
        hb = HostBall3(n_f=nf, n_s=ns, h=h)
        assert (hb.N, hb.n_shell, hb.grid_m) == (dz.N, dz.n_shell, dz.grid_m)
        nd = hb.nodes()
        assert np.max(np.abs(nd["x"] - dz.x)) < 1e-15
        assert np.max(np.abs(nd["w"] - dz.w) / dz.w) < 1e-14
        assert np.max(np.abs(nd["omega"] - dz.omega)) < 1e-15
        assert np.max(np.abs(nd["psi"] - dz.psi)) < 1e-15
        assert np.array_equal(nd["face"], dz.face)
        assert np.array_equal(nd["grid"][:dz.n_shell], dz.fijk[:dz.n_shell])
        assert np.array_equal(nd["grid"][dz.n_shell:], np.rint(dz.x[dz.n_shell:] / h).astype(int) + dz.grid_m)
    with pytest.raises(LSError, match="multiple of Q - 1"):
        HostBall3(n_s=8)
    with pytest.raises(LSError, match="tau0"):
        HostBall3(tau0=0.9, tau1=0.5)


def test_host_interior_window3_matches_oracle(lib):
    """The library's window of the 3-D interior singular rule against the
    oracle's (same rule, same interpolation), at two wavenumbers and spacings."""
    from paper_1509_05063_gb300 import LSError, interior_window3
    from oracle.quadrature3d import interior_singular_window
    for k, h in ((2.0, 0.1), (5.0, 0.05)):
        w0, W0 = interior_singular_window(k, h, 3.0, 5)
        w1, W1 = interior_window3(k, h, 3.0, 5)
        assert W1 == W0
        assert np.max(np.abs(w1 - w0)) < 1e-13 * np.max(np.abs(w0))
    with pytest.raises(LSError, match="interior rule"):
        interior_window3(2.0, -0.1)


def test_host_ball3_rows_match_oracle(lib):
    """Rows of the library's 3-D operator (interior spherical rule, shell
    boundary and interior-type rules with split Newton-Cotes, regular sums with
    1 - eta) against the oracle's rows at random shell and interior targets."""
    from paper_1509_05063_gb300 import HostBall3, LSError
    from oracle.geometry3d import Ball3, Discretisation3
    from oracle.quadrature3d import k_row
    rng = np.random.default_rng(12)
    for nf, ns, h, n in ((13, 5, 0.2, 4), (25, 9, 0.1, 3)):
        dz = Discretisation3(Ball3(n_f=nf, n_s=ns, h=h))
        hb = HostBall3(n_f=nf, n_s=ns, h=h)
        tg = np.concatenate([rng.choice(dz.n_shell, n, replace=False),
                             dz.n_shell + rng.choice(dz.n_cart, n, replace=False)])
        # targets whose direction lies in three face charts at once (a cube corner)
        corner = dz.x @ (np.ones(3) / np.sqrt(3)) / np.maximum(np.linalg.norm(dz.x, axis=1), 1e-300)
        shell_c = int(np.argmax(np.where(np.arange(dz.N) < dz.n_shell, corner, -1)))
        deep = np.linalg.norm(dz.x, axis=1) > 1.0 - dz.b.w              # interior nodes under the shell
        inner_c = int(np.argmax(np.where((np.arange(dz.N) >= dz.n_shell) & deep, corner, -1)))
        tg = np.concatenate([tg, [shell_c, inner_c]])
        for q in tg:
            ref = k_row(dz, 2.0, int(q))
            got, eta = hb.row(2.0, int(q))
            assert np.max(np.abs(got - ref)) < 1e-13 * np.max(np.abs(ref))
            assert eta.min() >= 0.0 and eta.max() <= 1.0
    with pytest.raises(LSError, match="out of range"):
        hb.row(2.0, hb.N)


def test_host_ball3_near_plus_exact_far_sum_is_the_row(lib):
    """The library's adjacent part of the 3-D operator (singular rules plus the
    regular terms of the 3 x 3 x 3 cell block) plus the exact non-adjacent sum
    equals the oracle's whole row, and its entries inside the block equal the
    row's; a cut-off reaching past the block is rejected.  Cut-off radii of 3
    index units keep the support inside cells of side 0.32 at this level."""
    from paper_1509_05063_gb300 import HostBall3, LSError
    from oracle.accel3d import Accelerator3
    from oracle.geometry3d import Ball3, Discretisation3
    from oracle.quadrature3d import Rules3, k_row
    dz = Discretisation3(Ball3(n_f=25, n_s=9, h=0.1))
    hb = HostBall3(n_f=25, n_s=9, h=0.1)
    L, H, x0 = 7, 2.26 / 7, -1.13
    rng = np.random.default_rng(13)
    rows = np.concatenate([rng.choice(dz.n_shell, 4, replace=False),
                           dz.n_shell + rng.choice(dz.n_cart, 4, replace=False)])
    near = hb.near(2.0, [x0] * 3, H, L, rows=rows, rules=dict(rc=3.0, rs=3.0))
    wfac = dz.w * dz.omega
    acc = Accelerator3(dz.x, wfac, 2.0, x0, H, L, 2, p=2)
    u = W.random_density(dz.N)[0]
    far = acc.direct_far(u, rows=rows)
    ru = Rules3(rc=3.0, rs=3.0)
    for i, q in enumerate(rows):
        ref = k_row(dz, 2.0, int(q), ru)
        got = near[i].toarray()[0]
        assert abs(got @ u + far[i] - ref @ u) < 1e-13 * np.sum(np.abs(ref * u))
        blk = acc.cells.near_mask([q])[0]
        assert np.max(np.abs(got[blk] - ref[blk])) < 1e-14 * np.max(np.abs(ref))
    # stored stencils plus the block's plain regular sum computed on the fly
    st = hb.near(2.0, [x0] * 3, H, L, rows=rows, rules=dict(rc=3.0, rs=3.0), stencils_only=True)
    assert st.nnz < near.nnz / 2
    for i, q in enumerate(rows):
        blk = np.nonzero(acc.cells.near_mask([q])[0])[0]
        blk = blk[blk != q]
        dist = np.linalg.norm(dz.x[blk] - dz.x[q], axis=1)
        reg = wfac[blk] * np.exp(2j * dist) / (4 * np.pi * dist)
        full = near[i].toarray()[0] @ u
        assert abs(st[i].toarray()[0] @ u + reg @ u[blk] - full) < 1e-13 * np.sum(np.abs(near[i].toarray()[0] * u))
    # the whole accelerated 3-D operator on the host: adjacent part plus the
    # library's equivalent-source far part (N_eq = 6)
    from paper_1509_05063_gb300 import HostAccel3
    ha = HostAccel3(dz.x, wfac, 2.0, [x0] * 3, H, L, 6)
    far_es = _apply_far3(ha.get(), u, L, 6, ha.n_es, ha.M)[rows]
    assert np.linalg.norm(far_es - far) < 1e-5 * np.linalg.norm(far)
    with pytest.raises(LSError, match="3 x 3 x 3"):
        hb.near(2.0, [x0] * 3, H, L, rows=rows)          # default radii 6 reach past the block
    with pytest.raises(LSError, match="outside the cell box"):
        hb.near(2.0, [-0.5] * 3, H, L, rows=rows, rules=dict(rc=3.0, rs=3.0))
    with pytest.raises(LSError, match="out of range"):
        hb.near(2.0, [x0] * 3, H, L, rows=[hb.N], rules=dict(rc=3.0, rs=3.0))
    with pytest.raises(LSError, match="rule parameters"):
        hb.near(2.0, [x0] * 3, H, L, rows=rows, rules=dict(n_rho=1))


def test_native_3d_operator_solves_the_sphere_problem(lib):
    """Dense solve of u + kappa^2 K[m u] = u^i with the library's 3-D rows (one
    cell, so every row is whole) on the penetrable sphere at 3935 unknowns: the
    error against the series solution lies within the paper's 3-D convergence
    table at this size (log-interpolated between its 2187- and 14 739-unknown
    entries)."""
    import json
    from oracle import exact
    from paper_1509_05063_gb300 import HostBall3
    gold = json.load(open(os.path.join(ROOT, "tests", "golden", "paper_tables.json")))["sphere_Q5_kappa2_n_sqrt2"]
    hb = HostBall3(n_f=13, n_s=5, h=0.2)
    x = hb.nodes()["x"]
    k, n2 = 2.0, 2.0
    K = hb.near(k, [-1.13] * 3, 2.26, 1).toarray()
    u = np.linalg.solve(np.eye(hb.N) + k * k * (1 - n2) * K, np.exp(1j * k * x[:, 2]))
    ue = exact.sphere_total_field(k, n2, 1.0, x)
    err = np.linalg.norm(u - ue) / np.linalg.norm(ue)
    band = np.exp(np.interp(np.log(hb.N), np.log(gold["unknowns"]), np.log(gold["eps2"])))
    assert hb.N == 3935 and err < band
