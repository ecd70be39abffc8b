"""Three-dimensional singular quadrature of the interior patch (test
infrastructure only): the extension of the interior-type rule (Section 3.1.1,
Eq. K-Int-Sing-Polar) in Section 5, in spherical coordinates about the target.

For a target x on the interior grid the cut-off part of the patch integral,
int G(x, y) eta(|y - x| / (R h)) phi_I(y) dy, is taken in spherical coordinates
about x: the volume element rho^2 cancels the 1/rho of
G = exp(i kappa rho) / (4 pi rho); rho = R s^q in grid units with the trapezoid
rule in s, Gauss-Legendre in cos(theta) (the paper names Clenshaw-Curtis; any
rule exact for the smooth angular dependence serves) and the trapezoid rule in
the azimuth.  phi_I at the off-grid points comes from tensor-product Lagrange
interpolation of degree p on the grid (zero off the interior node set).  On a
uniform grid the rule is the same for every grid-point target, so it is
computed once as a window of coefficients over grid offsets.
"""
from __future__ import annotations

import math

import numpy as np

from .quadrature import chi, lagrange


def interior_singular_window(kappa: float, h: float, R: float, p: int, q: int = 3, n_rho: int = 16,
                             n_mu: int = 16, n_phi: int = 32, chi_s0: float = 0.1):
    """Coefficients c[o] (o: integer grid offsets, window [-W, W]^3) with
    int G eta phi_I dy ~ sum_o c[o] phi_I(x + o h) for a grid-point target x."""
    s = np.arange(1, n_rho) / n_rho
    rho = R * s ** q                                                   # grid units
    wr = (1.0 / n_rho) * R * q * s ** (q - 1) * chi(s ** q, chi_s0)
    mu, wmu = np.polynomial.legendre.leggauss(n_mu)
    ph = 2 * np.pi * np.arange(n_phi) / n_phi
    RHO, MU, PH = np.meshgrid(rho, mu, ph, indexing="ij")
    W = (wr[:, None, None] * wmu[None, :, None] * (2 * np.pi / n_phi)) * np.ones(RHO.shape)
    st = np.sqrt(1 - MU ** 2)
    o = np.stack([RHO * st * np.cos(PH), RHO * st * np.sin(PH), RHO * MU], -1).reshape(-1, 3)
    r = RHO.ravel()
    # rho^2 h^3 G(rho h) = rho h^2 exp(i kappa rho h) / (4 pi)
    f = W.ravel() * r * h * h * np.exp(1j * kappa * r * h) / (4 * np.pi)
    keep = f != 0
    o, f = o[keep], f[keep]
    Wn = int(math.ceil(R)) + p // 2 + 2
    win = np.zeros((2 * Wn + 1,) * 3, np.complex128)
    st_ = np.floor(o).astype(np.int64) - p // 2                       # stencil starts
    L = [lagrange(o[:, k], st_[:, k], p) for k in range(3)]            # (P, p+1) each
    ar = np.arange(p + 1)
    for i in range(p + 1):
        for j in range(p + 1):
            cij = f * L[0][:, i] * L[1][:, j]
            for k in range(p + 1):
                np.add.at(win, (st_[:, 0] + i + Wn, st_[:, 1] + j + Wn, st_[:, 2] + k + Wn), cij * L[2][:, k])
    del ar
    return win, Wn


def interior_K(dz, kappa: float, targets, density, R: float = 3.0, p: int = 5, **rule):
    """K[phi](x_q) = int_ball G(x_q, y) phi(y) dy for interior grid-point targets
    whose cut-off ball and interpolation stencils stay in the region where the
    shell's integrand is regular (the shell partition vanishes near them);
    density: u at the nodes, phi = u omega with the node's partition value
    (m = 1).  Returns K at the targets."""
    b = dz.b
    win, Wn = interior_singular_window(kappa, b.h, R, p, **rule)
    m = dz.grid_m + Wn                                  # zero padding: omega_I vanishes off the ball
    om_grid = np.pad(dz.grid_omega, Wn)
    u_grid = np.zeros(om_grid.shape, np.complex128)
    cart = np.nonzero(dz.chart == 1)[0]
    gi = np.rint(dz.x[cart] / b.h).astype(np.int64) + m
    u_grid[gi[:, 0], gi[:, 1], gi[:, 2]] = density[cart]
    phi_grid = u_grid * om_grid
    out = np.zeros(len(targets), np.complex128)
    for t, qn in enumerate(targets):
        x = dz.x[qn]
        c = np.rint(x / b.h).astype(np.int64) + m
        lo, hi = c - Wn, c + Wn + 1
        if np.any(lo < 0) or np.any(hi > om_grid.shape[0]):
            raise ValueError("target too close to the grid edge")
        sing = np.sum(win * phi_grid[lo[0]:hi[0], lo[1]:hi[1], lo[2]:hi[2]])
        # regular parts: every node, (1 - eta) on the interior patch's own nodes
        d = np.linalg.norm(dz.x - x, axis=1)
        G = np.zeros(dz.N, np.complex128)
        nz = d > 0
        G[nz] = np.exp(1j * kappa * d[nz]) / (4 * np.pi * d[nz])
        eta = np.where(dz.chart == 1, chi(d / (R * b.h), rule.get("chi_s0", 0.1)), 0.0)
        out[t] = sing + np.sum(dz.w * dz.omega * density * G * (1 - eta))
    return out


# ---------------------------------------------------------------- the whole operator (rows)
from dataclasses import dataclass  # noqa: E402

from .geometry import newton_cotes  # noqa: E402,F401
from .geometry3d import FACES, face_coords, face_direction  # noqa: E402
from .quadrature import split_newton_cotes  # noqa: E402


@dataclass
class Rules3:
    """Parameters of the 3-D singular rules (index units of the grids)."""
    R: float = 3.0          # interior patch: cut-off radius in grid units
    p: int = 5              # Lagrange degree
    q: int = 3              # radial map rho = r s^q
    n_rho: int = 16
    n_mu: int = 16
    n_phi: int = 32
    rc: float = 6.0         # shell: cut-off radius in (xi, eta) index units
    rs: float = 6.0         # shell: cut-off half-width across the depth (s index units)
    n_sig: int = 20
    n_th: int = 32
    chi_s0: float = 0.1


def _lagrange_cols(t, p, n=None, clamp=False):
    """Stencil starts and Lagrange weights (P, p+1) of positions t (P,) on the
    integer grid 0..n-1 (clamped stencils when clamp)."""
    st = np.floor(t).astype(np.int64) - p // 2
    if clamp:
        st = np.clip(st, 0, n - 1 - p)
    return st, lagrange(t, st, p)


def _accumulate(row, node_of, shape, starts, L, f, factor):
    """row[node] += f * prod_axis L_axis * factor[node] over each point's tensor
    stencil; node_of: grid -> node id (-1: none), shape: grid shape."""
    pa, pb, pc = (Lk.shape[1] - 1 for Lk in L)
    for i in range(pa + 1):
        ia = starts[0] + i
        oka = (ia >= 0) & (ia < shape[0])
        for j in range(pb + 1):
            ib = starts[1] + j
            okab = oka & (ib >= 0) & (ib < shape[1])
            fij = f * L[0][:, i] * L[1][:, j]
            for k in range(pc + 1):
                ic = starts[2] + k
                ok = okab & (ic >= 0) & (ic < shape[2])
                nid = np.full(len(f), -1, np.int64)
                nid[ok] = node_of[ia[ok], ib[ok], ic[ok]]
                good = nid >= 0
                np.add.at(row, nid[good], (fij * L[2][:, k])[good] * factor[nid[good]])


def _unit_dirs(n_mu, n_phi):
    mu, wmu = np.polynomial.legendre.leggauss(n_mu)
    ph = 2 * np.pi * np.arange(n_phi) / n_phi
    MU, PH = np.meshgrid(mu, ph, indexing="ij")
    st = np.sqrt(1 - MU ** 2)
    d = np.stack([st * np.cos(PH), st * np.sin(PH), MU], -1).reshape(-1, 3)
    return d, (wmu[:, None] * np.full(n_phi, 2 * np.pi / n_phi)).ravel()


def k_row(dz, kappa: float, qn: int, ru: Rules3 = Rules3()):
    """Row of K: K[u](x_q) = row . u for the density u at the nodes (phi = u times
    the node's partition values psi omega; m folded in by the caller).  Sum of
    the regular rule with (1 - eta) and every singular rule that reaches x_q."""
    b = dz.b
    x = dz.x[qn]
    row = np.zeros(dz.N, np.complex128)
    eta = np.zeros(dz.N)
    ns = len(dz.s)
    ps = min(ru.p, ns - 1)
    fac_shell = dz.psi * dz.omega                     # phi_F / u on face grids
    fac_cart = dz.omega                               # phi_I / u on the interior grid
    # ---- interior patch: spherical rule about x (any position), if it reaches interior nodes
    cart = np.arange(dz.n_shell, dz.N)
    dc = np.linalg.norm(dz.x[cart] - x, axis=1)
    if np.any(dc < ru.R * b.h):
        s = np.arange(1, ru.n_rho) / ru.n_rho
        rho = ru.R * s ** ru.q
        wr = (1.0 / ru.n_rho) * ru.R * ru.q * s ** (ru.q - 1) * chi(s ** ru.q, ru.chi_s0)
        d, wd = _unit_dirs(ru.n_mu, ru.n_phi)
        RH = np.repeat(rho, len(d))
        W = np.repeat(wr, len(d)) * np.tile(wd, len(rho))
        D = np.tile(d, (len(rho), 1))
        f = W * RH * b.h * b.h * np.exp(1j * kappa * RH * b.h) / (4 * np.pi)
        c = x / b.h + dz.grid_m + RH[:, None] * D                 # grid index coordinates
        st, L = zip(*[_lagrange_cols(c[:, k], ru.p) for k in range(3)])
        _accumulate(row, dz.cart_node, dz.cart_node.shape, st, L, f, fac_cart)
        eta[cart] = chi(dc / (ru.R * b.h), ru.chi_s0)
    # ---- shell patches: a rule on every face whose extended chart holds x
    r_x = np.linalg.norm(x)
    s_x = (b.a - r_x) / b.w                            # depth parameter of x
    is_shell = qn < dz.n_shell
    if s_x < 1.0:
        dirx = x / r_x
        for G in range(6):
            if dirx @ FACES[G][2] <= 1e-12:
                continue
            xi, et = face_coords(G, dirx[None])
            cx, cy = (xi[0] + dz.half) / dz.dg, (et[0] + dz.half) / dz.dg
            if not (0.0 <= cx <= len(dz.g) - 1 and 0.0 <= cy <= len(dz.g) - 1):
                continue
            fn = np.nonzero(dz.face[:dz.n_shell] == G)[0]
            fi, fj, fk = dz.fijk[fn, 0], dz.fijk[fn, 1], dz.fijk[fn, 2]
            if is_shell:
                k0 = int(dz.fijk[qn, 2])
                lines = split_newton_cotes(k0, ns, b.Q)
                sl = np.array([t for t in lines if abs(t - k0) < ru.rs])
                wsl = np.array([lines[t] for t in sl]) * chi((sl - k0) / ru.rs, ru.chi_s0)
                sg = np.arange(1, ru.n_sig) / ru.n_sig
                rho = ru.rc * sg ** ru.q
                wsg = (1.0 / ru.n_sig) * ru.rc * ru.q * sg ** (ru.q - 1) * chi(sg ** ru.q, ru.chi_s0)
                th = 2 * np.pi * np.arange(ru.n_th) / ru.n_th
                SL, RH, TH = np.meshgrid(np.arange(len(sl)), np.arange(len(rho)), th, indexing="ij")
                tk = sl[SL.ravel()]
                rr = rho[RH.ravel()]
                ti = cx + rr * np.cos(TH.ravel())
                tj = cy + rr * np.sin(TH.ravel())
                wq = wsl[SL.ravel()] * wsg[RH.ravel()] * (2 * np.pi / ru.n_th) * rr
                eta_f = chi(np.hypot(fi - cx, fj - cy) / ru.rc, ru.chi_s0) * chi((fk - k0) / ru.rs, ru.chi_s0)
            else:
                cz = s_x / dz.ds
                rsp = min(ru.rs, b.tau0 * (ns - 1))
                s = np.arange(1, ru.n_rho) / ru.n_rho
                rho = s ** ru.q
                wr = (1.0 / ru.n_rho) * ru.q * s ** (ru.q - 1) * chi(rho, ru.chi_s0)
                d, wd = _unit_dirs(ru.n_mu, ru.n_phi)
                RH = np.repeat(rho, len(d))
                wq = np.repeat(wr, len(d)) * np.tile(wd, len(rho)) * RH ** 2 * ru.rc * ru.rc * rsp
                D = np.tile(d, (len(rho), 1))
                ti = cx + ru.rc * RH * D[:, 0]
                tj = cy + ru.rc * RH * D[:, 1]
                tk = cz + rsp * RH * D[:, 2]
                # past the chart's bottom line phi_F is exactly zero (omega_B vanishes
                # from s = tau1 < 1 on): drop those points rather than extrapolate
                wq = np.where(tk <= ns - 1, wq, 0.0)
                eta_f = chi(np.sqrt(((fi - cx) / ru.rc) ** 2 + ((fj - cy) / ru.rc) ** 2 + ((fk - cz) / rsp) ** 2),
                            ru.chi_s0)
            # physical points, Jacobian and kernel
            xi_p = ti * dz.dg - dz.half
            et_p = tj * dz.dg - dz.half
            s_p = tk * dz.ds
            dd, dom = face_direction(G, xi_p, et_p)
            rp = b.a - s_p * b.w
            y = rp[:, None] * dd
            J = b.w * rp ** 2 * dom * dz.dg * dz.dg * dz.ds
            dist = np.linalg.norm(y - x, axis=1)
            f = wq * J * np.exp(1j * kappa * dist) / (4 * np.pi * dist)
            sa, La = _lagrange_cols(ti, ru.p)
            sb, Lb = _lagrange_cols(tj, ru.p)
            sc, Lc = _lagrange_cols(tk, ps, ns, clamp=True)
            _accumulate(row, dz.face_node[G], dz.face_node[G].shape, (sa, sb, sc), (La, Lb, Lc), f, fac_shell)
            eta[fn] = eta_f
    # ---- regular rule with (1 - eta)
    dist = np.linalg.norm(dz.x - x, axis=1)
    G_ = np.zeros(dz.N, np.complex128)
    nz = dist > 0
    G_[nz] = np.exp(1j * kappa * dist[nz]) / (4 * np.pi * dist[nz])
    row += dz.w * dz.omega * G_ * (1.0 - eta)
    return row
