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
