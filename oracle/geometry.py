"""Charts, partition of unity and the Nystrom node set (test infrastructure only).

Follows Section 2 of the paper: the scatterer is covered by overlapping patches
P_k = xi_k(H_k) with a smooth partition of unity omega_k; the Nystrom nodes are
the images of equispaced parameter grids (the node-set equation of Section 2).
Readings (the paper leaves these open): one periodic boundary "collar" chart
built along the inward normal, plus one Cartesian interior patch; omega_B is a
C-infinity step in the transverse coordinate and omega_I = 1 - omega_B.

Everything is expressed in *grid-index units*: the collar chart is
X(a, b) = gamma(2 pi a / n1) - (b / (n2 - 1)) w nu(2 pi a / n1), so a unit step
in a or b is one grid spacing, and its Jacobian J(a, b) includes the
index-to-parameter scaling.  The Cartesian chart is X(a, b) = (x0 + a h, y0 + b h).
"""
from __future__ import annotations

import math

import numpy as np
from scipy.spatial import cKDTree

from workloads import Workload, n2_eval


# ---------------------------------------------------------------- curves
def curve(wl: Workload, s):
    """gamma(s), gamma'(s), gamma''(s) for the workload's boundary curve."""
    s = np.asarray(s, dtype=np.float64)
    c1, s1 = np.cos(s), np.sin(s)
    if wl.shape == "disc":
        a, cx, cy = wl.shape_params
        g = np.stack([cx + a * c1, cy + a * s1], -1)
        g1 = np.stack([-a * s1, a * c1], -1)
        g2 = np.stack([-a * c1, -a * s1], -1)
    elif wl.shape == "kite":
        sc, cx, cy = wl.shape_params
        c2, s2 = np.cos(2 * s), np.sin(2 * s)
        g = np.stack([cx + sc * (c1 + 0.65 * c2 - 0.65), cy + sc * 1.5 * s1], -1)
        g1 = np.stack([sc * (-s1 - 1.3 * s2), sc * 1.5 * c1], -1)
        g2 = np.stack([sc * (-c1 - 2.6 * c2), -sc * 1.5 * s1], -1)
    elif wl.shape == "star":
        # gamma = c + r(s) (cos s, sin s), r = a0 + sum_k c_k cos(k s), k = 1..5
        a0, cx, cy = wl.shape_params[:3]
        ck = np.zeros(5)
        ck[:len(wl.shape_params) - 3] = wl.shape_params[3:]
        k = np.arange(1, 6)
        ks = np.multiply.outer(s, k)
        r = a0 + np.cos(ks) @ ck
        r1 = -np.sin(ks) @ (k * ck)
        r2 = -np.cos(ks) @ (k * k * ck)
        g = np.stack([cx + r * c1, cy + r * s1], -1)
        g1 = np.stack([r1 * c1 - r * s1, r1 * s1 + r * c1], -1)
        g2 = np.stack([r2 * c1 - 2 * r1 * s1 - r * c1, r2 * s1 + 2 * r1 * c1 - r * s1], -1)
    else:
        raise ValueError(wl.shape)
    return g, g1, g2


def outward_normal(g1, g2):
    """nu and d nu / ds for a counter-clockwise curve."""
    sp = np.sqrt(g1[..., 0] ** 2 + g1[..., 1] ** 2)
    nu = np.stack([g1[..., 1], -g1[..., 0]], -1) / sp[..., None]
    dot = g1[..., 0] * g2[..., 0] + g1[..., 1] * g2[..., 1]
    dnu = (np.stack([g2[..., 1], -g2[..., 0]], -1) / sp[..., None]
           - np.stack([g1[..., 1], -g1[..., 0]], -1) * (dot / sp ** 3)[..., None])
    return nu, dnu


def collar_map(wl: Workload, a, b):
    """Collar chart X(a, b) and its Jacobian |det DX| in grid-index units."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    s = 2.0 * math.pi * a / wl.n1
    t = b / (wl.n2 - 1)
    g, g1, g2 = curve(wl, s)
    nu, dnu = outward_normal(g1, g2)
    w = wl.collar_w
    X = g - (t * w)[..., None] * nu
    Xs = g1 - (t * w)[..., None] * dnu          # dX/ds
    Xt = -w * nu                                   # dX/dt
    det = Xs[..., 0] * Xt[..., 1] - Xs[..., 1] * Xt[..., 0]
    J = np.abs(det) * (2.0 * math.pi / wl.n1) / (wl.n2 - 1)
    return X, J


def cart_map(wl: Workload, a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    X = np.stack([wl.cart_x0 + a * wl.h, wl.cart_y0 + b * wl.h], -1)
    J = np.full(a.shape, wl.h * wl.h)
    return X, J


def closest_point(wl: Workload, x, nsamp: int = 16384, iters: int = 40):
    """Foot point s* of x on the boundary curve and the signed depth d = (gamma - x) . nu.

    d > 0 inside the scatterer.  Newton on f(s) = (x - gamma(s)) . gamma'(s)
    started from the nearest of nsamp equispaced samples in s.
    """
    x = np.atleast_2d(np.asarray(x, dtype=np.float64))
    ss = 2.0 * math.pi * np.arange(nsamp) / nsamp
    gs, _, _ = curve(wl, ss)
    _, k = cKDTree(gs).query(x)
    s = ss[k]
    for _ in range(iters):
        g, g1, g2 = curve(wl, s)
        dx = x - g
        f = np.sum(dx * g1, -1)
        fp = -np.sum(g1 * g1, -1) + np.sum(dx * g2, -1)
        ok = np.abs(fp) > 1e-300
        ds = np.where(ok, f / np.where(ok, fp, 1.0), 0.0)
        s = s - ds
        if np.max(np.abs(ds)) < 1e-15:
            break
    s = np.mod(s, 2.0 * math.pi)
    g, g1, g2 = curve(wl, s)
    nu, _ = outward_normal(g1, g2)
    d = np.sum((g - x) * nu, -1)
    return s, d


# ---------------------------------------------------------------- POU
def smooth_step(u):
    """S(u) = 1 for u <= 0, 0 for u >= 1, C-infinity in between."""
    u = np.asarray(u, dtype=np.float64)
    out = np.where(u <= 0.0, 1.0, 0.0)
    mid = (u > 0.0) & (u < 1.0)
    um = u[mid]
    f1 = np.exp(-1.0 / (1.0 - um))
    f0 = np.exp(-1.0 / um)
    out[mid] = f1 / (f1 + f0)
    return out


def omega_collar(wl: Workload, t):
    """omega_B as a function of the transverse parameter t = b / (n2 - 1)."""
    return smooth_step((np.asarray(t) - wl.tau0) / (wl.tau1 - wl.tau0))


# ---------------------------------------------------------------- Newton-Cotes
def newton_cotes(Q: int) -> np.ndarray:
    """Closed Q-point Newton-Cotes weights for unit node spacing."""
    table = {
        2: [1, 1], 3: [1, 4, 1], 4: [1, 3, 3, 1], 5: [7, 32, 12, 32, 7],
    }
    scale = {2: 1 / 2, 3: 1 / 3, 4: 3 / 8, 5: 2 / 45}
    return np.array(table[Q], dtype=np.float64) * scale[Q]


def composite_nc(n: int, Q: int) -> np.ndarray:
    """Composite Q-point Newton-Cotes weights on nodes 0..n-1 (unit spacing)."""
    if (n - 1) % (Q - 1):
        raise ValueError("n - 1 must be a multiple of Q - 1")
    w = np.zeros(n)
    nc = newton_cotes(Q)
    for blk in range((n - 1) // (Q - 1)):
        w[blk * (Q - 1): blk * (Q - 1) + Q] += nc
    return w


# ---------------------------------------------------------------- node set
class Discretisation:
    """The Nystrom node set T = union of the collar and Cartesian grids.

    Canonical node order: collar nodes first, id = i * n2 + j (i tangential,
    j transverse), then the Cartesian nodes with omega_I > 0 in increasing
    ix * cart_ny + iy order.
    """

    def __init__(self, wl: Workload, interp=None):
        self.wl = wl
        # None: degree-p Lagrange interpolation in the singular rules; (F, pf):
        # the Fourier-refined comparison variant (see quadrature.py)
        self.interp = interp
        n1, n2 = wl.n1, wl.n2
        ii, jj = np.meshgrid(np.arange(n1), np.arange(n2), indexing="ij")
        ii, jj = ii.ravel(), jj.ravel()
        Xc, Jc = collar_map(wl, ii.astype(float), jj.astype(float))
        ncw = composite_nc(n2, wl.Q)
        w_c = Jc * ncw[jj]
        om_c = omega_collar(wl, jj / (n2 - 1))

        # Cartesian candidates: keep omega_I > 0, i.e. inside and t > tau0.
        gx, gy = np.meshgrid(np.arange(wl.cart_nx), np.arange(wl.cart_ny), indexing="ij")
        gx, gy = gx.ravel(), gy.ravel()
        Xg, _ = cart_map(wl, gx.astype(float), gy.astype(float))
        s, d = closest_point(wl, Xg)
        t = d / wl.collar_w
        keep = t > wl.tau0
        gx, gy, Xg, s, t = gx[keep], gy[keep], Xg[keep], s[keep], t[keep]
        om_g = 1.0 - omega_collar(wl, t)

        self.n_collar = n1 * n2
        self.n_cart = len(gx)
        self.N = self.n_collar + self.n_cart
        self.x = np.concatenate([Xc, Xg])
        self.chart = np.concatenate([np.zeros(self.n_collar, np.int8), np.ones(self.n_cart, np.int8)])
        self.gi = np.concatenate([ii, gx])
        self.gj = np.concatenate([jj, gy])
        self.w = np.concatenate([w_c, np.full(self.n_cart, wl.h * wl.h)])
        self.omega = np.concatenate([om_c, om_g])
        self.n2 = n2_eval(wl.n2_kind, wl.n2_params, self.x)
        self.m = 1.0 - self.n2
        self.phifac = self.omega * self.m          # phi_k = m u omega_k at the node
        self.wfac = self.w * self.phifac           # regular-rule factor w m omega

        # collar coordinates (a, b) of every node; Cartesian nodes from the inverse map
        self.ca = np.concatenate([ii.astype(float), s * n1 / (2.0 * math.pi)])
        self.cb = np.concatenate([jj.astype(float), t * (n2 - 1)])
        # Cartesian index coordinates of every node
        self.ga = (self.x[:, 0] - wl.cart_x0) / wl.h
        self.gb = (self.x[:, 1] - wl.cart_y0) / wl.h
        self.ga[self.n_collar:] = gx
        self.gb[self.n_collar:] = gy

        self.cart_id = -np.ones((wl.cart_nx, wl.cart_ny), np.int64)
        self.cart_id[gx, gy] = self.n_collar + np.arange(self.n_cart)
        self.collar_id = np.arange(self.n_collar).reshape(n1, n2)

        self._check()

    def _check(self):
        wl = self.wl
        if not (0.0 < wl.tau0 < wl.tau1 < 1.0):
            raise ValueError("need 0 < tau0 < tau1 < 1")
        if wl.n2 < wl.p + 1:
            raise ValueError("collar needs at least p+1 transverse lines")
