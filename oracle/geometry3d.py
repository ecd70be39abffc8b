"""Three-dimensional discretisation of a penetrable ball (test infrastructure
only): Nystrom nodes, quadrature weights and partitions of unity for the
extension of Section 5.

As in two dimensions (Section 2), the scatterer is covered by boundary patches
along the interface and one interior Cartesian patch, blended by a partition of
unity omega_B + omega_I = 1 that depends on the depth below the surface.  The
paper does not give its shell charts; the reading used here:

* shell: the six faces of a cubed sphere in equiangular coordinates
  (xi, eta) in [-pi/4 - delta, pi/4 + delta]^2 (face frame (e1, e2, e3),
  direction d = normalise(e3 + tan(xi) e1 + tan(eta) e2)), each extended by an
  overlap margin delta and blended on the sphere by a C-infinity partition of
  unity psi_F (normalised products of cut-offs that vanish to all orders at the
  extended edges); depth s in [0, 1] below the surface, radius r = a - s w;
  trapezoid rule in xi and eta (the blended integrand vanishes smoothly at the
  patch edges) and composite Q-point Newton-Cotes in s;
* omega_B(s) = S((s - tau0) / (tau1 - tau0)) on the shell, as in 2-D;
* interior: Cartesian nodes of spacing h with omega_I = 1 - omega_B(depth / w)
  kept where omega_I > 0; weight h^3.

Each node carries its quadrature weight w and its partition value omega, so a
smooth f is integrated over the ball as sum_q w_q omega_q f(x_q).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from .geometry import composite_nc, smooth_step

# face frames (e1, e2, e3): e3 is the face centre direction
FACES = np.array([
    [[0, 1, 0], [0, 0, 1], [1, 0, 0]],
    [[0, 0, 1], [0, 1, 0], [-1, 0, 0]],
    [[0, 0, 1], [1, 0, 0], [0, 1, 0]],
    [[1, 0, 0], [0, 0, 1], [0, -1, 0]],
    [[1, 0, 0], [0, 1, 0], [0, 0, 1]],
    [[0, 1, 0], [1, 0, 0], [0, 0, -1]],
], dtype=np.float64)


@dataclass
class Ball3:
    """Parameters of the 3-D discretisation (radius, shell and interior grids)."""
    a: float = 1.0            # radius
    w: float = 0.5            # shell thickness
    n_f: int = 17             # points per shell-face side (xi and eta)
    n_s: int = 9              # points across the shell ((Q - 1) k + 1)
    Q: int = 5                # Newton-Cotes points across the shell
    delta: float = 0.25       # angular overlap of the faces
    h: float = 0.1            # interior grid spacing
    tau0: float = 0.3
    tau1: float = 0.95
    kappa: float = 2.0
    n2c: float = 2.0          # constant n^2 inside


def face_direction(F: int, xi, eta):
    """Unit direction of equiangular coordinates (xi, eta) on face F, and the
    solid-angle element dOmega / (dxi deta)."""
    e1, e2, e3 = FACES[F]
    t1, t2 = np.tan(xi), np.tan(eta)
    v = e3 + t1[..., None] * e1 + t2[..., None] * e2
    nrm = np.sqrt(1.0 + t1 ** 2 + t2 ** 2)
    d = v / nrm[..., None]
    dom = (1.0 + t1 ** 2) * (1.0 + t2 ** 2) / nrm ** 3
    return d, dom


def face_coords(F: int, d):
    """Equiangular coordinates of direction d (..., 3) on face F (valid where
    d . e3 > 0)."""
    e1, e2, e3 = FACES[F]
    z = d @ e3
    return np.arctan2(d @ e1, z), np.arctan2(d @ e2, z)


def face_bump(xi, eta, delta):
    """1 on |xi|, |eta| <= pi/4 - delta, 0 from pi/4 + delta on, C-infinity."""
    lo, hi = math.pi / 4 - delta, math.pi / 4 + delta
    c = lambda x: smooth_step((np.abs(x) - lo) / (hi - lo))
    return c(xi) * c(eta)


def surface_pou(F: int, d, delta):
    """psi_F(d): face F's share of the smooth partition of unity on the sphere."""
    num = np.zeros(d.shape[:-1])
    den = np.zeros(d.shape[:-1])
    for G in range(6):
        ok = d @ FACES[G][2] > 1e-12
        xi, eta = np.zeros(den.shape), np.zeros(den.shape)
        xi[ok], eta[ok] = face_coords(G, d[ok])
        b = np.where(ok, face_bump(xi, eta, delta), 0.0)
        den += b
        if G == F:
            num = b
    return num / den


class Discretisation3:
    """Nystrom node set of the ball: six shell patches, then the interior grid.

    Per node: position x, weight w, partition value omega, chart (0 shell, 1
    interior), and for shell nodes the face, (xi, eta) and depth s."""

    def __init__(self, b: Ball3):
        self.b = b
        nf, ns = b.n_f, b.n_s
        half = math.pi / 4 + b.delta
        g = np.linspace(-half, half, nf)
        dg = g[1] - g[0]
        s = np.linspace(0.0, 1.0, ns)
        ws = composite_nc(ns, b.Q) * (s[1] - s[0])
        XI, ETA, S = np.meshgrid(g, g, s, indexing="ij")
        WS = np.broadcast_to(ws, S.shape)
        self.g, self.dg, self.s, self.ds, self.half = g, dg, s, s[1] - s[0], half
        X, W, OM, CH, FC, PS, IJK = [], [], [], [], [], [], []
        II, JJ, KK = np.meshgrid(np.arange(nf), np.arange(nf), np.arange(ns), indexing="ij")
        for F in range(6):
            d, dom = face_direction(F, XI, ETA)
            r = b.a - S * b.w
            psi = surface_pou(F, d, b.delta)
            wq = dg * dg * WS * b.w * r ** 2 * dom * psi
            keep = wq > 0.0
            X.append((r[..., None] * d)[keep])
            W.append(wq[keep])
            OM.append(smooth_step((S[keep] - b.tau0) / (b.tau1 - b.tau0)))
            CH.append(np.zeros(int(keep.sum()), np.int8))
            FC.append(np.full(int(keep.sum()), F, np.int8))
            PS.append(psi[keep])
            IJK.append(np.stack([II[keep], JJ[keep], KK[keep]], -1))
        # interior Cartesian grid: omega_I = 1 - omega_B(depth / w), kept where > 0
        m = int(math.ceil(b.a / b.h))
        ax = b.h * np.arange(-m, m + 1)
        GX, GY, GZ = np.meshgrid(ax, ax, ax, indexing="ij")
        P = np.stack([GX.ravel(), GY.ravel(), GZ.ravel()], -1)
        depth = (b.a - np.linalg.norm(P, axis=-1)) / b.w
        omi = np.where(depth > 0, 1.0 - smooth_step((depth - b.tau0) / (b.tau1 - b.tau0)), 0.0)
        keep = omi > 0.0
        self.grid_m = m                               # grid indices -m..m per axis
        self.grid_omega = omi.reshape(GX.shape)       # omega_I on the whole grid (0 outside)
        X.append(P[keep])
        W.append(np.full(int(keep.sum()), b.h ** 3))
        OM.append(omi[keep])
        CH.append(np.ones(int(keep.sum()), np.int8))
        FC.append(np.full(int(keep.sum()), -1, np.int8))
        gidx = np.stack(np.unravel_index(np.nonzero(keep)[0], GX.shape), -1)
        self.x = np.concatenate(X)
        self.w = np.concatenate(W)
        self.omega = np.concatenate(OM)
        self.chart = np.concatenate(CH)
        self.face = np.concatenate(FC)
        self.N = len(self.x)
        self.n_shell = int((self.chart == 0).sum())
        self.n_cart = self.N - self.n_shell
        # shell nodes: partition share psi_F and face-grid indices; grid -> node maps
        self.psi = np.concatenate(PS + [np.zeros(self.n_cart)])
        self.fijk = np.concatenate(IJK + [np.full((self.n_cart, 3), -1)])
        self.face_node = np.full((6, nf, nf, ns), -1, np.int64)
        sh = np.arange(self.n_shell)
        self.face_node[self.face[sh], self.fijk[sh, 0], self.fijk[sh, 1], self.fijk[sh, 2]] = sh
        self.cart_node = np.full(GX.shape, -1, np.int64)
        self.cart_node[gidx[:, 0], gidx[:, 1], gidx[:, 2]] = self.n_shell + np.arange(self.n_cart)

    def integrate(self, f):
        """sum_q w_q omega_q f(x_q) for values f (N,) or a callable of x (N, 3)."""
        v = f(self.x) if callable(f) else np.asarray(f)
        return np.sum(self.w * self.omega * v)
