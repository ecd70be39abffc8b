"""Three-dimensional equivalent-source / lattice-FFT accelerator (test
infrastructure only): the extension of Section 3.2 that Section 5 names, with
two-face equivalent sources on cube cells and a three-dimensional FFT.

The steps mirror the two-dimensional accelerator:

1. cube cells C_ijk of side H = A / L cover the bounding cube; N(x) is the
   3 x 3 x 3 block around the cell of x.  Only the non-adjacent part (every
   node outside N(x)) is accelerated; the adjacent part and the singular rules
   stay with the direct rows.
2. per cell, monopoles and x1-dipoles (d/dy_1) sit on the (N_eq + 1)^2 lattice
   points of each of the cell's two x1-faces (4 (N_eq + 1)^2 unknowns); they
   are the least-squares fit to the cell's true-source field at collocation
   points on the boundary of the 3H cube centred on the cell (one shared
   factorisation: all cells have the same geometry).
3. the field of all equivalent sources on the lattice of spacing
   delta = H / N_eq is a discrete convolution done by a zero-padded 3-D FFT;
   the 27 neighbours' equivalent-source fields are subtracted with the same
   kernel tables (zero at coincident points).
4. per cell, the non-adjacent field on the closed cell's lattice points is
   fitted by a truncated spherical-wave expansion
   j_l(kappa r) Y_l^m(theta, phi) / j_l(kappa R_ref), l <= p (the 3-D form of
   the 2-D Fourier-Bessel reading of Eq. PWE) and evaluated at the nodes.

Kernel: G(x, y) = exp(i kappa |x - y|) / (4 pi |x - y|) (Section 5).
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import lpmv, spherical_jn

from .accel import RCOND, _fft_size, _lstsq_apply, _svd  # noqa: F401  (shared linear algebra)


def mono3(kappa, dx, dy, dz):
    """G(x - z) = exp(i kappa r) / (4 pi r)."""
    r = np.sqrt(dx * dx + dy * dy + dz * dz)
    return np.exp(1j * kappa * r) / (4 * np.pi * r)


def dip3(kappa, dx, dy, dz):
    """dG(x, z)/dz_1 = exp(i kappa r) (1 - i kappa r) (x_1 - z_1) / (4 pi r^3)."""
    r = np.sqrt(dx * dx + dy * dy + dz * dz)
    return np.exp(1j * kappa * r) * (1 - 1j * kappa * r) * dx / (4 * np.pi * r ** 3)


def spherical_wave_basis(kappa, x, y, z, p, Rref):
    """Columns j_l(kappa r) N_lm P_l^|m|(cos theta) e^{i m phi} / j_l(kappa R_ref),
    0 <= l <= p, -l <= m <= l ((p + 1)^2 regular Helmholtz solutions)."""
    r = np.sqrt(x * x + y * y + z * z)
    ct = np.where(r > 0, z / np.where(r > 0, r, 1.0), 1.0)
    ph = np.arctan2(y, x)
    cols = []
    for l in range(p + 1):
        jl = spherical_jn(l, kappa * r) / spherical_jn(l, kappa * Rref)
        for m in range(-l, l + 1):
            am = abs(m)
            nrm = math.sqrt((2 * l + 1) / (4 * math.pi) * math.exp(math.lgamma(l - am + 1) - math.lgamma(l + am + 1)))
            cols.append(jl * nrm * lpmv(am, l, ct) * np.exp(1j * m * ph))
    return np.stack(cols, -1)


class Cells3:
    """Cube cells of side H covering [x0, x0 + L H]^3."""

    def __init__(self, x, x0: float, H: float, L: int):
        self.x0, self.H, self.L = x0, H, L
        c = np.floor((x - x0) / H).astype(np.int64)
        if c.min() < 0 or c.max() >= L:
            raise ValueError("nodes outside the cell box")
        self.ci = c
        self.cell = (c[:, 2] * L + c[:, 1]) * L + c[:, 0]
        order = np.argsort(self.cell, kind="stable")
        bounds = np.searchsorted(self.cell[order], np.arange(L ** 3 + 1))
        self.members = [order[bounds[k]:bounds[k + 1]] for k in range(L ** 3)]

    def near_mask(self, rows, cols=None):
        rows = np.asarray(rows)
        cs = self.ci if cols is None else self.ci[cols]
        return np.all(np.abs(cs[None, :, :] - self.ci[rows, None, :]) <= 1, axis=-1)


class Accelerator3:
    """Non-adjacent part of the 3-D operator by equivalent sources and a 3-D FFT.

    wfac: per-node factor w omega m that multiplies u in the sum (Eq.
    disctete-conv's weights in 3-D); p: degree of the local expansion;
    m_coll: collocation points per side of each face of the 3H cube."""

    def __init__(self, x, wfac, kappa: float, x0: float, H: float, L: int, Ne: int,
                 p: int | None = None, m_coll: int | None = None, local_points: str = "cell"):
        if local_points not in ("cell", "boundary"):
            raise ValueError(local_points)
        self.x, self.wfac = np.asarray(x, float), np.asarray(wfac)
        self.kappa, self.H, self.L, self.Ne = kappa, H, L, Ne
        self.cells = Cells3(self.x, x0, H, L)
        self.delta = H / Ne
        self.Rref = math.sqrt(3.0) * H / 2
        if kappa * self.Rref >= math.pi:
            raise ValueError("kappa R_ref must stay below the first zero of j_0")
        self.p = p if p is not None else 2 * Ne + 1
        # equivalent sources (lattice units, corner frame): two x1-faces, mono + dipole
        bb, cc = np.meshgrid(np.arange(Ne + 1), np.arange(Ne + 1), indexing="ij")
        bb, cc = bb.ravel(), cc.ravel()
        nf = len(bb)
        a = np.concatenate([np.zeros(nf), np.full(nf, Ne)]).astype(np.int64)
        b = np.concatenate([bb, bb])
        c = np.concatenate([cc, cc])
        self.es = np.stack([np.concatenate([a, a]), np.concatenate([b, b]), np.concatenate([c, c])], -1)
        self.es_kind = np.concatenate([np.zeros(2 * nf, np.int64), np.ones(2 * nf, np.int64)])
        self.n_es = 4 * nf
        m = m_coll if m_coll is not None else int(math.ceil(math.sqrt(2.0 * self.n_es / 6.0))) + 1
        self.coll = self._collocation(m)
        self.Asvd = _svd(self._es_field(self.coll))
        # lattice points of the local fit (corner frame, lattice units)
        g = np.arange(Ne + 1)
        la = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
        if local_points == "boundary":
            la = la[np.any((la == 0) | (la == Ne), axis=1)]
        self.loc = la
        self.n_loc = len(la)
        B = self._basis(la * self.delta - H / 2)
        if B.shape[1] > self.n_loc:
            raise ValueError("local expansion has more terms than fit points")
        self.Bsvd = _svd(B)
        # neighbour tables T_o (n_loc, n_es) for o in {-1, 0, 1}^3
        self.T = {}
        for o in np.ndindex(3, 3, 3):
            off = np.array(o) - 1
            d = self.loc[:, None, :] - (self.es[None, :, :] + off * Ne)
            self.T[tuple(off)] = self._table(d, self.es_kind[None, :])
        # per-cell projection (w omega m folded in) and evaluation matrices
        self.P, self.Phi = {}, {}
        for cell, mem in enumerate(self.cells.members):
            if len(mem) == 0:
                continue
            rel = self.x[mem] - self._corner(cell)
            Gc = mono3(kappa, *(self.coll[:, None, k] - rel[None, :, k] for k in range(3)))
            self.P[cell] = _lstsq_apply(self.Asvd, Gc) * self.wfac[mem][None, :]
            self.Phi[cell] = self._basis(rel - H / 2)
        # lattice FFT
        self.n_lat = L * Ne + 1
        self.M = _fft_size(2 * self.n_lat - 1)
        off = np.arange(self.M)
        off = np.where(off < self.M - self.n_lat + 1, off, off - self.M)
        D = np.stack(np.meshgrid(off, off, off, indexing="ij"), -1)
        self.Ghat = np.fft.fftn(self._table(D, 0))
        self.Dhat = np.fft.fftn(self._table(D, 1))

    # ------------------------------------------------------------------ pieces
    def _corner(self, cell):
        L = self.L
        return self.cells.x0 + self.H * np.array([cell % L, (cell // L) % L, cell // (L * L)], float)

    def _collocation(self, m):
        """m x m face midpoints on each face of the cube [-H, 2H]^3 (corner frame)."""
        H = self.H
        t = -H + (np.arange(m) + 0.5) / m * 3 * H
        U, V = np.meshgrid(t, t, indexing="ij")
        U, V = U.ravel(), V.ravel()
        pts = []
        for ax in range(3):
            for side in (-H, 2 * H):
                q = np.empty((len(U), 3))
                q[:, ax] = side
                q[:, (ax + 1) % 3] = U
                q[:, (ax + 2) % 3] = V
                pts.append(q)
        return np.concatenate(pts)

    def _es_field(self, pts):
        z = self.es * self.delta
        d = [pts[:, None, k] - z[None, :, k] for k in range(3)]
        return np.where(self.es_kind[None, :] == 0, mono3(self.kappa, *d), dip3(self.kappa, *d))

    def _table(self, d, kind):
        """G or dG/dz_1 at lattice offsets d (..., 3), zero at the origin."""
        d = np.asarray(d, float)
        zero = np.all(d == 0, axis=-1)
        dx = np.where(zero, 1.0, d[..., 0]) * self.delta
        dy, dz = d[..., 1] * self.delta, d[..., 2] * self.delta
        val = np.where(np.asarray(kind) == 0, mono3(self.kappa, dx, dy, dz), dip3(self.kappa, dx, dy, dz))
        return np.where(zero, 0.0, val)

    def _basis(self, rel):
        return spherical_wave_basis(self.kappa, rel[:, 0], rel[:, 1], rel[:, 2], self.p, self.Rref)

    # ------------------------------------------------------------------ apply
    def project(self, u):
        return {c: P @ u[self.cells.members[c]] for c, P in self.P.items()}

    def lattice_field(self, sig):
        Sm = np.zeros((self.M,) * 3, np.complex128)
        Sd = np.zeros((self.M,) * 3, np.complex128)
        L, Ne = self.L, self.Ne
        mono = self.es_kind == 0
        for cell, s in sig.items():
            g = np.array([cell % L, (cell // L) % L, cell // (L * L)]) * Ne + self.es
            np.add.at(Sm, (g[mono, 0], g[mono, 1], g[mono, 2]), s[mono])
            np.add.at(Sd, (g[~mono, 0], g[~mono, 1], g[~mono, 2]), s[~mono])
        V = np.fft.ifftn(np.fft.fftn(Sm) * self.Ghat + np.fft.fftn(Sd) * self.Dhat)
        n = self.n_lat
        return V[:n, :n, :n]

    def local_data(self, V, sig):
        """beta_c: non-adjacent field on the cell's fit points."""
        L, Ne = self.L, self.Ne
        out = {}
        for cell in self.P:
            ijk = np.array([cell % L, (cell // L) % L, cell // (L * L)])
            g = ijk * Ne + self.loc
            beta = V[g[:, 0], g[:, 1], g[:, 2]].copy()
            for off, T in self.T.items():
                nb = ijk + np.array(off)
                if np.all((nb >= 0) & (nb < L)):
                    nc = int((nb[2] * L + nb[1]) * L + nb[0])
                    if nc in sig:
                        beta -= T @ sig[nc]
            out[cell] = beta
        return out

    def evaluate(self, beta):
        v = np.zeros(len(self.x), np.complex128)
        for cell, b in beta.items():
            v[self.cells.members[cell]] = self.Phi[cell] @ _lstsq_apply(self.Bsvd, b[:, None])[:, 0]
        return v

    def apply_far(self, u):
        sig = self.project(np.asarray(u, np.complex128))
        return self.evaluate(self.local_data(self.lattice_field(sig), sig))

    def direct_far(self, u, rows=None):
        """Exact non-adjacent sum for comparison."""
        rows = np.arange(len(self.x)) if rows is None else np.asarray(rows)
        out = np.zeros(len(rows), np.complex128)
        y = self.wfac * np.asarray(u, np.complex128)
        for s in range(0, len(rows), 256):
            r = rows[s:s + 256]
            far = ~self.cells.near_mask(r)
            d = [self.x[None, :, k] - self.x[r, None, k] for k in range(3)]
            d[0] = np.where(far, d[0], 1.0)
            out[s:s + 256] = np.where(far, mono3(self.kappa, *d), 0.0) @ y
        return out
