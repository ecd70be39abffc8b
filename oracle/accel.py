"""Equivalent-source / lattice-FFT accelerator of Section 3.2 (test infrastructure only).

The steps follow the paper's order and notation:

1. cells C_ij of side H = A / L cover the bounding square; N(x) is the 3 x 3
   block around the cell of x (Eq. setdef-Adj).  The adjacent part of the
   operator (regular (1 - eta) terms within N(x) plus every singular rule) is
   applied directly; eta must vanish outside N(x) (checked here).
2. per cell, monopoles sigma^(m) and dipoles sigma^(d) (d/dy_1) sit at
   equispaced points on the two x_1-faces of the cell (Eq. equiv-conv-loc);
   they are the least-squares fit A sigma = b to the cell's true-source field
   at n_coll points on the boundary of the 3 x 3 block.  The pseudo-inverse of
   A is computed once (all cells share the geometry).
3. the field of all equivalent sources on the lattice of spacing
   delta = H / N_eq is a discrete convolution done by zero-padded FFT; the
   3 x 3 neighbours' equivalent-source fields are subtracted with the same
   kernel tables (zero at coincident points), which leaves the non-adjacent
   field on every lattice point of the closed cell.
4. per cell, the non-adjacent field is fitted by a truncated expansion of
   Helmholtz solutions and evaluated at the cell's Nystrom nodes (the paper's
   Eq. PWE).  Reading: the plane-wave expansion is used in its Jacobi-Anger
   (Fourier-Bessel) form J_n(kappa r) e^{i n theta} / J_|n|(kappa R_ref),
   |n| <= n_fb, which spans the same Helmholtz solutions but stays well
   conditioned for kappa H ~ 1; the fit uses every lattice point of the
   closed cell (faces and interior).  local_basis="pw" keeps the literal plane
   waves instead (the paper's form, for comparison).
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp
from scipy.special import j0, j1, jv, y0, y1

from . import quadrature as qd
from .geometry import Discretisation
from .operator import regular_rows, singular_matrix

RCOND = 1e-13


def h0(z):
    return j0(z) + 1j * y0(z)


def h1(z):
    return j1(z) + 1j * y1(z)


def mono_kernel(kappa, dx, dy):
    """G(x - z) = (i/4) H_0(kappa r)."""
    r = np.hypot(dx, dy)
    return 0.25j * h0(kappa * r)


def dip_kernel(kappa, dx, dy):
    """dG(x, z)/dz_1 = (i kappa / 4) H_1(kappa r) (x_1 - z_1) / r."""
    r = np.hypot(dx, dy)
    return 0.25j * kappa * h1(kappa * r) * dx / r


class Cells:
    """Cell decomposition of the bounding square (Section 3, adjacency)."""

    def __init__(self, dz: Discretisation):
        wl = dz.wl
        self.L, self.H = wl.L, wl.H
        self.x0, self.y0 = wl.box_x0, wl.box_y0
        ci = np.floor((dz.x[:, 0] - self.x0) / self.H).astype(np.int64)
        cj = np.floor((dz.x[:, 1] - self.y0) / self.H).astype(np.int64)
        if ci.min() < 0 or cj.min() < 0 or ci.max() >= self.L or cj.max() >= self.L:
            raise ValueError("nodes outside the cell box")
        self.ci, self.cj = ci, cj
        self.cell = cj * self.L + ci
        self.members = [np.nonzero(self.cell == c)[0] for c in range(self.L * self.L)]

    def near_mask(self, rows, cols=None):
        rows = np.asarray(rows)
        ci_s = self.ci if cols is None else self.ci[cols]
        cj_s = self.cj if cols is None else self.cj[cols]
        return ((np.abs(ci_s[None, :] - self.ci[rows, None]) <= 1)
                & (np.abs(cj_s[None, :] - self.cj[rows, None]) <= 1))


def near_matrix(dz: Discretisation, cells: Cells, rows=None, chunk: int = 512):
    """Adjacent part of K: (1 - eta) regular terms restricted to N(x) plus all
    singular rules (first two terms of Eq. VolInt-Adj-NonAdj-I)."""
    if rows is None:
        rows = np.arange(dz.N)
    rows = np.asarray(rows)
    parts = []
    for s in range(0, len(rows), chunk):
        r = rows[s:s + chunk]
        reg = regular_rows(dz, r)
        near = cells.near_mask(r)
        eta_far = qd.eta_regular(dz, r)[~near]
        if np.any(eta_far != 0.0):
            raise ValueError("cut-off support leaves N(x): enlarge H or shrink R")
        reg[~near] = 0.0
        parts.append(sp.csr_matrix(reg))
    reg = sp.vstack(parts).tocsr()
    return reg + singular_matrix(dz, rows)


class Accelerator:
    """Far (non-adjacent) part of K via equivalent sources and the lattice FFT."""

    def __init__(self, dz: Discretisation, cells: Cells | None = None, local_basis: str = "fb",
                 local_points: str = "cell"):
        wl = dz.wl
        self.dz = dz
        if local_basis not in ("fb", "pw"):
            raise ValueError(local_basis)
        if local_points not in ("cell", "boundary", "two_faces"):
            raise ValueError(local_points)
        self.local_basis = local_basis
        self.cells = cells if cells is not None else Cells(dz)
        k = self.kappa = wl.kappa
        Ne = self.Ne = wl.N_eq
        H = self.H = wl.H
        L = self.L = wl.L
        self.delta = H / Ne
        if k * H / math.sqrt(2.0) >= 2.4:
            raise ValueError("kappa H / sqrt(2) must stay below the first zero of J_0")
        # equivalent sources relative to the cell's lower-left corner (lattice units)
        kk = np.arange(Ne + 1)
        es_a = np.concatenate([np.zeros(Ne + 1), np.full(Ne + 1, Ne)])
        es_b = np.concatenate([kk, kk]).astype(float)
        self.es_a = np.concatenate([es_a, es_a]).astype(np.int64)
        self.es_b = np.concatenate([es_b, es_b]).astype(np.int64)
        self.es_kind = np.concatenate([np.zeros(2 * (Ne + 1), np.int64), np.ones(2 * (Ne + 1), np.int64)])
        self.n_es = 4 * (Ne + 1)
        ncoll = wl.n_coll if wl.n_coll else 4 * self.n_es
        self.coll = self._collocation(ncoll)
        A = self._es_field(self.coll[:, 0], self.coll[:, 1])        # (ncoll, n_es)
        self.Asvd = _svd(A)
        # lattice points of the local fit relative to the corner: the closed cell
        # (faces and interior; the build's reading), or comparison variants: its
        # boundary only (the points on all four faces), or only the two
        # x1-faces that carry equivalent sources (the paper-literal two-face data)
        la, lb = np.meshgrid(np.arange(Ne + 1), np.arange(Ne + 1), indexing="ij")
        la, lb = la.ravel(), lb.ravel()
        on_x1_face = (la == 0) | (la == Ne)
        keep = {"cell": np.ones(la.shape, bool), "two_faces": on_x1_face,
                "boundary": on_x1_face | (lb == 0) | (lb == Ne)}[local_points]
        self.loc_a, self.loc_b = la[keep], lb[keep]
        self.n_loc = len(self.loc_a)
        # local expansion (Fourier-Bessel form of Eq. PWE)
        self.nfb = wl.n_fb
        self.Rref = H / math.sqrt(2.0)
        xb = self.loc_a * self.delta - H / 2
        yb = self.loc_b * self.delta - H / 2
        B = self._local_basis(xb, yb)                                # (n_loc, 2 nfb + 1)
        self.Bpinv = _lstsq_apply(_svd(B), np.eye(self.n_loc))
        # neighbour tables T_o (n_loc, n_es) for offsets o in {-1,0,1}^2
        self.T = {}
        for oi in (-1, 0, 1):
            for oj in (-1, 0, 1):
                da = self.loc_a[:, None] - (self.es_a[None, :] + oi * Ne)
                db = self.loc_b[:, None] - (self.es_b[None, :] + oj * Ne)
                self.T[(oi, oj)] = self._table(da, db, self.es_kind[None, :])
        # per-cell projection P_c (with w m omega folded in) and evaluation Phi_c
        self.P, self.Phi = {}, {}
        for c, mem in enumerate(self.cells.members):
            if len(mem) == 0:
                continue
            ci, cj = c % L, c // L
            rx = dz.x[mem, 0] - (self.cells.x0 + ci * H)
            ry = dz.x[mem, 1] - (self.cells.y0 + cj * H)
            Gc = mono_kernel(k, self.coll[:, 0][:, None] - rx[None, :],
                             self.coll[:, 1][:, None] - ry[None, :])       # (ncoll, n_c)
            self.P[c] = _lstsq_apply(self.Asvd, Gc) * dz.wfac[mem][None, :]
            self.Phi[c] = self._local_basis(rx - H / 2, ry - H / 2)
        # lattice FFT plan
        self.n_lat = L * Ne + 1
        self.M = _fft_size(2 * self.n_lat - 1)
        off = np.arange(self.M)
        off = np.where(off < self.M - self.n_lat + 1, off, off - self.M)   # signed offsets
        DA, DB = np.meshgrid(off, off, indexing="ij")
        self.Ghat = np.fft.fft2(self._table(DA, DB, 0))
        self.Dhat = np.fft.fft2(self._table(DA, DB, 1))

    # ------------------------------------------------------------------ pieces
    def _collocation(self, n):
        """n points on the boundary of the 3H x 3H square centred on the cell."""
        H = self.H
        m = n // 4
        t = (np.arange(m) + 0.5) / m * 3 * H - H          # from -H to 2H
        lo, hi = -H, 2 * H
        bottom = np.stack([t, np.full(m, lo)], -1)
        right = np.stack([np.full(m, hi), t], -1)
        top = np.stack([t[::-1], np.full(m, hi)], -1)
        left = np.stack([np.full(m, lo), t[::-1]], -1)
        return np.concatenate([bottom, right, top, left])

    def _es_field(self, px, py):
        """Field matrix of the cell's equivalent sources at points (px, py) (corner frame)."""
        zx = self.es_a * self.delta
        zy = self.es_b * self.delta
        dx = px[:, None] - zx[None, :]
        dy = py[:, None] - zy[None, :]
        mono = mono_kernel(self.kappa, dx, dy)
        dip = dip_kernel(self.kappa, dx, dy)
        return np.where(self.es_kind[None, :] == 0, mono, dip)

    def _table(self, da, db, kind):
        """Lattice kernel tables: G or dG/dz_1 at lattice offsets, zero at the origin."""
        da = np.asarray(da, float)
        db = np.asarray(db, float)
        zero = (da == 0) & (db == 0)
        dax = np.where(zero, 1.0, da) * self.delta
        dbx = np.where(zero, 0.0, db) * self.delta
        mono = mono_kernel(self.kappa, dax, dbx)
        dip = dip_kernel(self.kappa, dax, dbx)
        val = np.where(np.asarray(kind) == 0, mono, dip)
        return np.where(zero, 0.0, val)

    def _local_basis(self, x, y):
        return self._fb_basis(x, y) if self.local_basis == "fb" else self._pw_basis(x, y)

    def _pw_basis(self, x, y):
        """The paper's literal form of Eq. PWE: plane waves exp(i kappa d_l . x) in
        2 n_fb + 1 equally spaced directions d_l (comparison variant)."""
        m = 2 * self.nfb + 1
        th = 2 * math.pi * np.arange(m) / m
        return np.exp(1j * self.kappa * (x[:, None] * np.cos(th)[None, :] + y[:, None] * np.sin(th)[None, :]))

    def _fb_basis(self, x, y):
        n = np.arange(-self.nfb, self.nfb + 1)
        r = np.hypot(x, y)
        th = np.arctan2(y, x)
        kr = self.kappa * r
        return (jv(n[None, :], kr[:, None]) / jv(np.abs(n), self.kappa * self.Rref)[None, :]
                * np.exp(1j * n[None, :] * th[:, None]))

    # ------------------------------------------------------------------ apply
    def project(self, u):
        """sigma_c = P_c (w m omega u)_c for every occupied cell: dict c -> (n_es,)."""
        return {c: P @ u[self.cells.members[c]] for c, P in self.P.items()}

    def lattice_sources(self, sig):
        Sm = np.zeros((self.M, self.M), np.complex128)
        Sd = np.zeros((self.M, self.M), np.complex128)
        Ne, L = self.Ne, self.L
        for c, s in sig.items():
            ci, cj = c % L, c // L
            a = ci * Ne + self.es_a
            b = cj * Ne + self.es_b
            mono = self.es_kind == 0
            np.add.at(Sm, (a[mono], b[mono]), s[mono])
            np.add.at(Sd, (a[~mono], b[~mono]), s[~mono])
        return Sm, Sd

    def lattice_field(self, Sm, Sd):
        V = np.fft.ifft2(np.fft.fft2(Sm) * self.Ghat + np.fft.fft2(Sd) * self.Dhat)
        return V[:self.n_lat, :self.n_lat]

    def local_data(self, V, sig):
        """beta_c: non-adjacent field on the closed cell's lattice points."""
        Ne, L = self.Ne, self.L
        out = {}
        for c in self.P:
            ci, cj = c % L, c // L
            beta = V[ci * Ne + self.loc_a, cj * Ne + self.loc_b].copy()
            for (oi, oj), T in self.T.items():
                nb = (cj + oj) * L + (ci + oi)
                if 0 <= ci + oi < L and 0 <= cj + oj < L and nb in sig:
                    beta -= T @ sig[nb]
            out[c] = beta
        return out

    def evaluate(self, beta, N):
        v = np.zeros(N, np.complex128)
        for c, b in beta.items():
            v[self.cells.members[c]] = self.Phi[c] @ (self.Bpinv @ b)
        return v

    def apply_far(self, u):
        sig = self.project(np.asarray(u, np.complex128))
        V = self.lattice_field(*self.lattice_sources(sig))
        return self.evaluate(self.local_data(V, sig), self.dz.N)

    def direct_far(self, u, rows=None):
        """Exact non-adjacent sum (Eq. disctete-conv) for comparison."""
        dz = self.dz
        if rows is None:
            rows = np.arange(dz.N)
        out = np.zeros(len(rows), np.complex128)
        for s in range(0, len(rows), 512):
            r = rows[s:s + 512]
            far = ~self.cells.near_mask(r)
            dx = dz.x[None, :, 0] - dz.x[r, None, 0]
            dy = dz.x[None, :, 1] - dz.x[r, None, 1]
            G = np.where(far, mono_kernel(self.kappa, np.where(far, dx, 1.0), dy), 0.0)
            out[s:s + 512] = G @ (dz.wfac * u)
        return out


def _svd(A):
    """Thin SVD truncated at RCOND relative to the largest singular value."""
    U, s, Vh = np.linalg.svd(A, full_matrices=False)
    k = int(np.sum(s > RCOND * s[0]))
    return U[:, :k], s[:k], Vh[:k]


def _lstsq_apply(svd, Bm):
    """Least-squares solution X of A X = Bm from the factors, applied factor by
    factor (V (S^-1 (U^H Bm))) so that the rounding stays relative to the data;
    forming the pseudo-inverse explicitly would cost cond(A) digits."""
    U, s, Vh = svd
    return Vh.conj().T @ ((U.conj().T @ Bm) / s[:, None])


def _fft_size(n: int) -> int:
    """Smallest 2^a 3^b 5^c >= n."""
    best = None
    p2 = 1
    while p2 < 2 * n:
        p3 = p2
        while p3 < 2 * n:
            p5 = p3
            while p5 < 2 * n:
                if p5 >= n and (best is None or p5 < best):
                    best = p5
                p5 *= 5
            p3 *= 3
        p2 *= 2
    return best


class AcceleratedOperator:
    """K u = (adjacent part) u + (equivalent-source far part) u; A = I + kappa^2 K."""

    def __init__(self, dz: Discretisation):
        self.dz = dz
        self.cells = Cells(dz)
        self.Wnear = near_matrix(dz, self.cells)
        self.acc = Accelerator(dz, self.cells)

    def apply_K(self, u):
        u = np.asarray(u, np.complex128)
        return self.Wnear @ u + self.acc.apply_far(u)

    def apply(self, u):
        return np.asarray(u, np.complex128) + self.dz.wl.kappa ** 2 * self.apply_K(u)
