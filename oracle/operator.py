"""Direct O(N^2) Nystrom operator (test infrastructure only).

(A u)_q = u_q + kappa^2 K[u](x_q) with (Eq. Lippmann, Eq. VolInt-B-II and
Eq. VolInt-Adj-NonAdj-I, far part summed exactly as in Eq. disctete-conv)

  K[u](x_q) = sum_l w_l m_l omega_l G(x_q, y_l) (1 - eta_{k(l)}(y_l; x_q)) u_l
            + sum_k K_k^sing[u](x_q)

where eta_k(.; x_q) is the cut-off of the patch k carrying node l (zero when
patch k needs no singular treatment at x_q) and K_k^sing is the singular rule of
quadrature.py.  The cell decomposition of the accelerator does not enter here.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import quadrature as qd
from .geometry import Discretisation


def regular_rows(dz: Discretisation, rows) -> np.ndarray:
    """Dense rows K_reg[q, :] = w m omega G(x_q, y) (1 - eta) for q in rows."""
    wl = dz.wl
    rows = np.asarray(rows)
    one_m_eta = 1.0 - qd.eta_regular(dz, rows)
    r = np.hypot(dz.x[None, :, 0] - dz.x[rows, None, 0], dz.x[None, :, 1] - dz.x[rows, None, 1])
    nz = one_m_eta != 0.0
    out = np.zeros((len(rows), dz.N), np.complex128)
    out[nz] = 0.25j * qd.hankel0(wl.kappa * r[nz]) * (dz.wfac[None, :] * one_m_eta)[nz]
    return out


def singular_matrix(dz: Discretisation, rows=None, chunk: int = 512) -> sp.csr_matrix:
    """Sparse matrix of all singular-rule coefficients for the given target rows."""
    if rows is None:
        rows = np.arange(dz.N)
    rows = np.asarray(rows)
    parts = []
    for s in range(0, len(rows), chunk):
        ri, ci, vv = qd.singular_triplets(dz, rows[s:s + chunk])
        parts.append(sp.coo_matrix((vv, (ri + s, ci)), shape=(len(rows), dz.N)).tocsr())
    m = parts[0]
    for p in parts[1:]:
        m = m + p
    m.sum_duplicates()
    return m


class DirectOperator:
    """The discrete operator K (and A = I + kappa^2 K) assembled row by row."""

    def __init__(self, dz: Discretisation, dense_limit: int = 6000):
        self.dz = dz
        self.kappa = dz.wl.kappa
        self._K = None
        if dz.N <= dense_limit:
            K = np.zeros((dz.N, dz.N), np.complex128)
            for s in range(0, dz.N, 512):
                K[s:s + 512] = regular_rows(dz, np.arange(s, min(s + 512, dz.N)))
            K += singular_matrix(dz).toarray()
            self._K = K

    def K_rows(self, rows) -> np.ndarray:
        if self._K is not None:
            return self._K[np.asarray(rows)]
        return regular_rows(self.dz, rows) + singular_matrix(self.dz, rows).toarray()

    def dense_K(self) -> np.ndarray:
        if self._K is None:
            raise ValueError("operator too large for dense assembly")
        return self._K

    def dense_A(self) -> np.ndarray:
        return np.eye(self.dz.N) + self.kappa ** 2 * self.dense_K()

    def apply_K(self, u: np.ndarray, rows=None, chunk: int = 256) -> np.ndarray:
        """K u on all rows (or the given rows); u is (N,) or (nrhs, N)."""
        u = np.asarray(u, np.complex128)
        if rows is None:
            rows = np.arange(self.dz.N)
        rows = np.asarray(rows)
        if self._K is not None:
            return (self._K[rows] @ u.T).T
        out = np.zeros(u.shape[:-1] + (len(rows),), np.complex128)
        for s in range(0, len(rows), chunk):
            r = rows[s:s + chunk]
            out[..., s:s + chunk] = (self.K_rows(r) @ u.T).T
        return out

    def apply(self, u: np.ndarray, rows=None) -> np.ndarray:
        """(A u)[rows] = u[rows] + kappa^2 (K u)[rows]."""
        u = np.asarray(u, np.complex128)
        if rows is None:
            rows = np.arange(self.dz.N)
        return u[..., rows] + self.kappa ** 2 * self.apply_K(u, rows)
