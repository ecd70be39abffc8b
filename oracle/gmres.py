"""Restarted GMRES in complex FP64 (test infrastructure only).

The paper solves the Nystrom system with matrix-free GMRES in fully complex
arithmetic (Section 2, Saad-Schultz 1986); restart length, initial guess and
stopping rule are not stated.  Reading: GMRES(m) with modified Gram-Schmidt and
one re-orthogonalisation pass, Givens rotations, x0 = 0 unless given, stop when
||b - A x||_2 / ||b||_2 <= tol (true residual checked at every restart).
"""
from __future__ import annotations

import numpy as np


def gmres(apply, b: np.ndarray, tol: float = 1e-10, restart: int = 100, max_iter: int = 1000,
          x0: np.ndarray | None = None):
    b = np.asarray(b, np.complex128)
    n = b.shape[0]
    x = np.zeros(n, np.complex128) if x0 is None else np.array(x0, np.complex128)
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return x, 0, [0.0]
    hist = []
    it = 0
    while True:
        r = b - apply(x)
        beta = np.linalg.norm(r)
        hist.append(beta / bnorm)
        if beta / bnorm <= tol or it >= max_iter:
            return x, it, hist
        m = restart
        V = np.zeros((m + 1, n), np.complex128)
        H = np.zeros((m + 1, m), np.complex128)
        cs = np.zeros(m, np.complex128)
        sn = np.zeros(m, np.complex128)
        g = np.zeros(m + 1, np.complex128)
        g[0] = beta
        V[0] = r / beta
        k_used = 0
        for k in range(m):
            w = apply(V[k])
            for _ in range(2):
                for j in range(k + 1):
                    hjk = np.vdot(V[j], w)
                    H[j, k] += hjk
                    w = w - hjk * V[j]
            H[k + 1, k] = np.linalg.norm(w)
            if H[k + 1, k] != 0:
                V[k + 1] = w / H[k + 1, k]
            for j in range(k):
                t = np.conj(cs[j]) * H[j, k] + np.conj(sn[j]) * H[j + 1, k]
                H[j + 1, k] = -sn[j] * H[j, k] + cs[j] * H[j + 1, k]
                H[j, k] = t
            # unitary rotation [[conj c, conj s], [-s, c]] with c = a/den, s = b/den
            a, bb = H[k, k], H[k + 1, k]
            den = np.sqrt(abs(a) ** 2 + abs(bb) ** 2)
            cs[k] = a / den if den else 1.0
            sn[k] = bb / den if den else 0.0
            H[k, k] = den
            H[k + 1, k] = 0.0
            g[k + 1] = -sn[k] * g[k]
            g[k] = np.conj(cs[k]) * g[k]
            it += 1
            k_used = k + 1
            if abs(g[k + 1]) / bnorm <= tol or it >= max_iter:
                break
        y = np.linalg.solve(np.triu(H[:k_used, :k_used]), g[:k_used])
        x = x + V[:k_used].T @ y
