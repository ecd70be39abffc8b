"""Far-field pattern of the computed total field (test infrastructure only).

Not in the paper (it reports near-field errors only).  From the Lippmann-Schwinger
equation (Eq. Lippmann), u^s = kappa^2 int G (n^2 - 1) u dy, and the large-argument
form of H_0^(1), u^s(x) ~ exp(i kappa |x|) / sqrt(|x|) A(x_hat) with

  A(x_hat) = exp(i pi / 4) / sqrt(8 pi kappa) kappa^2 int exp(-i kappa x_hat . y) (n^2 - 1) u dy,

evaluated with the same node weights w omega of the Nystrom rule.
"""
from __future__ import annotations

import math

import numpy as np


def far_field(dz, u: np.ndarray, theta: np.ndarray) -> np.ndarray:
    wl = dz.wl
    k = wl.kappa
    c2 = np.exp(1j * math.pi / 4) / math.sqrt(8 * math.pi * k)
    xh = np.stack([np.cos(theta), np.sin(theta)], -1)
    ph = np.exp(-1j * k * (xh @ dz.x.T))             # (ndir, N)
    wq = dz.w * dz.omega * (dz.n2 - 1.0)
    return c2 * k * k * (ph @ (wq * np.asarray(u)).T).T
