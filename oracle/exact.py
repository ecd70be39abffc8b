"""Closed-form references used to pin the oracle (test infrastructure only).

* Penetrable disc, constant n: separation of variables (Bessel series) for the
  total field of a plane wave, with continuity of u and du/dr at r = a, the
  transmission conditions that follow from the Helmholtz problem (Eq. HE) and
  u in C^1 across the interface.
* Volume potential of the constant density over a disc:
  K[1](x) = -1/kappa^2 + (i pi a / (2 kappa)) H_1(kappa a) J_0(kappa |x|), |x| < a.
* Far-field pattern of the disc from the same series.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import h1vp, hankel1, jv, jvp


def disc_coeffs(kappa: float, n: float, a: float, mmax: int):
    m = np.arange(-mmax, mmax + 1)
    ka, nka = kappa * a, n * kappa * a
    J, Jp = jv(m, ka), jvp(m, ka)
    Jn, Jnp = jv(m, nka), jvp(m, nka)
    Hk, Hkp = hankel1(m, ka), h1vp(m, ka)
    b = (n * Jnp * J - Jp * Jn) / (Jn * Hkp - n * Jnp * Hk)
    am = (J + b * Hk) / Jn
    return m, am, b


def disc_total_field(kappa, n2, a, x, d=(1.0, 0.0), center=(0.0, 0.0), mmax=None):
    """Total field u for a plane wave exp(i kappa d.x) on a disc of radius a with
    constant n^2 inside."""
    n = math.sqrt(n2)
    if mmax is None:
        mmax = int(n * kappa * a + 40)
    m, am, b = disc_coeffs(kappa, n, a, mmax)
    x = np.asarray(x, np.float64)
    dx, dy = x[..., 0] - center[0], x[..., 1] - center[1]
    r = np.hypot(dx, dy)
    th = np.arctan2(dy, dx)
    thd = math.atan2(d[1], d[0])
    ph = np.exp(1j * np.outer(th - thd, m)) * (1j ** m)
    inside = r < a
    u = np.zeros(r.shape, np.complex128)
    rr = r[inside][:, None]
    u[inside] = np.sum(ph[inside] * am * jv(m, n * kappa * rr), -1)
    ro = r[~inside][:, None]
    u[~inside] = np.sum(ph[~inside] * (jv(m, kappa * ro) + b * hankel1(m, kappa * ro)), -1)
    # plane-wave phase relative to the disc centre
    u *= np.exp(1j * kappa * (center[0] * d[0] + center[1] * d[1]))
    return u


def disc_far_field(kappa, n2, a, theta, d=(1.0, 0.0), mmax=None):
    """Far-field pattern A(theta) with u^s ~ exp(i kappa r)/sqrt(r) A."""
    n = math.sqrt(n2)
    if mmax is None:
        mmax = int(n * kappa * a + 40)
    m, _, b = disc_coeffs(kappa, n, a, mmax)
    thd = math.atan2(d[1], d[0])
    th = np.asarray(theta, np.float64)
    # H_m(kr) ~ sqrt(2/(pi k r)) exp(i(kr - m pi/2 - pi/4))
    ph = np.exp(1j * np.outer(th - thd, m)) * (1j ** m) * np.exp(-1j * m * math.pi / 2)
    return math.sqrt(2.0 / (math.pi * kappa)) * np.exp(-1j * math.pi / 4) * np.sum(ph * b, -1)


def disc_volume_potential_const(kappa, a, x):
    """K[1](x) for |x| < a: integral over the disc of G(x, y) dy."""
    r = np.hypot(x[..., 0], x[..., 1])
    return -1.0 / kappa ** 2 + (1j * math.pi * a / (2 * kappa)) * hankel1(1, kappa * a) * jv(0, kappa * r)
