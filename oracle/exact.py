"""Closed-form references used to pin the oracle (test infrastructure only).

* Penetrable disc, constant n: separation of variables (Bessel series) for the
  total field of a plane wave, with continuity of u and du/dr at r = a, the
  transmission conditions that follow from the Helmholtz problem (Eq. HE) and
  u in C^1 across the interface.
* Volume potential of the constant density over a disc:
  K[1](x) = -1/kappa^2 + (i pi a / (2 kappa)) H_1(kappa a) J_0(kappa |x|), |x| < a.
* Far-field pattern of the disc from the same series.
* Three dimensions (Section 5, the extension to 3-D), for the 3-D path to come:
  penetrable sphere of radius a, constant n, plane wave exp(i kappa z):
  separation of variables in spherical Bessel functions and Legendre
  polynomials with the same transmission conditions; its far-field pattern
  f(theta), u^s ~ f exp(i kappa r) / r; and the volume potential of the
  constant density over a ball with G = exp(i kappa |x - y|) / (4 pi |x - y|):
  -1/kappa^2 + (1 - i kappa a) exp(i kappa a) j_0(kappa |x|) / kappa^2 inside,
  (the solution of (Laplacian + kappa^2) v = -1 in the ball, smooth across
  r = a and outgoing outside).
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import eval_legendre, h1vp, hankel1, jv, jvp, spherical_jn, spherical_yn


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


# ---------------------------------------------------------------- three dimensions
def sphere_coeffs(kappa: float, n: float, a: float, lmax: int):
    """Coefficients of the penetrable sphere: inside c_l j_l(n kappa r), outside
    j_l(kappa r) + b_l h_l(kappa r), each times i^l (2l+1) P_l(cos theta)."""
    l = np.arange(lmax + 1)
    ka, nka = kappa * a, n * kappa * a
    j, jp = spherical_jn(l, ka), spherical_jn(l, ka, derivative=True)
    jn_, jnp = spherical_jn(l, nka), spherical_jn(l, nka, derivative=True)
    h = j + 1j * spherical_yn(l, ka)
    hp = jp + 1j * spherical_yn(l, ka, derivative=True)
    b = (n * jnp * j - jp * jn_) / (jn_ * hp - n * jnp * h)
    c = (j + b * h) / jn_
    return l, c, b


def sphere_total_field(kappa, n2, a, x, lmax=None):
    """Total field u for the plane wave exp(i kappa z) on a sphere of radius a
    (centred at the origin) with constant n^2 inside; x: (..., 3)."""
    n = math.sqrt(n2)
    if lmax is None:
        lmax = int(n * kappa * a + 30)
    l, c, b = sphere_coeffs(kappa, n, a, lmax)
    x = np.asarray(x, np.float64)
    r = np.linalg.norm(x, axis=-1)
    ct = np.where(r > 0, x[..., 2] / np.where(r > 0, r, 1.0), 1.0)
    P = eval_legendre(l, ct[..., None])                          # (..., lmax+1)
    w = (1j ** l) * (2 * l + 1) * P
    inside = r < a
    u = np.zeros(r.shape, np.complex128)
    ri = r[inside][:, None]
    u[inside] = np.sum(w[inside] * c * spherical_jn(l, n * kappa * ri), -1)
    ro = r[~inside][:, None]
    ho = spherical_jn(l, kappa * ro) + 1j * spherical_yn(l, kappa * ro)
    u[~inside] = np.sum(w[~inside] * (spherical_jn(l, kappa * ro) + b * ho), -1)
    return u


def sphere_far_field(kappa, n2, a, theta, lmax=None):
    """f(theta) with u^s ~ f exp(i kappa r) / r (theta from the incidence
    direction): h_l(z) ~ (-i)^(l+1) exp(i z) / z gives
    f = (-i / kappa) sum (2l+1) b_l P_l(cos theta)."""
    n = math.sqrt(n2)
    if lmax is None:
        lmax = int(n * kappa * a + 30)
    l, _, b = sphere_coeffs(kappa, n, a, lmax)
    P = eval_legendre(l, np.cos(np.asarray(theta, np.float64))[..., None])
    return (-1j / kappa) * np.sum((2 * l + 1) * b * P, -1)


def ball_volume_potential_const(kappa, a, x):
    """Integral over the ball |y| < a of exp(i kappa |x - y|) / (4 pi |x - y|) dy
    at x (..., 3): -1/kappa^2 + A j_0(kappa r) inside, B h_0(kappa r) outside,
    A = (1 - i kappa a) exp(i kappa a) / kappa^2, B from continuity at r = a."""
    x = np.asarray(x, np.float64)
    r = np.linalg.norm(x, axis=-1)
    ka = kappa * a
    A = (1.0 - 1j * ka) * np.exp(1j * ka) / kappa ** 2
    h0a = np.exp(1j * ka) / (1j * ka)
    B = (-1.0 / kappa ** 2 + A * math.sin(ka) / ka) / h0a
    kr = kappa * np.where(r > 0, r, 1.0)
    inner = -1.0 / kappa ** 2 + A * np.where(r > 0, np.sin(kr) / kr, 1.0)
    outer = B * np.exp(1j * kr) / (1j * kr)
    return np.where(r < a, inner, outer)
