"""Seeded synthetic workloads for the Lippmann-Schwinger solver (2-D).

This module only *describes* inputs: the scatterer family and its parameters,
the refractive-index profile n^2(x), the incident plane wave, the wavenumber,
the resolution / quadrature parameters of the Nystrom discretisation and the
seeded random densities used for apply-throughput runs.  It holds none of the
method's arithmetic (no charts, weights, quadratures, Green's functions or
acceleration), so both the CPU oracle and the CUDA library consume it without
sharing any of the method with each other.

The shapes mirror the paper's experiments (disc, Section 3.3 Example 1 / the
timing table; the kite stands in for the paper's "bean", whose parametrisation
is not given).  All randomness comes from numpy's PCG64 seeded with 150905063.
"""
from __future__ import annotations

import dataclasses
import math
from dataclasses import dataclass, field

import numpy as np

SEED = 150905063

SHAPES = {"disc": 0, "kite": 1, "star": 2}
N2_KINDS = {"const": 0, "gauss": 1, "sincos": 2}


@dataclass
class Workload:
    """All parameters that define one discrete LS operator (2-D).

    Geometry: boundary curve gamma(s), s in [0, 2pi).
      disc : shape_params = (a, cx, cy)      gamma = c + a(cos s, sin s)
      kite : shape_params = (scale, cx, cy)  gamma = c + scale(cos s + 0.65 cos 2s - 0.65, 1.5 sin s)
      star : shape_params = (a0, cx, cy, c1, ..., c5)  gamma = c + r(s)(cos s, sin s),
             r(s) = a0 + sum_k c_k cos(k s)
    Collar (boundary) chart: X(a, b) = gamma(2 pi a / n1) - (b / (n2 - 1)) * collar_w * nu,
      a in [0, n1) periodic, b in [0, n2 - 1]; b = 0 lies on the boundary.
    Interior chart: Cartesian grid x = cart_x0 + i h, y = cart_y0 + j h,
      0 <= i < cart_nx, 0 <= j < cart_ny; only points with omega_I > 0 are nodes.
    Partition of unity: omega_B = S((t - tau0) / (tau1 - tau0)) on the collar,
      omega_I = 1 - omega_B.
    Quadrature: Q-point composite Newton-Cotes across the collar, Lagrange
      interpolation of degree p, cut-off radii in grid-index units (R_a along
      and R_b across the collar, R_cart on the Cartesian patch), rho(tau) = R tau^(M+1) with N_tau trapezoid points for the boundary
      singular rule, polar rule with n_rho x n_theta points and rho = R s^q_polar.
    Acceleration: square box [box_x0, box_x0 + L H] x [box_y0, box_y0 + L H],
      L x L cells of side H, lattice spacing H / N_eq, Fourier-Bessel order n_fb,
      n_coll collocation points on the 3H x 3H square around a cell.
    """

    name: str
    shape: str
    shape_params: tuple
    kappa: float
    n2_kind: str
    n2_params: tuple
    inc_dir: tuple = (1.0, 0.0)
    collar_w: float = 0.4
    n1: int = 64
    n2: int = 9
    tau0: float = 0.35
    tau1: float = 0.8
    h: float = 0.1
    cart_x0: float = -1.0
    cart_y0: float = -1.0
    cart_nx: int = 21
    cart_ny: int = 21
    Q: int = 5
    p: int = 9
    R_a: float = 8.0
    R_b: float = 4.0
    R_cart: float = 6.0
    M: int = 4
    N_tau: int = 48
    q_polar: int = 3
    n_rho: int = 24
    n_theta: int = 32
    chi_s0: float = 0.1
    # acceleration (ignored by the direct operator)
    box_x0: float = -1.2
    box_y0: float = -1.2
    H: float = 0.3
    L: int = 8
    N_eq: int = 8
    n_fb: int = 15
    n_coll: int = 0  # 0 -> 4 * (4 (N_eq + 1))
    dim: int = 2

    def replace(self, **kw) -> "Workload":
        return dataclasses.replace(self, **kw)

    @property
    def n_collar(self) -> int:
        return self.n1 * self.n2


def n2_eval(kind: str, params: tuple, x: np.ndarray) -> np.ndarray:
    """Refractive index squared n^2 at points x (..., 2).  Input definition only."""
    x = np.asarray(x, dtype=np.float64)
    if kind == "const":
        return np.full(x.shape[:-1], float(params[0]))
    if kind == "gauss":  # n^2 = a + b exp(-|x - c|^2 / s)
        a, b, s, cx, cy = params
        r2 = (x[..., 0] - cx) ** 2 + (x[..., 1] - cy) ** 2
        return a + b * np.exp(-r2 / s)
    if kind == "sincos":  # n^2 = a + b sin(pi x1) cos(pi x2)
        a, b = params[:2]
        return a + b * np.sin(np.pi * x[..., 0]) * np.cos(np.pi * x[..., 1])
    raise ValueError(kind)


def plane_wave(kappa: float, d, x: np.ndarray) -> np.ndarray:
    """Incident field exp(i kappa d . x) at points x (..., 2)."""
    d = np.asarray(d, dtype=np.float64)
    d = d / np.linalg.norm(d)
    return np.exp(1j * kappa * (x[..., 0] * d[0] + x[..., 1] * d[1]))


def random_density(n: int, nrhs: int = 1, seed: int = SEED) -> np.ndarray:
    """u ~ CN(0, 1), shape (nrhs, n), complex128, seeded."""
    rng = np.random.default_rng(seed)
    re = rng.standard_normal((nrhs, n))
    im = rng.standard_normal((nrhs, n))
    return ((re + 1j * im) / math.sqrt(2.0)).astype(np.complex128)


def random_rows(n: int, k: int, seed: int = SEED + 1) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(n, size=min(k, n), replace=False))


# --------------------------------------------------------------------------
# Named workloads.  Resolutions follow the paper's grid families
# (boundary patch n1 x n2 plus an interior Cartesian patch).
# --------------------------------------------------------------------------

def place_cells(wl: Workload, L: int, m: int, center=(0.0, 0.0), N_eq: int | None = None) -> Workload:
    """Accelerator cells of side H = m h whose faces fall half a Cartesian
    spacing off the grid lines, so that no Nystrom node lies on a cell face and
    the cell of every node is decided the same way in any rounding."""
    H = m * wl.h
    A = L * H
    kx = round((center[0] - A / 2 - wl.cart_x0) / wl.h)
    ky = round((center[1] - A / 2 - wl.cart_y0) / wl.h)
    kw = dict(box_x0=wl.cart_x0 + (kx + 0.5) * wl.h, box_y0=wl.cart_y0 + (ky + 0.5) * wl.h, H=H, L=L)
    if N_eq is not None:
        kw.update(N_eq=N_eq, n_fb=2 * N_eq - 1)
    return wl.replace(**kw)


def _cart_grid_for(h: float, lo: float, hi: float, anchor: float = 0.0):
    """Cartesian grid covering [lo, hi] with points anchor + i h."""
    i0 = math.floor((lo - anchor) / h) - 1
    i1 = math.ceil((hi - anchor) / h) + 1
    return anchor + i0 * h, i1 - i0 + 1


def disc(level: int = 1, kappa: float = 2.0, n2c: float = 2.0, a: float = 1.0,
         Q: int = 5, accel: dict | None = None, **kw) -> Workload:
    """Penetrable disc of radius a, constant n^2 inside, plane wave along x1.

    level l: collar n1 = 32 * 2^l tangential, n2 = (Q-1) 2^l + 1 transverse,
    Cartesian spacing matched to the collar's tangential spacing at radius a/2.
    """
    n1 = 32 * 2 ** level
    n2 = (Q - 1) * 2 ** (level) + 1
    w = kw.pop("collar_w", 0.45 * a)
    h = kw.pop("h", 2 * math.pi * a / n1 * 1.0)
    x0, nx = _cart_grid_for(h, -a, a)
    wl = Workload(name=f"disc_l{level}", shape="disc", shape_params=(a, 0.0, 0.0),
                  kappa=kappa, n2_kind="const", n2_params=(n2c,), collar_w=w,
                  n1=n1, n2=n2, h=h, cart_x0=x0, cart_y0=x0, cart_nx=nx, cart_ny=nx,
                  Q=Q, **kw)
    if accel:
        wl = wl.replace(**accel)
    return wl


def star(level: int = 1, kappa: float = 2.0, n2c: float = 2.0, a0: float = 1.0, coeffs=(0.0, 0.0, 0.0, 0.0, 0.1),
         Q: int = 5, **kw) -> Workload:
    """Penetrable Fourier star r(s) = a0 + sum_k c_k cos(k s) (default a five-pointed
    star, c_5 = 0.1), constant n^2 inside, grids as for the disc of the same level."""
    n1 = 32 * 2 ** level
    n2 = (Q - 1) * 2 ** level + 1
    w = kw.pop("collar_w", 0.2 * a0)
    h = kw.pop("h", 2 * math.pi * a0 / n1)
    rmax = a0 + sum(abs(c) for c in coeffs)
    x0, nx = _cart_grid_for(h, -rmax, rmax)
    wl = Workload(name=f"star_l{level}", shape="star", shape_params=(a0, 0.0, 0.0, *coeffs),
                  kappa=kappa, n2_kind="const", n2_params=(n2c,), collar_w=w,
                  n1=n1, n2=n2, h=h, cart_x0=x0, cart_y0=x0, cart_nx=nx, cart_ny=nx, Q=Q, **kw)
    return wl


def kite(n1: int, n2: int, h: float, kappa: float, scale: float = 1.0, collar_w: float = 0.07,
         n2_kind: str = "gauss", n2_params: tuple | None = None, **kw) -> Workload:
    if n2_params is None:
        n2_params = (1.5, 0.5, 0.1 * scale * scale, 0.0, 0.0)
    lo_x, hi_x = -1.5 * scale, 1.0 * scale
    lo_y, hi_y = -1.5 * scale, 1.5 * scale
    x0, nx = _cart_grid_for(h, lo_x, hi_x)
    y0, ny = _cart_grid_for(h, lo_y, hi_y)
    return Workload(name=f"kite_{n1}x{n2}", shape="kite", shape_params=(scale, 0.0, 0.0),
                    kappa=kappa, n2_kind=n2_kind, n2_params=n2_params, collar_w=collar_w,
                    n1=n1, n2=n2, h=h, cart_x0=x0, cart_y0=y0, cart_nx=nx, cart_ny=ny, **kw)


def cfg1() -> Workload:
    """Disc a = 1, n^2 = 2 inside, kappa = 2, plane wave along x1; ~4k nodes
    (collar 128 tangential x 17 transverse, Cartesian h = 0.03); complex128;
    checked against the Bessel series."""
    h = 0.03
    x0, nx = _cart_grid_for(h, -1.0, 1.0)
    return place_cells(
        Workload(name="cfg1_disc_kappa2", shape="disc", shape_params=(1.0, 0.0, 0.0), kappa=2.0,
                 n2_kind="const", n2_params=(2.0,), collar_w=0.48, n1=128, n2=17, tau0=0.35, tau1=0.9,
                 h=h, cart_x0=x0, cart_y0=x0, cart_nx=nx, cart_ny=nx, R_a=5, R_b=5, R_cart=6,
                 N_eq=8, n_fb=15), L=8, m=10)


def cfg2(h: float = 0.0045, n1: int = 3200, L: int = 61, m: int = 11, N_eq: int = 8) -> Workload:
    """Kite x = cos t + 0.65 cos 2t - 0.65, y = 1.5 sin t; n^2 = 1.5 + 0.5 exp(-|x|^2/0.1)
    inside, 1 outside; kappa = 20, ~274k nodes, 1024^2 padded lattice FFT, GMRES tol 1e-10.
    Cells of 11 h (L = 61): the layout the library's autotuner picks for this
    scatterer (smallest admissible cells)."""
    wl = kite(n1=n1, n2=17, h=h, kappa=20.0, collar_w=0.07, tau0=0.4, tau1=0.9,
              R_a=10, R_b=6, R_cart=8)
    return place_cells(wl.replace(name="cfg2_kite_kappa20"), L=L, m=m, center=(-0.25, 0.0), N_eq=N_eq)


def n2_of(wl: Workload):
    """Callable x -> n^2(x) for the workload (input definition)."""
    return lambda x: n2_eval(wl.n2_kind, wl.n2_params, x)


def scatterer(shape: str, scale: float, kappa: float, N_target: float, ppw_min: float = 24.0) -> Workload:
    """A disc (radius `scale`, n^2 = 2) or kite (scaled by `scale`, n^2 = 1.5 +
    0.5 exp(-|x/scale|^2 / 0.1)) with about N_target nodes: Cartesian spacing h
    from the interior area, a 17-line collar of width 16 h (at most 0.07 scale
    for the kite, below its smallest radius of curvature), tangential spacing
    0.6 h, the cut-off radii of the kite workload in grid units; h is refined
    to at least ppw_min points per wavelength.  The cell layout is left to the
    library (L = 0, H = 11 h as a starting point)."""
    if shape == "disc":
        area, perim = math.pi * scale ** 2, 2 * math.pi * scale
    else:
        area, perim = 4.45 * scale ** 2, 8.5 * scale
    # N ~ area / h^2 + 17 perim / (0.6 h): positive root of the quadratic in 1/h
    b = 17 * perim / 0.6
    inv_h = (-b + math.sqrt(b * b + 4 * area * N_target)) / (2 * area)
    h = min(1.0 / inv_h, 2 * math.pi / (kappa * ppw_min))
    n1 = max(64, int(round(perim / (0.6 * h) / 8)) * 8)
    if shape == "disc":
        x0, nx = _cart_grid_for(h, -scale, scale)
        wl = Workload(name=f"disc_s{scale:.2f}_k{kappa:.1f}", shape="disc", shape_params=(scale, 0.0, 0.0),
                      kappa=kappa, n2_kind="const", n2_params=(2.0,), collar_w=16 * h, n1=n1, n2=17,
                      tau0=0.4, tau1=0.9, h=h, cart_x0=x0, cart_y0=x0, cart_nx=nx, cart_ny=nx,
                      R_a=10, R_b=6, R_cart=8)
        center = (0.0, 0.0)
    else:
        w = min(16 * h, 0.07 * scale)        # below the kite's radius of curvature (0.085 scale)
        wl = kite(n1=n1, n2=17, h=h, kappa=kappa, scale=scale, collar_w=w, tau0=0.4, tau1=0.9,
                  R_a=10, R_b=6, R_cart=8).replace(name=f"kite_s{scale:.2f}_k{kappa:.1f}")
        center = (-0.25 * scale, 0.0)
    wl = place_cells(wl, L=1, m=11, center=center, N_eq=8)
    return wl.replace(L=0)


def cfg3_instances(n: int = 48, seed: int = SEED + 3, N_lo: float = 2e4, N_hi: float = 1e6,
                   scale_range=(0.5, 2.0), kappa_range=(5.0, 60.0)):
    """The seed-drawn scatterers of the batched configuration: shape disc or
    kite with probability 1/2, scale ~ U[scale_range], kappa ~ U[kappa_range],
    N log-uniform in [N_lo, N_hi] (raised where 24 points per wavelength need
    more), one plane wave along x1 each."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        shape = "disc" if rng.random() < 0.5 else "kite"
        scale = rng.uniform(*scale_range)
        kappa = rng.uniform(*kappa_range)
        N = math.exp(rng.uniform(math.log(N_lo), math.log(N_hi)))
        out.append(scatterer(shape, scale, kappa, N))
    return out
