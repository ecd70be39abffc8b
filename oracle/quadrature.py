"""Localised singular quadratures of Section 3.1 (test infrastructure only).

For a target x and a patch k the integral of G phi_k over the patch is split by
a cut-off eta (Eq. VolInt-B-III): the eta part is done by a singularity-resolving
rule, the (1 - eta) part by the regular rule on the patch grid.

* interior-type rule (Section 3.1.1, Eq. K-Int-Sing-Polar): circular
  eta = chi(|t - t_x| / r); polar coordinates about the target.  Reading: the
  radial variable is taken on [0, r] with rho = r s^q so that the rho log rho
  behaviour of the 2-D kernel becomes C^(2q-2) in s; trapezoid in s and theta.
  Used for every target on the Cartesian patch and for Cartesian targets on the
  collar chart (their cut-off disc stays clear of the boundary line b = 0).
* boundary rule (Section 3.1.2, Eqs. VolInt-Adj-Sing-1, I, POLYCOB, I-inTau,
  VolInt-Adj-Sing-MultiSplit): rectangular eta; the tangential integral J(t_2; x)
  uses t_1 = t_1^x + varrho(tau), varrho(tau) = r tau^(M+1), trapezoid in tau; the
  transverse integral is split at t_2^x into Q-point composite Newton-Cotes
  blocks, with single-spacing remainder intervals near the ends done by a Q-point
  rule on extra fractional lines.  Used for every collar node as target.
* off-grid values phi_k are obtained by tensor-product Lagrange interpolation of
  degree p on the patch grid (reading of the paper's "Fourier refined polynomial
  interpolation"; one-sided near the ends of the transverse direction,
  periodic along the collar).  A comparison variant takes the paper's words
  literally (Discretisation(..., interp=(F, pf))): the samples are first refined
  F-fold by band-limited (FFT) interpolation, then Lagrange of degree pf on the
  refined grid; along the collar (periodic) and along both axes of the
  Cartesian patch (whose density vanishes near the edges of its grid), while
  the transverse collar direction keeps degree-p Lagrange.

All rules act in grid-index units (see geometry.py); a rule returns, for one
target, node ids and coefficients c such that the rule equals sum c[k] u[ids[k]]
(the coefficients already contain m omega of the source node).
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import j0, y0

from . import geometry as geo


def chi(s, s0: float):
    """C-infinity cut-off: 1 for |s| <= s0, 0 for |s| >= 1."""
    s = np.abs(np.asarray(s, dtype=np.float64))
    out = np.where(s <= s0, 1.0, 0.0)
    mid = (s > s0) & (s < 1.0)
    u = (s[mid] - s0) / (1.0 - s0)
    out[mid] = np.exp(2.0 * np.exp(-1.0 / u) / (u - 1.0))
    return out


def green(kappa: float, x, y):
    """G_kappa(x, y) = (i/4) H_0^(1)(kappa |x - y|) (Eq. G, 2-D)."""
    r = np.sqrt(np.sum((np.asarray(x) - np.asarray(y)) ** 2, -1))
    return hankel0(kappa * r) * 0.25j


def hankel0(z):
    """H_0^(1)(z) = J_0(z) + i Y_0(z) (scipy's cephes j0 / y0)."""
    return j0(z) + 1j * y0(z)


def lagrange(x, start, p: int):
    """Lagrange basis weights on the integer nodes start..start+p at x; shape (..., p+1)."""
    x = np.asarray(x, dtype=np.float64)[..., None]
    d = x - (np.asarray(start)[..., None] + np.arange(p + 1))      # x - node_m
    out = np.empty(d.shape)
    for k in range(p + 1):
        den = np.array([float(k - m) if m != k else 1.0 for m in range(p + 1)])
        f = d / den
        f[..., k] = 1.0
        out[..., k] = np.prod(f, -1)
    return out


def stencil_start(x, p: int):
    return np.floor(x).astype(np.int64) - p // 2


# ---------------------------------------------------------------- interpolation
def window_accumulate(f, a, b, sa, sb, oa, ob, Wa, Wb, p, pb=None):
    """sum over quadrature points of f * l_i(a) l_j(b) into per-target windows.

    f, a, b, sa, sb: (T, P) values, positions and stencil starts; oa, ob: (T,)
    window origins; degree p along a and pb (default p) along b.  Returns
    (T, Wa, Wb): coefficient of grid point (oa + i, ob + j) in the
    interpolated quadrature sum."""
    pb = p if pb is None else pb
    T, P = a.shape
    la = lagrange(a, sa, p)                      # (T, P, p+1)
    lb = lagrange(b, sb, pb)
    Ma = np.zeros((T, P, Wa), np.complex128)
    Mb = np.zeros((T, P, Wb))
    ia = (sa - oa[:, None])[..., None] + np.arange(p + 1)
    ib = (sb - ob[:, None])[..., None] + np.arange(pb + 1)
    # the p+1 stencil columns of one point are distinct, so plain assignment suffices
    np.put_along_axis(Ma, ia, la * f[..., None], axis=2)
    np.put_along_axis(Mb, ib, lb, axis=2)
    return np.matmul(np.swapaxes(Ma, 1, 2), Mb)   # (T, Wa, Wb)


def trig_kernel(t, n: int):
    """Band-limited interpolation kernel of n periodic unit-spaced samples at
    offset t: (1/n) sum over the n lowest frequencies of exp(2 pi i k t / n),
    the Nyquist term of even n split symmetrically; closed forms
    sin(pi t) / (n sin(pi t / n)) (n odd) and sin(pi t) / (n tan(pi t / n)) (n
    even).  1 at t = 0 (mod n), 0 at the other integers."""
    t = np.asarray(t, np.float64)
    tm = t - n * np.round(t / n)                 # in [-n/2, n/2]
    small = np.abs(tm) < 1e-12
    tt = np.where(small, 0.5, tm)
    den = n * (np.sin(np.pi * tt / n) if n % 2 else np.tan(np.pi * tt / n))
    return np.where(small, 1.0, np.sin(np.pi * tt) / den)


def refine_matrix(origin, W: int, n: int, F: int):
    """(T, W, n): the band-limited interpolant of n periodic coarse samples at
    the fine points (origin + m) / F, m < W, as weights on the coarse samples."""
    m = np.asarray(origin)[:, None] + np.arange(W)
    return trig_kernel(m[:, :, None] / F - np.arange(n)[None, None, :], n)


def fourier_windows(f, a, b, a_c, b_c, Ra, Rb, p, F, pf, na, nb, refine_b):
    """Windows of the Fourier-refined variant.  Along a (periodic, na samples):
    degree-pf Lagrange at a F on the F-fold refined grid, then the refined
    samples as band-limited interpolants of the coarse ones; along b the same
    when refine_b (nb samples), else degree-p Lagrange on the coarse lines
    (clamped to 0..nb-1).  a_c, b_c: (T,) window centres (coarse index units).
    Returns (T, na, Wb) windows with origins 0 (and Wb = nb)."""
    af = a * F
    saf = stencil_start(af, pf)
    oaf = np.floor((a_c - Ra) * F).astype(np.int64) - pf // 2 - 1
    Waf = 2 * int(math.ceil(Ra * F)) + pf + 4
    if refine_b:
        bf = b * F
        sbf = stencil_start(bf, pf)
        obf = np.floor((b_c - Rb) * F).astype(np.int64) - pf // 2 - 1
        Wbf = 2 * int(math.ceil(Rb * F)) + pf + 4
        Mf = window_accumulate(f, af, bf, saf, sbf, oaf, obf, Waf, Wbf, pf)
        Db = refine_matrix(obf, Wbf, nb, F)                 # (T, Wbf, nb)
        Mf = np.matmul(Mf, Db)                               # (T, Waf, nb)
    else:
        sb = np.clip(stencil_start(b, p), 0, nb - 1 - p)
        Mf = window_accumulate(f, af, b, saf, sb, oaf, np.zeros(len(a), np.int64), Waf, nb, pf, p)
    Da = refine_matrix(oaf, Waf, na, F)                      # (T, Waf, na)
    return np.matmul(np.swapaxes(Da, 1, 2), Mf)               # (T, na, nb)


# ---------------------------------------------------------------- rules
def collar_rb_interior(wl) -> float:
    """Transverse semi-axis of the collar cut-off for Cartesian targets: R_b, but
    no larger than tau0 (n2 - 1) so that the ellipse never reaches b = 0 (every
    Cartesian node has b > tau0 (n2 - 1))."""
    return min(wl.R_b, wl.tau0 * (wl.n2 - 1))


def polar_template(wl, Ra: float, Rb: float):
    """Nodes and weights of the polar rule of Eq. K-Int-Sing-Polar on the ellipse
    with index-unit semi-axes (Ra, Rb): (a, b) = (Ra rho cos theta, Rb rho sin theta),
    rho = s^q, s_k = k / n_rho, theta_m = 2 pi m / n_theta, trapezoid in both; the
    weight carries Ra Rb rho drho/ds and chi(rho)."""
    q = wl.q_polar
    s = np.arange(1, wl.n_rho) / wl.n_rho
    th = 2.0 * math.pi * np.arange(wl.n_theta) / wl.n_theta
    S, TH = np.meshgrid(s, th, indexing="ij")
    S, TH = S.ravel(), TH.ravel()
    rho = S ** q
    wq = (2.0 * math.pi / wl.n_theta) * (1.0 / wl.n_rho) * Ra * Rb * q * S ** (2 * q - 1) \
        * chi(rho, wl.chi_s0)
    keep = wq != 0.0
    return Ra * rho[keep] * np.cos(TH[keep]), Rb * rho[keep] * np.sin(TH[keep]), wq[keep]


def polar_rule(dz, chart: int, tgt, ax, bx):
    """eta-localised singular integrals (interior-type rule) for targets tgt
    centred at index points (ax, bx) of the chart (0 collar, 1 Cartesian).
    Returns COO triplets (target position in tgt, node id, coefficient)."""
    wl = dz.wl
    p = wl.p
    Ra, Rb = (wl.R_a, collar_rb_interior(wl)) if chart == 0 else (wl.R_cart, wl.R_cart)
    da, db, wq = polar_template(wl, Ra, Rb)
    tgt = np.asarray(tgt)
    ax = np.asarray(ax, np.float64)
    bx = np.asarray(bx, np.float64)
    a = ax[:, None] + da
    b = bx[:, None] + db
    w = np.broadcast_to(wq, a.shape).copy()
    if chart == 0:
        w[(b < 0.0) | (b > wl.n2 - 1)] = 0.0
        b = np.clip(b, 0.0, wl.n2 - 1)
        Y, J = geo.collar_map(wl, a, b)
    else:
        Y, J = geo.cart_map(wl, a, b)
    f = w * J * green(wl.kappa, dz.x[tgt][:, None, :], Y)
    fr = getattr(dz, "interp", None)
    if fr is not None:
        F, pf = fr
        na, nb = (wl.n1, wl.n2) if chart == 0 else (wl.cart_nx, wl.cart_ny)
        Mw = fourier_windows(f, a, b, ax, bx, Ra, Rb, p, F, pf, na, nb, refine_b=chart == 1)
        z = np.zeros(len(tgt), np.int64)
        return window_triplets(dz, chart, Mw, z, z)
    sa = stencil_start(a, p)
    sb = stencil_start(b, p)
    oa = np.floor(ax - Ra).astype(np.int64) - p // 2 - 1
    Wa = 2 * int(math.ceil(Ra)) + p + 4
    if chart == 0:
        sb = np.clip(sb, 0, wl.n2 - 1 - p)
        ob = np.zeros(len(tgt), np.int64)
        Wb = wl.n2
    else:
        ob = np.floor(bx - Rb).astype(np.int64) - p // 2 - 1
        Wb = 2 * int(math.ceil(Rb)) + p + 4
    Mw = window_accumulate(f, a, b, sa, sb, oa, ob, Wa, Wb, p)
    return window_triplets(dz, chart, Mw, oa, ob)


def window_triplets(dz, chart, Mw, oa, ob):
    """Map per-target windows (T, Wa, Wb) to COO triplets over node ids,
    multiplying by m omega of each node (phi = m omega u)."""
    wl = dz.wl
    T, Wa, Wb = Mw.shape
    ia = oa[:, None] + np.arange(Wa)                      # (T, Wa)
    ib = ob[:, None] + np.arange(Wb)
    if chart == 0:
        ia = np.mod(ia, wl.n1)
        okb = (ib >= 0) & (ib < wl.n2)
        ids = np.where(okb[:, None, :], dz.collar_id[ia[:, :, None], np.clip(ib, 0, wl.n2 - 1)[:, None, :]], -1)
    else:
        oka = (ia >= 0) & (ia < wl.cart_nx)
        okb = (ib >= 0) & (ib < wl.cart_ny)
        ids = np.where(oka[:, :, None] & okb[:, None, :],
                       dz.cart_id[np.clip(ia, 0, wl.cart_nx - 1)[:, :, None],
                                  np.clip(ib, 0, wl.cart_ny - 1)[:, None, :]], -1)
    rows = np.broadcast_to(np.arange(T)[:, None, None], ids.shape)
    keep = (ids >= 0) & (Mw != 0.0)
    ids = ids[keep]
    return rows[keep], ids, Mw[keep] * dz.phifac[ids]


def split_newton_cotes(j: int, nb: int, Q: int):
    """Transverse nodes and weights of Eq. VolInt-Adj-Sing-MultiSplit for a
    target on grid line j of a patch with lines 0..nb-1 (unit spacing).

    Q-point composite blocks run outward from j; the intervals left over near
    the ends (fewer than Q-1 of them) each get a Q-point rule on fractional
    lines k + m/(Q-1).  Returns dict {b: weight}."""
    nc = geo.newton_cotes(Q)
    out: dict[float, float] = {}

    def add(b, w):
        out[b] = out.get(b, 0.0) + w

    # downward from j
    L1 = j // (Q - 1)
    for l in range(1, L1 + 1):
        lo = j - l * (Q - 1)
        for m in range(Q):
            add(float(lo + m), nc[m])
    I1 = j - L1 * (Q - 1)
    for i in range(1, I1 + 1):
        lo = j - L1 * (Q - 1) - i
        for m in range(Q):
            add(lo + m / (Q - 1), nc[m] / (Q - 1))
    # upward from j
    top = nb - 1
    L2 = (top - j) // (Q - 1)
    for l in range(1, L2 + 1):
        lo = j + (l - 1) * (Q - 1)
        for m in range(Q):
            add(float(lo + m), nc[m])
    I2 = (top - j) - L2 * (Q - 1)
    for i in range(1, I2 + 1):
        lo = j + L2 * (Q - 1) + (i - 1)
        for m in range(Q):
            add(lo + m / (Q - 1), nc[m] / (Q - 1))
    return out


def boundary_rule(dz, tgt, i, j: int):
    """Singular integral over the collar for collar nodes (i, j) (all on the same
    transverse line j) as targets: rectangular cut-off chi(|a-i|/R_a) chi(|b-j|/R_b),
    varrho(tau) = R_a tau^(M+1) along the collar with N_tau trapezoid points on
    [-1, 1), split Newton-Cotes across.  Returns COO triplets."""
    wl = dz.wl
    p = wl.p
    Ra, Rb = wl.R_a, wl.R_b
    tgt = np.asarray(tgt)
    i = np.asarray(i, np.int64)
    tb = split_newton_cotes(j, wl.n2, wl.Q)
    bl = np.array([b for b in tb if abs(b - j) < Rb])
    wb = np.array([tb[b] for b in bl]) * chi((bl - j) / Rb, wl.chi_s0)
    tau = -1.0 + 2.0 * np.arange(wl.N_tau) / wl.N_tau
    rho = Ra * tau ** (wl.M + 1)
    drho = Ra * (wl.M + 1) * tau ** wl.M
    wt = (2.0 / wl.N_tau) * drho * chi(rho / Ra, wl.chi_s0)
    B, T = np.meshgrid(np.arange(len(bl)), np.arange(wl.N_tau), indexing="ij")
    B, T = B.ravel(), T.ravel()
    w1 = wb[B] * wt[T]
    keep = w1 != 0.0
    B, T, w1 = B[keep], T[keep], w1[keep]
    a = i[:, None] + rho[T][None, :]
    b = np.broadcast_to(bl[B], a.shape)
    Y, J = geo.collar_map(wl, a, b)
    f = w1 * J * green(wl.kappa, dz.x[tgt][:, None, :], Y)
    fr = getattr(dz, "interp", None)
    if fr is not None:
        F, pf = fr
        Mw = fourier_windows(f, a, b, i.astype(np.float64), np.full(len(tgt), float(j)), Ra, Rb, p, F, pf,
                             wl.n1, wl.n2, refine_b=False)
        z = np.zeros(len(tgt), np.int64)
        return window_triplets(dz, 0, Mw, z, z)
    sa = stencil_start(a, p)
    sb = np.clip(stencil_start(b, p), 0, wl.n2 - 1 - p)
    oa = i - int(math.ceil(Ra)) - p // 2 - 1
    Wa = 2 * int(math.ceil(Ra)) + p + 4
    ob = np.zeros(len(tgt), np.int64)
    Mw = window_accumulate(f, a, b, sa, sb, oa, ob, Wa, wl.n2, p)
    return window_triplets(dz, 0, Mw, oa, ob)


def needs_cart_rule(dz, q: int) -> bool:
    """True when a Cartesian node lies within reach of the Cartesian cut-off
    around target q (otherwise the Cartesian singular rule and its eta vanish)."""
    wl = dz.wl
    ga, gb = dz.ga[q], dz.gb[q]
    reach = wl.R_cart + wl.p / 2 + 2
    lo_a, hi_a = int(max(math.floor(ga - reach), 0)), int(min(math.ceil(ga + reach), wl.cart_nx - 1))
    lo_b, hi_b = int(max(math.floor(gb - reach), 0)), int(min(math.ceil(gb + reach), wl.cart_ny - 1))
    return lo_a <= hi_a and lo_b <= hi_b and bool(np.any(dz.cart_id[lo_a:hi_a + 1, lo_b:hi_b + 1] >= 0))


def singular_triplets(dz, targets):
    """COO triplets (row position, node id, coefficient) of every singular rule
    for the given target nodes."""
    wl = dz.wl
    targets = np.asarray(targets)
    out = []
    # Cartesian patch, interior-type rule
    sel = np.array([k for k, q in enumerate(targets) if needs_cart_rule(dz, int(q))], np.int64)
    if len(sel):
        r, c, v = polar_rule(dz, 1, targets[sel], dz.ga[targets[sel]], dz.gb[targets[sel]])
        out.append((sel[r], c, v))
    # collar patch, boundary rule for collar targets (grouped by transverse line)
    isc = dz.chart[targets] == 0
    for j in np.unique(dz.gj[targets[isc]]):
        sel = np.nonzero(isc & (dz.gj[targets] == j))[0]
        r, c, v = boundary_rule(dz, targets[sel], dz.gi[targets[sel]], int(j))
        out.append((sel[r], c, v))
    # collar patch, interior-type rule for Cartesian targets inside the collar chart
    sel = np.nonzero((~isc) & (dz.cb[targets] <= wl.n2 - 1))[0]
    if len(sel):
        r, c, v = polar_rule(dz, 0, targets[sel], dz.ca[targets[sel]], dz.cb[targets[sel]])
        out.append((sel[r], c, v))
    if not out:
        z = np.zeros(0, np.int64)
        return z, z, np.zeros(0, np.complex128)
    rows = np.concatenate([o[0] for o in out])
    cols = np.concatenate([o[1] for o in out])
    vals = np.concatenate([o[2] for o in out])
    keep = cols >= 0
    return rows[keep], cols[keep], vals[keep]


def eta_regular(dz, tgt, src=None):
    """eta_k(y_l; x_q) for targets tgt (T,) and source nodes src (S,): the cut-off
    of the patch that carries l, as used in the (1 - eta) regular term.  (T, S)."""
    wl = dz.wl
    tgt = np.atleast_1d(np.asarray(tgt))
    if src is None:
        src = np.arange(dz.N)
    eta = np.zeros((len(tgt), len(src)))
    isc = dz.chart[src] == 1
    sc = src[isc]
    # Cartesian sources: circular cut-off in Cartesian index units
    da = dz.ga[sc][None, :] - dz.ga[tgt][:, None]
    db = dz.gb[sc][None, :] - dz.gb[tgt][:, None]
    eta[:, isc] = chi(np.hypot(da, db) / wl.R_cart, wl.chi_s0)
    # collar sources
    icol = ~isc
    sl = src[icol]
    da = np.mod(dz.ca[sl][None, :] - dz.ca[tgt][:, None] + wl.n1 / 2, wl.n1) - wl.n1 / 2
    db = dz.cb[sl][None, :] - dz.cb[tgt][:, None]
    t_collar = (dz.chart[tgt] == 0)[:, None]
    t_inside = ((dz.chart[tgt] == 1) & (dz.cb[tgt] <= wl.n2 - 1))[:, None]
    rect = chi(da / wl.R_a, wl.chi_s0) * chi(db / wl.R_b, wl.chi_s0)
    circ = chi(np.hypot(da / wl.R_a, db / collar_rb_interior(wl)), wl.chi_s0)
    eta[:, icol] = np.where(t_collar, rect, np.where(t_inside, circ, 0.0))
    return eta
