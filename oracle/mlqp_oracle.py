"""Plain FP64 CPU oracle of the periodizing multilayer scheme of Cho & Barnett,
"Robust fast direct integral equation solver for quasi-periodic scattering
problems with a large number of layers" (arXiv 1410.5003).

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and the
CPU-baseline leg of bench.py, never by the product path.

Everything here is written for a reader checking it against the paper by eye:
NumPy arrays, SciPy's AMOS Hankel functions and LAPACK triangular / LU
routines as the only library primitives, no blocking or fusion.  Steps follow
the paper's order:

  Sec. 1        Bloch phase alpha, kappa_n, k^U_n, k^D_n            bloch()
  Sec. 2.5      nodes and weights on interfaces, walls, U, D;
                proxy points (eq. phi)                             *_nodes(), proxies()
  Sec. 2.1-2.2  kernels S, D, D*, T of G = (i/4) H0(k r)            green_kernels()
  eq. Ablocks   A_{i,i} (Mueller-Rokhlin differences), A_{i,i+-1}   self_block(), cross_block()
  eq. Bblocks   B_{i,i}, B_{i,i+1} (Bblockmat)                      b_block()
  eq. Cii, Qi   C_{j,j}, C_{j,j-1}, Q_j                             c_block(), q_block()
  eq. VUD, WUD  Z_U, Z_D, V_U, V_D, W_U, W_D                        z_block(), v_block(), w_block()
  Sec. 3.1      rearranged per-layer systems Q'_j, C'_j (linsys)    layer_system()
  Sec. 3.2      X_j = Q'_j \\ C'_j by column-pivoted QR; A' (Schur1-Schuri)
  Sec. 3.3      block-tridiagonal LU sweep, recovery of a^U, a^D
  Remark r:flux flux error

Readings of the paper that this oracle fixes:
  * Self-interaction quadrature: instead of Alpert's corrections the paper
    also names Kress' periodic log-split with cut-off functions (Remark
    phasewrap).  The three Bloch-phased copies are one integral over the
    unwrapped parameter s' in [-2pi, 4pi) with quasi-periodic density; the
    kernel nearest the target is split as chi(s'-t) K1 log(4 sin^2((t-s')/2))
    + K2, the first part integrated with Kress weights R_q, K2 with the plain
    trapezoid rule; chi is a C-infinity window (1 for |s'-t|<=a, 0 for >=b).
  * Flux error uses the incident vertical flux k_1 |sin theta|.
  * Forward sweep f~_i = f_i - A'_{i,i-1} A~_{i-1}^{-1} f~_{i-1}.
  * C'_{I+1,I} = [C_{I+1,I}; Z_D];  C entries use targets x_m + 2d and x_m - d.
  * "Backslash" (a backward-stable dense least-squares solve) is the
    regularised least squares min ||Q X - C||^2 + lam^2 ||X||^2 with
    lam = rcond * (largest column norm of Q), rcond = 1e-10, by Householder
    QR of [Q; lam I].  The truncated pivoted-QR basic solution (MATLAB's
    rectangular backslash) gives the same amplitudes to discretisation
    accuracy but jumps with rounding-level changes of Q (pivot and rank
    flips); the regularised solution is smooth in the data.
  * Corner (polyline) interfaces: graded Gauss-Legendre panels, `levels`
    panels per corner side halving toward the corner; the log-singular part
    of the self kernels is integrated by product integration on the target's
    own panel (Legendre log moments, exact) and on panels within one panel
    length (composite Gauss-Legendre graded toward the nearest point); the
    rest by the panel Gauss-Legendre rule.
  * U/D nodes x_m = -d/2 + d (m - 1/2)/M; y_U = y0_1 + sum_m |c_m| + gap_U
    (an upper bound of Gamma_1), y_D likewise below Gamma_I; the wall of
    layer j spans x = -d/2 between its bounding interfaces (or U, D); proxy
    circle centred at x = 0, mid-height of that wall; proxy p at angle
    2 pi (p-1)/P with outward normals.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
import scipy.linalg as sla
from scipy.special import hankel1, jv

TWO_PI = 2.0 * math.pi
EPS = np.finfo(np.float64).eps


# ----------------------------------------------------------------------------
# Sec. 1: Bloch phase, horizontal and vertical Rayleigh-Bloch wavenumbers
# ----------------------------------------------------------------------------
def vertical_wavenumber(k, kappa):
    """sqrt(k^2 - kappa^2) with the sign that makes it positive real or with
    positive imaginary part (upward/downward outgoing or decaying, eq. RB1)."""
    w = np.sqrt(np.asarray(k, np.complex128) ** 2 - np.asarray(kappa) ** 2 + 0j)
    return np.where(w.imag < 0, -w, w)


def bloch(prob, theta):
    """alpha = exp(i d k_1 cos theta) (eq. al); kappa_n = k_1 cos theta + 2 pi n/d,
    n = -K..K; k^U_n from k_1, k^D_n from k_{I+1}."""
    k1 = prob.k[0].real
    K = prob.params.K
    n = np.arange(-K, K + 1)
    kappa = k1 * math.cos(theta) + TWO_PI * n / prob.d
    return dict(alpha=np.exp(1j * prob.d * k1 * math.cos(theta)),
                kappa=kappa,
                kU=vertical_wavenumber(prob.k[0], kappa),
                kD=vertical_wavenumber(prob.k[-1], kappa))


# ----------------------------------------------------------------------------
# Sec. 2.5: quadrature nodes
# ----------------------------------------------------------------------------
@dataclass
class Nodes:
    x: np.ndarray
    y: np.ndarray
    nx: np.ndarray
    ny: np.ndarray
    speed: np.ndarray   # |Z'(s)|
    w: np.ndarray       # (2 pi / N) |Z'(s)|
    s: np.ndarray       # parameter values


def is_polyline(iface):
    return hasattr(iface, "vx")


def polyline_breaks(iface, d):
    """Breakpoints of a polyline interface: (-d/2, y0), the corners, (d/2, y0)."""
    xs = np.concatenate([[-d / 2], iface.vx, [d / 2]])
    ys = np.concatenate([[iface.y0], iface.vy, [iface.y0]])
    return xs, ys


def interface_height(iface, d, x):
    if is_polyline(iface):
        xs, ys = polyline_breaks(iface, d)
        return np.interp(np.atleast_1d(x), xs, ys)
    m = np.arange(1, len(iface.a) + 1)
    ph = TWO_PI * np.outer(np.atleast_1d(x), m) / d
    return iface.y0 + np.cos(ph) @ iface.a + np.sin(ph) @ iface.b


def interface_nodes(iface, d):
    if is_polyline(iface):
        return polyline_panels(iface, d).nodes
    return fourier_nodes(iface, d)


def fourier_nodes(iface, d):
    """Periodic trapezoid rule s_j = 2 pi (j - 1/2)/N on the graph
    parametrisation Z(s) = (-d/2 + s d/(2 pi), y(x(s))); unit normals point
    down, into the layer below (Sec. 2.1)."""
    N = iface.N
    s = TWO_PI * (np.arange(N) + 0.5) / N
    x = -d / 2 + s * d / TWO_PI
    m = np.arange(1, len(iface.a) + 1)
    ph = TWO_PI * np.outer(x, m) / d
    y = iface.y0 + np.cos(ph) @ iface.a + np.sin(ph) @ iface.b
    fp = (np.sin(ph) * (-TWO_PI * m / d)) @ iface.a + \
         (np.cos(ph) * (TWO_PI * m / d)) @ iface.b
    h = np.sqrt(1.0 + fp * fp)
    speed = (d / TWO_PI) * h
    return Nodes(x, y, fp / h, -1.0 / h, speed, (TWO_PI / N) * speed, s)


@dataclass
class Panels:
    """Gauss-Legendre panels of a polyline interface, in curve order.
    Panel q runs from (xa[q], ya[q]) to (xb[q], yb[q]) (length h[q]); node j
    lies on panel pan[j] at local coordinate loc[j] in [-1, 1]."""
    xa: np.ndarray
    ya: np.ndarray
    xb: np.ndarray
    yb: np.ndarray
    h: np.ndarray
    pan: np.ndarray
    loc: np.ndarray
    gl_x: np.ndarray    # reference nodes and weights on [-1, 1]
    gl_w: np.ndarray
    nodes: Nodes


def polyline_panels(iface, d):
    """Panels of a polyline interface.  A segment with corners at both ends is
    split at its midpoint; every corner side (corner c to far point f) carries
    `levels` panels with breakpoints c + (f - c) * {0, 2^-(L-1), ..., 1/2, 1},
    i.e. panel sizes halving toward the corner.  `order` Gauss-Legendre nodes
    per panel; arc-length parametrisation (speed 1), downward unit normals
    (dy, -dx)/h for a panel running in the +x direction."""
    xs, ys = polyline_breaks(iface, d)
    L, order = iface.levels, iface.order
    fr = np.concatenate([[0.0], 2.0 ** -np.arange(L - 1, -1, -1)])
    pts = []
    nseg = len(xs) - 1
    for g in range(nseg):
        a = np.array([xs[g], ys[g]])
        b = np.array([xs[g + 1], ys[g + 1]])
        ca, cb = g > 0, g < nseg - 1
        if ca and cb:
            m = 0.5 * (a + b)
            side = [a + (m - a) * f for f in fr] + [b + (m - b) * f for f in fr[::-1]][1:]
        elif cb:
            side = [b + (a - b) * f for f in fr[::-1]]
        else:
            side = [a + (b - a) * f for f in fr]
        if pts:
            side = side[1:]
        pts.extend(side)
    pts = np.array(pts)
    xa, ya = pts[:-1, 0], pts[:-1, 1]
    xb, yb = pts[1:, 0], pts[1:, 1]
    h = np.hypot(xb - xa, yb - ya)
    g, w = np.polynomial.legendre.leggauss(order)
    npan = len(h)
    pan = np.repeat(np.arange(npan), order)
    loc = np.tile(g, npan)
    t = 0.5 * (loc + 1.0)
    x = xa[pan] + (xb - xa)[pan] * t
    y = ya[pan] + (yb - ya)[pan] * t
    nx = (yb - ya)[pan] / h[pan]
    ny = -(xb - xa)[pan] / h[pan]
    wts = 0.5 * h[pan] * np.tile(w, npan)
    nodes = Nodes(x, y, nx, ny, np.ones_like(x), wts, loc)
    return Panels(xa, ya, xb, yb, h, pan, loc, g, w, nodes)


def legendre_log_moments(t, nmax):
    """L_n(t) = int_{-1}^{1} P_n(s) log|s - t| ds, n = 0..nmax, for -1 < t < 1.
    L_0 = (1 - t) log(1 - t) + (1 + t) log(1 + t) - 2; for n >= 1, integrating
    (2n+1) P_n = P'_{n+1} - P'_{n-1} by parts and using Neumann's formula
    PV int P_m(s)/(s - t) ds = -2 Q_m(t):  L_n = 2 (Q_{n+1}(t) - Q_{n-1}(t))/(2n+1),
    with Q_0 = (1/2) log((1+t)/(1-t)), Q_1 = t Q_0 - 1 and Bonnet's recursion
    (m+1) Q_{m+1} = (2m+1) t Q_m - m Q_{m-1} (stable on the cut)."""
    Q = np.zeros(nmax + 2)
    Q[0] = 0.5 * math.log((1.0 + t) / (1.0 - t))
    Q[1] = t * Q[0] - 1.0
    for m in range(1, nmax + 1):
        Q[m + 1] = ((2 * m + 1) * t * Q[m] - m * Q[m - 1]) / (m + 1)
    out = np.empty(nmax + 1)
    out[0] = (1 - t) * math.log(1 - t) + (1 + t) * math.log(1 + t) - 2.0
    for n in range(1, nmax + 1):
        out[n] = 2.0 * (Q[n + 1] - Q[n - 1]) / (2 * n + 1)
    return out


def lagrange_legendre(gl_x, gl_w, s):
    """Values l_j(s) of the Lagrange basis of the Gauss-Legendre nodes at the
    points s, through l_j = sum_n (2n+1)/2 w_j P_n(x_j) P_n (exact: the
    Gauss rule integrates l_j P_n, of degree <= 2p-2, exactly)."""
    p = len(gl_x)
    c = (2 * np.arange(p) + 1) / 2.0
    Pj = np.polynomial.legendre.legvander(gl_x, p - 1)          # (p, p): P_n(x_j)
    Ps = np.polynomial.legendre.legvander(np.atleast_1d(s), p - 1)  # (m, p)
    return (Ps * c) @ (Pj * gl_w[:, None]).T                       # (m, p): l_j(s_i)


def own_panel_log_weights(t, half, gl_x, gl_w):
    """W_j = int_panel l_j log|x(t) - y| ds_arc for the target at local
    coordinate t of the same straight panel (half-length `half`):
    |x(t) - y(s)| = half |t - s|, so W_j = half (w_j log(half) + int l_j log|t - s| ds)."""
    p = len(gl_x)
    c = (2 * np.arange(p) + 1) / 2.0
    Pj = np.polynomial.legendre.legvander(gl_x, p - 1)
    Lm = legendre_log_moments(t, p - 1)
    return half * (gl_w * math.log(half) + gl_w * (Pj @ (c * Lm)))


def near_panel_log_weights(px, py, xa, ya, xb, yb, gl_x, gl_w, pieces_min=1e-14):
    """W_j = int_panel l_j(s) log|x - y(s)| ds_arc for a target x = (px, py) off
    the panel: composite Gauss-Legendre rule on pieces of [-1, 1] graded
    geometrically (ratio 2) toward the local coordinate of the panel point
    nearest the target, starting from the target's distance."""
    dx, dy = xb - xa, yb - ya
    h = math.hypot(dx, dy)
    half = 0.5 * h
    cx, cy = 0.5 * (xa + xb), 0.5 * (ya + yb)
    sstar = ((px - cx) * dx + (py - cy) * dy) / (h * half)
    sstar = min(1.0, max(-1.0, sstar))
    qx, qy = cx + half * sstar * dx / h, cy + half * sstar * dy / h
    dist = max(math.hypot(px - qx, py - qy) / half, pieces_min)
    cuts = {-1.0, 1.0, sstar}
    step = dist
    while step < 2.0:
        cuts.update({sstar - step, sstar + step})
        step *= 2.0
    cuts = np.array(sorted(c for c in cuts if -1.0 <= c <= 1.0))
    W = np.zeros(len(gl_x))
    for u0, u1 in zip(cuts[:-1], cuts[1:]):
        su = 0.5 * (u0 + u1) + 0.5 * (u1 - u0) * gl_x
        wu = 0.5 * (u1 - u0) * gl_w
        yx, yy = cx + half * su * dx / h, cy + half * su * dy / h
        f = np.log(np.hypot(px - yx, py - yy))
        W += (lagrange_legendre(gl_x, gl_w, su) * (f * wu)[:, None]).sum(axis=0)
    return half * W


def panel_distance(px, py, xa, ya, xb, yb):
    dx, dy = xb - xa, yb - ya
    t = np.clip(((px - xa) * dx + (py - ya) * dy) / (dx * dx + dy * dy), 0.0, 1.0)
    return np.hypot(px - (xa + t * dx), py - (ya + t * dy))


def y_upper(prob):
    f = prob.ifaces[0]
    if is_polyline(f):
        return max(f.y0, float(np.max(f.vy))) + prob.params.gap_U
    return f.y0 + np.sum(np.hypot(f.a, f.b)) + prob.params.gap_U


def y_lower(prob):
    f = prob.ifaces[-1]
    if is_polyline(f):
        return min(f.y0, float(np.min(f.vy))) - prob.params.gap_D
    return f.y0 - np.sum(np.hypot(f.a, f.b)) - prob.params.gap_D


def wall_extent(prob, j):
    """(bottom, top) of the left wall L_j of layer j (1-based) at x = -d/2."""
    d, I = prob.d, prob.I
    bot = y_lower(prob) if j == I + 1 else interface_height(prob.ifaces[j - 1], d, -d / 2)[0]
    top = y_upper(prob) if j == 1 else interface_height(prob.ifaces[j - 2], d, -d / 2)[0]
    return bot, top


def wall_nodes(prob, j):
    """M_w Gauss-Legendre nodes on L_j (Sec. 2.5, eq. Qi)."""
    g, _ = np.polynomial.legendre.leggauss(prob.params.Mw)
    bot, top = wall_extent(prob, j)
    y = 0.5 * (top + bot) + 0.5 * (top - bot) * g
    return np.full_like(y, -prob.d / 2), y


def ud_nodes(prob, which):
    """M equispaced nodes on U (which='U') or D, x in (-d/2, d/2)."""
    M = prob.params.M
    x = -prob.d / 2 + prob.d * (np.arange(M) + 0.5) / M
    yv = y_upper(prob) if which == "U" else y_lower(prob)
    return x, np.full_like(x, yv)


def proxies(prob, j):
    """P proxy points on the circle of radius R about the centre of layer j's
    cell, with outward unit normals (eq. phi)."""
    P, R = prob.params.P, prob.params.R
    bot, top = wall_extent(prob, j)
    cy = 0.5 * (bot + top)
    ang = TWO_PI * np.arange(P) / P
    return R * np.cos(ang), cy + R * np.sin(ang), np.cos(ang), np.sin(ang)


# ----------------------------------------------------------------------------
# Sec. 2.1-2.2: kernels of G = (i/4) H0^(1)(k |r - r'|)   (eq. Gi)
# ----------------------------------------------------------------------------
def green_kernels(k, tx, ty, tnx, tny, sx, sy, snx, sny, log_parts=False):
    """Kernel values at targets (t, normal n) and sources (s, normal n'):
         S  = G                     D  = dG/dn'
         Ds = dG/dn                 T  = d^2 G / dn dn'
    With u = t - s, rho = |u|, g(rho) = (i/4)H0(k rho):
         g'  = -(ik/4) H1(k rho),   g'' = -(ik^2/4)(H0(k rho) - H1(k rho)/(k rho))
         D  = -g' (u.n')/rho,       Ds = g' (u.n)/rho
         T  = -[(g'' - g'/rho)(u.n)(u.n')/rho^2 + g' (n.n')/rho].
    If log_parts, also the coefficients K1 of log(4 sin^2((t-s)/2)) in the
    kernels (from Y_n = (2/pi) J_n log(z/2) + ...), without the |Z'| factor."""
    ux = tx - sx
    uy = ty - sy
    rho = np.hypot(ux, uy)
    z = k * rho
    H0 = hankel1(0, z)
    H1 = hankel1(1, z)
    un = (ux * tnx + uy * tny) / rho
    unp = (ux * snx + uy * sny) / rho
    nn = tnx * snx + tny * sny
    gp = -0.25j * k * H1
    gpp = -0.25j * k * k * (H0 - H1 / z)
    out = dict(S=0.25j * H0, D=-gp * unp, Ds=gp * un,
               T=-((gpp - gp / rho) * un * unp + gp * nn / rho))
    if log_parts:
        J0 = jv(0, z)
        J1 = jv(1, z)
        q = 1.0 / (4.0 * math.pi)
        out["K1S"] = -q * J0
        out["K1D"] = -q * k * J1 * unp
        out["K1Ds"] = q * k * J1 * un
        out["K1T"] = -q * k * k * (J0 - 2.0 * J1 / z) * un * unp - q * k * J1 * nn / rho
    return out


def proxy_fields(k, tx, ty, tnx, tny, px, py, pnx, pny):
    """phi_p = dG/dn_p + i k G (eq. phi) and its target-normal derivative."""
    g = green_kernels(k, tx, ty, tnx, tny, px, py, pnx, pny)
    return g["D"] + 1j * k * g["S"], g["T"] + 1j * k * g["Ds"]


# ----------------------------------------------------------------------------
# Periodic log-split quadrature (Remark phasewrap, Kress' rule with cut-off)
# ----------------------------------------------------------------------------
def kress_weights(N):
    """R_q = -(2pi/n) sum_{m=1}^{n-1} cos(m t_q)/m - (pi/n^2) cos(n t_q),
    t_q = 2 pi q/N, N = 2n: weights of the N-point rule for
    int_0^{2pi} log(4 sin^2((t-s)/2)) f(s) ds, as a function of q = index
    difference between target and source."""
    if N % 2:
        raise ValueError("the periodic log-split needs an even node count")
    n = N // 2
    q = np.arange(N)
    m = np.arange(1, n)
    tq = TWO_PI * q / N
    return -(TWO_PI / n) * (np.cos(np.outer(tq, m)) @ (1.0 / m)) \
        - (math.pi / n ** 2) * np.cos(n * tq)


def cutoff(delta, a, b):
    """C-infinity window: 1 for |delta| <= a, 0 for |delta| >= b, in between
    psi(u) = e^{-1/u} / (e^{-1/u} + e^{-1/(1-u)}) with u = (b-|delta|)/(b-a)."""
    ad = np.abs(np.asarray(delta, float))
    u = np.clip((b - ad) / (b - a), 0.0, 1.0)
    out = np.zeros_like(u)
    mid = (u > 0) & (u < 1)
    e1 = np.exp(-1.0 / u[mid])
    e2 = np.exp(-1.0 / (1.0 - u[mid]))
    out[mid] = e1 / (e1 + e2)
    out[u >= 1] = 1.0
    return out


def self_diag_limits(k1, k2, speed):
    """Limits at s' = t of K2 = K - K1 log(4 sin^2((t-s')/2)) and of K1 for
    the difference kernels K^{k1} - K^{k2} (|Z'| included), from the small-
    argument series of H0 and H1 (Abramowitz & Stegun 9.1.11-9.1.13)."""
    lk1, lk2 = np.log(k1), np.log(k2)
    q = speed / (4.0 * math.pi)
    c = -0.5j * math.pi - 0.5 + np.euler_gamma - math.log(2.0) + np.log(speed)
    return dict(
        S2=-2.0 * q * (lk1 - lk2), S1=0.0 * speed,
        D2=0.0 * speed, D1=0.0 * speed,
        Ds2=0.0 * speed, Ds1=0.0 * speed,
        T2=-q * ((k1 * k1 - k2 * k2) * c + k1 * k1 * lk1 - k2 * k2 * lk2),
        T1=-0.5 * q * (k1 * k1 - k2 * k2))


def _copies_xy(nd, d):
    """Source coordinates of the three copies l = -1, 0, 1 (shape (3, N))."""
    ls = np.array([-1, 0, 1])[:, None]
    return nd.x[None, :] + ls * d, np.broadcast_to(nd.y, (3, len(nd.y)))


# ----------------------------------------------------------------------------
# eq. Ablocks: near-field Nystrom blocks, as alpha-power -> matrix dictionaries
# (Sec. 3.4: the integrals of each copy do not depend on alpha)
# ----------------------------------------------------------------------------
NEAR_PANELS = 1.0  # a source panel closer to the target than this many of its lengths is "near"


def panel_self_block_terms(prob, i):
    """Per-copy parts of A_{i,i} for a polyline interface (graded
    Gauss-Legendre panels).  The difference kernels are split as
    K = K_L log(rho) + K_R, K_L = 2 K1 (the coefficient of log rho; K1 is
    the coefficient of log(4 sin^2(./2)), i.e. of 2 log rho).  Far panels
    take the Gauss-Legendre rule w_j K.  Near panels (the target's own panel
    and any panel within NEAR_PANELS of its lengths, in any copy) integrate
    the log part by product integration: w_j (K - K_L log rho_j) + W_j K_L,
    W_j = int_panel l_j log|x - y| ds.  At the target's own node the entry is
    w_j K_R(t,t) + W_j K_L(t,t), the diagonal limits at unit speed (arc
    length).  Identities -I, +I sit in l = 0."""
    d = prob.d
    P = polyline_panels(prob.ifaces[i - 1], d)
    nd = P.nodes
    N = len(nd.x)
    k1, k2 = prob.k[i - 1], prob.k[i]
    lim = self_diag_limits(k1, k2, 1.0)
    keys = ("S", "D", "Ds", "T")
    out = {}
    for l in (-1, 0, 1):
        TX, SX = np.meshgrid(nd.x, nd.x + l * d, indexing="ij")
        TY, SY = np.meshgrid(nd.y, nd.y, indexing="ij")
        TNX, SNX = np.meshgrid(nd.nx, nd.nx, indexing="ij")
        TNY, SNY = np.meshgrid(nd.ny, nd.ny, indexing="ij")
        off = np.ones((N, N), bool)
        if l == 0:
            off[np.arange(N), np.arange(N)] = False
        g1 = green_kernels(k1, TX[off], TY[off], TNX[off], TNY[off], SX[off], SY[off], SNX[off], SNY[off], log_parts=True)
        g2 = green_kernels(k2, TX[off], TY[off], TNX[off], TNY[off], SX[off], SY[off], SNX[off], SNY[off], log_parts=True)
        rho = np.full((N, N), np.nan)
        rho[off] = np.hypot(TX[off] - SX[off], TY[off] - SY[off])
        K, KL = {}, {}
        for key in keys:
            K[key] = np.zeros((N, N), np.complex128)
            KL[key] = np.zeros((N, N), np.complex128)
            K[key][off] = g1[key] - g2[key]
            KL[key][off] = 2.0 * (g1["K1" + key] - g2["K1" + key])
        M = {key: K[key] * nd.w[None, :] for key in keys}
        for m in range(N):
            for q in range(len(P.h)):
                xa, xb = P.xa[q] + l * d, P.xb[q] + l * d
                own = (l == 0 and P.pan[m] == q)
                if not own and panel_distance(nd.x[m], nd.y[m], xa, P.ya[q], xb, P.yb[q]) >= NEAR_PANELS * P.h[q]:
                    continue
                idx = np.nonzero(P.pan == q)[0]
                if own:
                    W = own_panel_log_weights(P.loc[m], 0.5 * P.h[q], P.gl_x, P.gl_w)
                else:
                    W = near_panel_log_weights(nd.x[m], nd.y[m], xa, P.ya[q], xb, P.yb[q], P.gl_x, P.gl_w)
                for jj, j in enumerate(idx):
                    for key in keys:
                        if own and j == m:
                            M[key][m, m] = nd.w[m] * lim[key + "2"] + W[jj] * 2.0 * lim[key + "1"]
                        else:
                            M[key][m, j] += (W[jj] - nd.w[j] * math.log(rho[m, j])) * KL[key][m, j]
        blk = np.block([[M["D"], M["S"]], [M["T"], M["Ds"]]])
        if l == 0:
            blk = blk + np.diag(np.concatenate([-np.ones(N), np.ones(N)]))
        out[l] = blk
    return out


def self_block_terms(prob, i):
    """Per-copy parts of A_{i,i} (i is 1-based): dict {l: (2N x 2N)} with
    A_{i,i} = sum_l alpha^l M_l.  Kernels are the differences of layer i and
    layer i+1 kernels (Mueller-Rokhlin pairs); identities -I, +I sit in l=0.
    Smooth interfaces: the periodic log-split below; polylines: panels."""
    if is_polyline(prob.ifaces[i - 1]):
        return panel_self_block_terms(prob, i)
    prm = prob.params
    nd = interface_nodes(prob.ifaces[i - 1], prob.d)
    N = len(nd.x)
    n = N // 2
    k1, k2 = prob.k[i - 1], prob.k[i]
    R = kress_weights(N)
    h = TWO_PI / N
    m_idx = np.arange(N)[:, None]
    out = {}
    for li, l in enumerate((-1, 0, 1)):
        j_idx = np.arange(N)[None, :]
        q = j_idx + l * N - m_idx                      # unwrapped index offset
        delta = h * q                                   # s' - t
        sx = nd.x[None, :] + l * prob.d
        sy = nd.y[None, :]
        T = dict(S=0, D=0, Ds=0, T=0)
        off = q != 0
        tx, ty = np.broadcast_to(nd.x[:, None], q.shape), np.broadcast_to(nd.y[:, None], q.shape)
        tnx, tny = np.broadcast_to(nd.nx[:, None], q.shape), np.broadcast_to(nd.ny[:, None], q.shape)
        sxb, syb = np.broadcast_to(sx, q.shape), np.broadcast_to(sy, q.shape)
        snx, sny = np.broadcast_to(nd.nx[None, :], q.shape), np.broadcast_to(nd.ny[None, :], q.shape)
        spd = np.broadcast_to(nd.speed[None, :], q.shape)
        g1 = green_kernels(k1, tx[off], ty[off], tnx[off], tny[off], sxb[off], syb[off],
                           snx[off], sny[off], log_parts=True)
        g2 = green_kernels(k2, tx[off], ty[off], tnx[off], tny[off], sxb[off], syb[off],
                           snx[off], sny[off], log_parts=True)
        chi = cutoff(delta[off], prm.cut_a, prm.cut_b)
        inwin = np.abs(q[off]) <= n - 1
        chi = np.where(inwin, chi, 0.0)
        qa = np.abs(q[off]) % N
        with np.errstate(divide="ignore"):
            lg = np.log(4.0 * np.sin(0.5 * delta[off]) ** 2)
        corr = np.where(inwin, chi * (R[qa] - h * np.where(inwin, lg, 0.0)), 0.0)
        for key in ("S", "D", "Ds", "T"):
            M = np.zeros((N, N), np.complex128)
            kv = (g1[key] - g2[key]) * spd[off]
            k1v = (g1["K1" + key] - g2["K1" + key]) * spd[off]
            M[off] = h * kv + corr * k1v
            if l == 0:
                lim = self_diag_limits(k1, k2, nd.speed)
                M[np.arange(N), np.arange(N)] = h * lim[key + "2"] + R[0] * lim[key + "1"]
            T[key] = M
        blk = np.block([[T["D"], T["S"]], [T["T"], T["Ds"]]])
        if l == 0:
            blk = blk + np.diag(np.concatenate([-np.ones(N), np.ones(N)]))
        out[l] = blk
    return out


def _plain_layer_terms(k, tx, ty, tnx, tny, nd, d, shifts, sign=1.0):
    """Plain Nystrom [[D, S], [T, Ds]] from interface nodes nd to targets, for
    each source copy shift l (sources at z + l d), weights w_j."""
    out = {}
    for l in shifts:
        g = green_kernels(k, tx[:, None], ty[:, None], tnx[:, None], tny[:, None],
                          nd.x[None, :] + l * d, nd.y[None, :], nd.nx[None, :], nd.ny[None, :])
        w = nd.w[None, :]
        out[l] = sign * np.block([[g["D"] * w, g["S"] * w], [g["T"] * w, g["Ds"] * w]])
    return out


def cross_block_terms(prob, i, j):
    """A_{i,j} for j = i+1 (layer i+1 kernels, minus sign) or j = i-1 (layer i
    kernels, plus sign): targets Gamma_i, sources Gamma_j and its copies."""
    ni = interface_nodes(prob.ifaces[i - 1], prob.d)
    nj = interface_nodes(prob.ifaces[j - 1], prob.d)
    if j == i + 1:
        k, sign = prob.k[i], -1.0
    elif j == i - 1:
        k, sign = prob.k[i - 1], 1.0
    else:
        raise ValueError("A is block tridiagonal")
    return _plain_layer_terms(k, ni.x, ni.y, ni.nx, ni.ny, nj, prob.d, (-1, 0, 1), sign)


def b_block(prob, i, j):
    """B_{i,i} = [phi^i_p; d phi^i_p/dn] on Gamma_i, B_{i,i+1} = -[phi^{i+1}_p; ...]
    (eqs. Bblocks, Bblockmat).  Independent of alpha."""
    nd = interface_nodes(prob.ifaces[i - 1], prob.d)
    px, py, pnx, pny = proxies(prob, j)
    k = prob.k[j - 1]
    v, dv = proxy_fields(k, nd.x[:, None], nd.y[:, None], nd.nx[:, None], nd.ny[:, None],
                         px[None, :], py[None, :], pnx[None, :], pny[None, :])
    sign = 1.0 if j == i else -1.0
    if j not in (i, i + 1):
        raise ValueError("B has blocks (i,i) and (i,i+1) only")
    return sign * np.vstack([v, dv])


def c_block_terms(prob, j, i):
    """C_{j,i} (layer j, interface i in {j-1, j}): rows = wall values then
    x-derivatives at the GL nodes x_m of L_j; entries
    (alpha^{-2} K(x_m + 2d, z) - alpha K(x_m - d, z)) w (eq. Cii)."""
    xw, yw = wall_nodes(prob, j)
    nd = interface_nodes(prob.ifaces[i - 1], prob.d)
    k = prob.k[j - 1]
    one, zero = np.ones_like(xw), np.zeros_like(xw)
    tp = _plain_layer_terms(k, xw + 2 * prob.d, yw, one, zero, nd, prob.d, (0,))[0]
    tm = _plain_layer_terms(k, xw - prob.d, yw, one, zero, nd, prob.d, (0,))[0]
    return {-2: tp, 1: -tm}


def q_block_terms(prob, j):
    """Q_j: alpha^{-1} phi_p(x_m + d) - phi_p(x_m) and the same for d/dx (eq. Qi)."""
    xw, yw = wall_nodes(prob, j)
    px, py, pnx, pny = proxies(prob, j)
    k = prob.k[j - 1]
    one, zero = np.ones_like(xw), np.zeros_like(xw)

    def at(xs):
        v, dv = proxy_fields(k, xs[:, None], yw[:, None], one[:, None], zero[:, None],
                             px[None, :], py[None, :], pnx[None, :], pny[None, :])
        return np.vstack([v, dv])
    return {-1: at(xw + prob.d), 0: -at(xw)}


def z_block_terms(prob, which):
    """Z_U = [[D~, S~], [T~, D~*]] from Gamma_1 to U (layer 1 kernels), Z_D from
    Gamma_I to D (layer I+1 kernels); target normals point up (eq. VUD)."""
    x, y = ud_nodes(prob, which)
    if which == "U":
        nd, k = interface_nodes(prob.ifaces[0], prob.d), prob.k[0]
    else:
        nd, k = interface_nodes(prob.ifaces[-1], prob.d), prob.k[-1]
    return _plain_layer_terms(k, x, y, np.zeros_like(x), np.ones_like(x), nd, prob.d, (-1, 0, 1))


def v_block(prob, which):
    x, y = ud_nodes(prob, which)
    j = 1 if which == "U" else prob.I + 1
    px, py, pnx, pny = proxies(prob, j)
    k = prob.k[j - 1]
    v, dv = proxy_fields(k, x[:, None], y[:, None], np.zeros((len(x), 1)), np.ones((len(x), 1)),
                         px[None, :], py[None, :], pnx[None, :], pny[None, :])
    return np.vstack([v, dv])


def w_block(prob, which, bl):
    """W_U = [-e^{i kappa_n x}; -i k^U_n e^{i kappa_n x}],
    W_D = [-e^{i kappa_n x};  +i k^D_n e^{i kappa_n x}] (eq. WUD)."""
    x, _ = ud_nodes(prob, which)
    e = np.exp(1j * np.outer(x, bl["kappa"]))
    if which == "U":
        return np.vstack([-e, -1j * bl["kU"][None, :] * e])
    return np.vstack([-e, 1j * bl["kD"][None, :] * e])


def assemble(terms, alpha):
    return sum((alpha ** l) * M for l, M in terms.items())


def rhs(prob, theta):
    """f_1 = [-u_inc; -du_inc/dn] on Gamma_1, u_inc = exp(i k_1 (cos th x + sin th y))."""
    nd = interface_nodes(prob.ifaces[0], prob.d)
    k1 = prob.k[0].real
    kx, ky = k1 * math.cos(theta), k1 * math.sin(theta)
    u = np.exp(1j * (kx * nd.x + ky * nd.y))
    return np.concatenate([-u, -1j * (kx * nd.nx + ky * nd.ny) * u])


# ----------------------------------------------------------------------------
# Sec. 3.1: per-layer rearranged blocks Q'_j and C'_j
# ----------------------------------------------------------------------------
def layer_columns(prob, j):
    """Interfaces (1-based) whose densities layer j's C' block acts on, in
    column order: layer 1 -> [1]; 2..I -> [j-1, j]; I+1 -> [I]."""
    I = prob.I
    if j == 1:
        return [1]
    if j == I + 1:
        return [I]
    return [j - 1, j]


class Assembler:
    """Caches the alpha-independent per-copy matrices (Sec. 3.4) and builds the
    blocks of eq. linsys for any angle."""

    def __init__(self, prob):
        self.prob = prob
        self._c = {}

    def _get(self, key, fn):
        if key not in self._c:
            self._c[key] = fn()
        return self._c[key]

    def A(self, i, j, alpha):
        p = self.prob
        if i == j:
            return assemble(self._get(("A", i, i), lambda: self_block_terms(p, i)), alpha)
        return assemble(self._get(("A", i, j), lambda: cross_block_terms(p, i, j)), alpha)

    def B(self, i, j):
        return self._get(("B", i, j), lambda: b_block(self.prob, i, j))

    def Qp(self, j, alpha, bl):
        """Q'_j: Q_j for middle layers; [[Q, 0], [V, W]] for layers 1 and I+1."""
        p = self.prob
        Q = assemble(self._get(("Q", j), lambda: q_block_terms(p, j)), alpha)
        if j not in (1, p.I + 1):
            return Q
        which = "U" if j == 1 else "D"
        V = self._get(("V", which), lambda: v_block(p, which))
        W = w_block(p, which, bl)
        Z0 = np.zeros((Q.shape[0], W.shape[1]), np.complex128)
        return np.block([[Q, Z0], [V, W]])

    def Cp(self, j, alpha):
        """C'_j: [C_{j,j-1}, C_{j,j}] for middle layers, [C_{1,1}; Z_U] and
        [C_{I+1,I}; Z_D] at the ends."""
        p = self.prob
        cols = [assemble(self._get(("C", j, i), lambda i=i: c_block_terms(p, j, i)), alpha)
                for i in layer_columns(p, j)]
        C = np.hstack(cols)
        if j == 1:
            Z = assemble(self._get(("Z", "U"), lambda: z_block_terms(p, "U")), alpha)
            C = np.vstack([C, Z])
        elif j == p.I + 1:
            Z = assemble(self._get(("Z", "D"), lambda: z_block_terms(p, "D")), alpha)
            C = np.vstack([C, Z])
        return C


# ----------------------------------------------------------------------------
# Sec. 3.2: least squares by column-pivoted Householder QR (Businger-Golub)
# ----------------------------------------------------------------------------
def pivoted_qr(A, rcond):
    """Householder QR with column pivoting: at step j pick, among columns
    j..n-1, the first one of largest 2-norm over rows j..m-1.  Returns the
    reflectors (v_j, beta_j), R, the permutation and the numerical rank
    #{leading |R_kk| > rcond |R_00|}."""
    R = np.array(A, dtype=np.complex128, copy=True)
    m, n = R.shape
    piv = np.arange(n)
    refl = []
    steps = min(m, n)
    for j in range(steps):
        norms = np.sqrt(np.sum(np.abs(R[j:, j:]) ** 2, axis=0))
        p = j + int(np.argmax(norms))
        if p != j:
            R[:, [j, p]] = R[:, [p, j]]
            piv[[j, p]] = piv[[p, j]]
        x = R[j:, j]
        nx = np.sqrt(np.sum(np.abs(x) ** 2))
        if nx == 0.0:
            refl.append((np.zeros_like(x), 0.0))
            continue
        ph = x[0] / abs(x[0]) if x[0] != 0 else 1.0
        alpha = -ph * nx
        v = x.copy()
        v[0] -= alpha
        beta = 2.0 / np.real(np.vdot(v, v))
        R[j:, j:] -= beta * np.outer(v, v.conj() @ R[j:, j:])
        refl.append((v, beta))
    diag = np.abs(np.diag(R[:steps, :steps]))
    tol = rcond * diag[0] if steps else 0.0
    rank = 0
    while rank < steps and diag[rank] > tol:
        rank += 1
    return refl, np.triu(R[:steps, :]), piv, rank


def lsq_pivoted(Q, C, rcond):
    """X = Q \\ C: least-squares basic solution (zeros in the non-pivot
    columns) via pivoted QR of numerical rank #{|R_kk| > rcond |R_00|}
    (MATLAB's rectangular backslash with a relative tolerance).  Kept as a
    cross-check of lsq(); the solver itself uses lsq()."""
    refl, R, piv, r = pivoted_qr(Q, rcond)
    B = np.array(C, dtype=np.complex128, copy=True)
    for j, (v, beta) in enumerate(refl):
        if beta:
            B[j:] -= beta * np.outer(v, v.conj() @ B[j:])
    X = np.zeros((Q.shape[1], C.shape[1]), np.complex128)
    if r:
        X[piv[:r]] = sla.solve_triangular(R[:r, :r], B[:r], lower=False)
    return X


def lsq(Q, C, rcond):
    """X_j = Q'_j \\ C'_j (Sec. 3.2) as the regularised least-squares solution
    argmin ||Q X - C||^2 + lam^2 ||X||^2, lam = rcond * max_c ||Q[:, c]||,
    computed by Householder QR of the stacked matrix [Q; lam I] (backward
    stable; the pseudo-inverse is never formed).  It selects small-norm proxy
    strengths, the property the remark after eq. Schuri relies on, and it
    depends smoothly on Q and C, unlike a rank-truncated basic solution."""
    m, p = Q.shape
    lam = rcond * np.max(np.sqrt(np.sum(np.abs(Q) ** 2, axis=0)))
    A = np.vstack([Q, lam * np.eye(p)])
    B = np.vstack([C, np.zeros((p, C.shape[1]), np.complex128)])
    q, r = np.linalg.qr(A)
    return sla.solve_triangular(r, q.conj().T @ B, lower=False)


def lsq_adjoint(Q, G, rcond):
    """Y = (Q^H Q + lam^2 I)^{-1} G, lam as in lsq(): the adjoint of the
    regularised least squares (a functional with sensitivity G to X has
    sensitivity Q Y to C), by two triangular solves with the R of [Q; lam I]."""
    m, p = Q.shape
    lam = rcond * np.max(np.sqrt(np.sum(np.abs(Q) ** 2, axis=0)))
    _, r = np.linalg.qr(np.vstack([Q, lam * np.eye(p)]))
    z = sla.solve_triangular(r.conj().T, G, lower=True)
    return sla.solve_triangular(r, z, lower=False)


# ----------------------------------------------------------------------------
# Sec. 3.2: Schur complements (eqs. Schur1 - Schuri)
# ----------------------------------------------------------------------------
def schur(prob, theta, asm=None):
    """Returns dict with alpha, the per-layer Q', C', X, the blocks of A'
    (diag, lower, upper), A (unreduced) and the right-hand side."""
    asm = asm or Assembler(prob)
    I, P = prob.I, prob.params.P
    bl = bloch(prob, theta)
    al = bl["alpha"]
    n = [2 * f.N for f in prob.ifaces]
    X, Qp, Cp = {}, {}, {}
    for j in range(1, I + 2):
        Qp[j] = asm.Qp(j, al, bl)
        Cp[j] = asm.Cp(j, al)
        X[j] = lsq(Qp[j], Cp[j], prob.params.lsq_rcond)

    def xcols(j, i):
        """Columns of X_j acting on eta_i, first P rows (proxy strengths)."""
        off = 0
        for ii in layer_columns(prob, j):
            if ii == i:
                return X[j][:P, off:off + n[i - 1]]
            off += n[ii - 1]
        raise KeyError

    Ad, Al, Au, A0d, A0l, A0u = {}, {}, {}, {}, {}, {}
    for i in range(1, I + 1):
        A0d[i] = asm.A(i, i, al)
        Ad[i] = A0d[i] - asm.B(i, i) @ xcols(i, i) - asm.B(i, i + 1) @ xcols(i + 1, i)
        if i < I:
            A0u[i] = asm.A(i, i + 1, al)
            Au[i] = A0u[i] - asm.B(i, i + 1) @ xcols(i + 1, i + 1)
        if i > 1:
            A0l[i] = asm.A(i, i - 1, al)
            Al[i] = A0l[i] - asm.B(i, i) @ xcols(i, i - 1)
    f = {i: np.zeros(n[i - 1], np.complex128) for i in range(1, I + 1)}
    f[1] = rhs(prob, theta)
    return dict(bloch=bl, Qp=Qp, Cp=Cp, X=X, Ad=Ad, Al=Al, Au=Au,
                A0d=A0d, A0l=A0l, A0u=A0u, f=f)


# ----------------------------------------------------------------------------
# Sec. 3.3: block-tridiagonal LU (forward and backward sweeps), recovery
# ----------------------------------------------------------------------------
def block_thomas(Ad, Al, Au, f, I):
    """Forward sweep A~_1 = A'_{1,1}, f~_1 = f_1;
    A~_i = A'_{i,i} - A'_{i,i-1} A~_{i-1}^{-1} A'_{i-1,i},
    f~_i = f_i - A'_{i,i-1} A~_{i-1}^{-1} f~_{i-1};
    backward A~_I eta_I = f~_I, A~_i eta_i = f~_i - A'_{i,i+1} eta_{i+1}."""
    At, ft, lu = {1: Ad[1]}, {1: f[1]}, {}
    for i in range(2, I + 1):
        lu[i - 1] = sla.lu_factor(At[i - 1])
        Y = sla.lu_solve(lu[i - 1], Au[i - 1])
        At[i] = Ad[i] - Al[i] @ Y
        ft[i] = f[i] - Al[i] @ sla.lu_solve(lu[i - 1], ft[i - 1])
    lu[I] = sla.lu_factor(At[I])
    eta = {I: sla.lu_solve(lu[I], ft[I])}
    for i in range(I - 1, 0, -1):
        eta[i] = sla.lu_solve(lu[i], ft[i] - Au[i] @ eta[i + 1])
    return eta


def adjoint_block_thomas(Ad, Al, Au, h, I):
    """mu = A'^{-H} h by the same block elimination on the conjugate-transposed
    system: (A'^H)_{i,i} = A'_{i,i}^H, (A'^H)_{i,i-1} = A'_{i-1,i}^H and
    (A'^H)_{i,i+1} = A'_{i+1,i}^H (the adjoint of the Sec. 3.3 system)."""
    H = lambda M: M.conj().T
    Bd = {i: H(Ad[i]) for i in range(1, I + 1)}
    Bl = {i: H(Au[i - 1]) for i in range(2, I + 1)}
    Bu = {i: H(Al[i + 1]) for i in range(1, I)}
    return block_thomas(Bd, Bl, Bu, h, I)


def recover_amplitudes(prob, X, eta):
    """x_1 = -Q'^+_1 C'_{1,1} eta_1, x_{I+1} = -Q'^+_{I+1} C'_{I+1,I} eta_I; the
    Bragg amplitudes are their last 2K+1 entries (n = -K..K)."""
    P, I = prob.params.P, prob.I
    aU = -(X[1][P:, :] @ eta[1])
    aD = -(X[I + 1][P:, :] @ eta[I])
    return aU, aD


def flux_error(prob, theta, bl, aU, aD):
    """(sum_{k^U_n>0} k^U_n |a^U_n|^2 + sum_{k^D_n>0} k^D_n |a^D_n|^2 - k_1|sin th|)
    / (k_1 |sin th|); NaN unless every layer wavenumber is real (Remark r:flux)."""
    if np.any(prob.k.imag != 0):
        return float("nan")
    k1 = prob.k[0].real
    inc = k1 * abs(math.sin(theta))
    pu = (bl["kU"].imag == 0) & (bl["kU"].real > 0)
    pd = (bl["kD"].imag == 0) & (bl["kD"].real > 0)
    out = np.sum(bl["kU"].real[pu] * np.abs(aU[pu]) ** 2) + \
        np.sum(bl["kD"].real[pd] * np.abs(aD[pd]) ** 2)
    return float((out - inc) / inc)


def solve(prob, itheta=0, asm=None, keep=False):
    """Full plain solve for angle prob.theta[itheta]."""
    theta = float(prob.theta[itheta])
    sc = schur(prob, theta, asm)
    eta = block_thomas(sc["Ad"], sc["Al"], sc["Au"], sc["f"], prob.I)
    aU, aD = recover_amplitudes(prob, sc["X"], eta)
    res = dict(theta=theta, aU=aU, aD=aD, eta=np.concatenate([eta[i] for i in range(1, prob.I + 1)]),
               flux=flux_error(prob, theta, sc["bloch"], aU, aD), bloch=sc["bloch"])
    if keep:
        res["schur"] = sc
    return res


# ----------------------------------------------------------------------------
# Adjoint gradient of a Bragg-efficiency objective (the differentiation form:
# transposed block solve, least-squares adjoint, block sensitivities).  The
# derivatives of the blocks with respect to a parameter are taken by central
# differences of this module's own assembly ("numeric kernel-derivative
# pass"); everything else is the adjoint of the solve.
# ----------------------------------------------------------------------------
def reflected_weights(prob, theta, bl, orders=(0, -1)):
    """w_n = k^U_n / (k_1 |sin theta|) for the propagating orders among
    `orders` (0 otherwise): the reflected efficiency of order n is w_n |a^U_n|^2."""
    K = prob.params.K
    inc = prob.k[0].real * abs(math.sin(theta))
    w = np.zeros(2 * K + 1)
    for n in orders:
        kv = bl["kU"][K + n]
        if kv.imag == 0 and kv.real > 0:
            w[K + n] = kv.real / inc
    return w


def bragg_objective(prob, asm=None, orders=(0, -1)):
    """J = sum over the angles of the reflected efficiencies of `orders`."""
    asm = asm or Assembler(prob)
    J = 0.0
    for a in range(prob.n_theta):
        th = float(prob.theta[a])
        r = solve(prob, a, asm)
        w = reflected_weights(prob, th, bloch(prob, th), orders)
        J += float(np.sum(w * np.abs(r["aU"]) ** 2))
    return J


def _blocks(prob, theta):
    """The parameter-dependent blocks of one angle: A (unreduced), B, Q', C', f."""
    asm = Assembler(prob)
    bl = bloch(prob, theta)
    al = bl["alpha"]
    I = prob.I
    A = {}
    for i in range(1, I + 1):
        for j in (i - 1, i, i + 1):
            if 1 <= j <= I:
                A[(i, j)] = asm.A(i, j, al)
    B = {(i, j): asm.B(i, j) for i in range(1, I + 1) for j in (i, i + 1)}
    Qp = {j: asm.Qp(j, al, bl) for j in range(1, I + 2)}
    Cp = {j: asm.Cp(j, al) for j in range(1, I + 2)}
    return dict(A=A, B=B, Qp=Qp, Cp=Cp, f=rhs(prob, theta), w=reflected_weights(prob, theta, bl))


def adjoint_gradient(prob, shifted, step, orders=(0, -1)):
    """dJ/dp for J = bragg_objective(prob) and each parameter p given by
    shifted[p](t) -> the problem with p moved by t.  Per angle: the forward
    solve; g = w a^U; the adjoint block solve A'^H mu = h, h = -X_1[P:]^H g on
    Gamma_1; Psi_j = sum B_{i,j}^H mu_i (proxy rows) and -g (Rayleigh rows of
    layer 1); Y_j = (Q'^H Q' + lam^2)^{-1} Psi_j eta_j^H; then
        dJ = 2 Re[ mu^H df - <mu eta^H, dA> + <mu (X eta)^H, dB>
                   + <Q' Y, dC'> + <(C' - Q' X) Y^H - Q' Y X^H, dQ'> ] + dw |a|^2,
    with the block derivatives by fourth-order central differences of the
    assembly (steps step[p], 2 step[p]); lam is held fixed."""
    I, P, K = prob.I, prob.params.P, prob.params.K
    rc = prob.params.lsq_rcond
    grad = {p: 0.0 for p in shifted}
    for a in range(prob.n_theta):
        th = float(prob.theta[a])
        sc = schur(prob, th)
        eta = block_thomas(sc["Ad"], sc["Al"], sc["Au"], sc["f"], I)
        X = sc["X"]
        aU = -(X[1][P:, :] @ eta[1])
        w = reflected_weights(prob, th, sc["bloch"], orders)
        g = w * aU
        h = {i: np.zeros_like(eta[i]) for i in range(1, I + 1)}
        h[1] = -(X[1][P:, :].conj().T @ g)
        mu = adjoint_block_thomas(sc["Ad"], sc["Al"], sc["Au"], h, I)
        etaL = {j: np.concatenate([eta[i] for i in layer_columns(prob, j)]) for j in range(1, I + 2)}
        asm = Assembler(prob)
        Bb = {(i, j): asm.B(i, j) for i in range(1, I + 1) for j in (i, i + 1)}
        SC, SQ, SB = {}, {}, {}
        for j in range(1, I + 2):
            Psi = np.zeros(X[j].shape[0], np.complex128)
            for i in (j - 1, j):  # interfaces whose A' uses X_j[:P] through B_{i,j}
                if 1 <= i <= I:
                    Psi[:P] += Bb[(i, j)].conj().T @ mu[i]
            if j == 1:
                Psi[P:] = -g
            Y = lsq_adjoint(sc["Qp"][j], np.outer(Psi, etaL[j].conj()), rc)
            SC[j] = sc["Qp"][j] @ Y
            SQ[j] = (sc["Cp"][j] - sc["Qp"][j] @ X[j]) @ Y.conj().T - sc["Qp"][j] @ Y @ X[j].conj().T
        for i in range(1, I + 1):
            for j in (i, i + 1):
                SB[(i, j)] = np.outer(mu[i], (X[j][:P, :] @ etaL[j]).conj())
        for p, make in shifted.items():
            t = step[p]
            Bk = {s_: _blocks(make(s_ * t), th) for s_ in (-2, -1, 1, 2)}
            d = lambda get: (-get(Bk[2]) + 8 * get(Bk[1]) - 8 * get(Bk[-1]) + get(Bk[-2])) / (12 * t)
            acc = np.vdot(mu[1], d(lambda b: b["f"]))
            for (i, j) in Bk[1]["A"]:
                acc -= np.vdot(mu[i], d(lambda b: b["A"][(i, j)]) @ eta[j])
            for key in SB:
                acc += np.vdot(SB[key], d(lambda b: b["B"][key]))
            for j in range(1, I + 2):
                acc += np.vdot(SC[j], d(lambda b: b["Cp"][j])) + np.vdot(SQ[j], d(lambda b: b["Qp"][j]))
            grad[p] += 2.0 * acc.real + float(np.sum(d(lambda b: b["w"]) * np.abs(aU) ** 2))
    return grad


def solve_streaming(prob, itheta=0):
    """solve() without holding every block at once, for stacks whose blocks
    do not fit in host memory together (the 1000-interface corner grating:
    about 25 GB of A, A' and per-copy terms).  Each quantity is formed by the
    same expression as in schur() and block_thomas(), in the order the
    forward sweep of Sec. 3.3 first needs it: X_j (Sec. 3.2) when interface
    j-1 or j is reached, A'_{i,i-1}, A'_{i,i}, A'_{i,i+1} (eqs. Schur1 -
    Schuri) at step i, then A~_i and f~_i.  Blocks are dropped once used; the
    LU factors of A~_i and A'_{i,i+1} are kept for the backward sweep.  The
    results are bitwise those of solve()."""
    theta = float(prob.theta[itheta])
    I, P = prob.I, prob.params.P
    bl = bloch(prob, theta)
    al = bl["alpha"]
    n = [2 * f.N for f in prob.ifaces]
    asm = Assembler(prob)
    X = {}

    def x_of(j):
        if j not in X:
            X[j] = lsq(asm.Qp(j, al, bl), asm.Cp(j, al), prob.params.lsq_rcond)
        return X[j]

    def xcols(j, i):
        off = 0
        for ii in layer_columns(prob, j):
            if ii == i:
                return x_of(j)[:P, off:off + n[i - 1]]
            off += n[ii - 1]
        raise KeyError

    def evict(below):
        """Drop cached per-copy terms and X blocks of interfaces and layers
        that no later step reads (all indices < below; X_1 stays for the
        amplitudes)."""
        for key in list(asm._c):
            idx = [v for v in key[1:] if isinstance(v, int)]
            if idx and max(idx) < below:
                del asm._c[key]
        for j in list(X):
            if 1 < j < below:
                del X[j]

    lu, Au, ft = {}, {}, {}
    f1 = rhs(prob, theta)
    for i in range(1, I + 1):
        Ad = asm.A(i, i, al) - asm.B(i, i) @ xcols(i, i) - asm.B(i, i + 1) @ xcols(i + 1, i)
        if i < I:
            Au[i] = asm.A(i, i + 1, al) - asm.B(i, i + 1) @ xcols(i + 1, i + 1)
        if i == 1:
            At, ft[1] = Ad, f1
        else:
            Al = asm.A(i, i - 1, al) - asm.B(i, i) @ xcols(i, i - 1)
            Y = sla.lu_solve(lu[i - 1], Au[i - 1])
            At = Ad - Al @ Y
            fi = np.zeros(n[i - 1], np.complex128)
            ft[i] = fi - Al @ sla.lu_solve(lu[i - 1], ft[i - 1])
            del Al, Y
        lu[i] = sla.lu_factor(At)
        del Ad, At
        evict(i)
    eta = {I: sla.lu_solve(lu[I], ft[I])}
    for i in range(I - 1, 0, -1):
        eta[i] = sla.lu_solve(lu[i], ft[i] - Au[i] @ eta[i + 1])
    aU = -(x_of(1)[P:, :] @ eta[1])
    aD = -(x_of(I + 1)[P:, :] @ eta[I])
    return dict(theta=theta, aU=aU, aD=aD, eta=np.concatenate([eta[i] for i in range(1, I + 1)]),
                flux=flux_error(prob, theta, bl, aU, aD), bloch=bl)


def solve_all(prob):
    asm = Assembler(prob)
    return [solve(prob, t, asm) for t in range(prob.n_theta)]


# ----------------------------------------------------------------------------
# Brute-force references for small I
# ----------------------------------------------------------------------------
def dense_reduced_system(prob, sc):
    """The block-tridiagonal A' of eq. Aschur assembled densely, with f."""
    I = prob.I
    n = [2 * f.N for f in prob.ifaces]
    off = np.concatenate([[0], np.cumsum(n)])
    A = np.zeros((off[-1], off[-1]), np.complex128)
    for i in range(1, I + 1):
        r = slice(off[i - 1], off[i])
        A[r, r] = sc["Ad"][i]
        if i < I:
            A[r, off[i]:off[i + 1]] = sc["Au"][i]
        if i > 1:
            A[r, off[i - 2]:off[i - 1]] = sc["Al"][i]
    f = np.concatenate([sc["f"][i] for i in range(1, I + 1)])
    return A, f


def full_linsys(prob, theta, asm=None):
    """The rectangular system of eq. linsys: unknowns [eta, x_1, ..., x_{I+1}],
    rows [interface rows; wall/radiation rows of layers 1..I+1]."""
    asm = asm or Assembler(prob)
    I, P = prob.I, prob.params.P
    bl = bloch(prob, theta)
    al = bl["alpha"]
    n = [2 * f.N for f in prob.ifaces]
    noff = np.concatenate([[0], np.cumsum(n)])
    Qp = {j: asm.Qp(j, al, bl) for j in range(1, I + 2)}
    Cp = {j: asm.Cp(j, al) for j in range(1, I + 2)}
    xs = [Qp[j].shape[1] for j in range(1, I + 2)]
    xoff = noff[-1] + np.concatenate([[0], np.cumsum(xs)])
    rs = [Qp[j].shape[0] for j in range(1, I + 2)]
    roff = noff[-1] + np.concatenate([[0], np.cumsum(rs)])
    A = np.zeros((roff[-1], xoff[-1]), np.complex128)
    for i in range(1, I + 1):
        r = slice(noff[i - 1], noff[i])
        A[r, r] = asm.A(i, i, al)
        if i < I:
            A[r, noff[i]:noff[i + 1]] = asm.A(i, i + 1, al)
        if i > 1:
            A[r, noff[i - 2]:noff[i - 1]] = asm.A(i, i - 1, al)
        A[r, xoff[i - 1]:xoff[i - 1] + P] = asm.B(i, i)
        A[r, xoff[i]:xoff[i] + P] = asm.B(i, i + 1)
    for j in range(1, I + 2):
        r = slice(roff[j - 1], roff[j])
        A[r, xoff[j - 1]:xoff[j]] = Qp[j]
        c0 = 0
        for ii in layer_columns(prob, j):
            A[r, noff[ii - 1]:noff[ii]] = Cp[j][:, c0:c0 + n[ii - 1]]
            c0 += n[ii - 1]
    f = np.zeros(roff[-1], np.complex128)
    f[:n[0]] = rhs(prob, theta)
    return A, f, dict(noff=noff, xoff=xoff, roff=roff)


def system_size(N_list, I, Mw, M, P, K):
    """Rows and columns of eq. linsys: rows = N_den + 2 M_w (I+1) + 4M,
    cols = N_den + P (I+1) + 2 (2K+1), N_den = 2 sum N_i (eq. Nden)."""
    nden = 2 * int(np.sum(N_list))
    return nden + 2 * Mw * (I + 1) + 4 * M, nden + P * (I + 1) + 2 * (2 * K + 1)
