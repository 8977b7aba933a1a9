"""Pins of the oracle's kernel formulas, log-split and quadrature pieces against
mathematics that does not go through the oracle's own formulas:
finite differences of G, the integral identity behind Kress' weights,
Richardson extrapolation of the smooth remainder, and adaptive quadrature of
the three-copy layer potentials."""
import math

import numpy as np
import pytest
from scipy import integrate
from scipy.special import hankel1

from oracle import mlqp_oracle as O
from workloads import config1, small_stack

RNG = np.random.default_rng(1234)


def G(k, x, y, sx, sy):
    return 0.25j * hankel1(0, k * np.hypot(x - sx, y - sy))


@pytest.mark.parametrize("k", [5.0, 17.3, 12.0 + 0.5j])
def test_kernel_derivatives_match_finite_differences(k):
    """D = dG/dn', Ds = dG/dn, T = d2G/dn dn' (Sec. 2.2) against 5-point
    central differences of G = (i/4) H0(k r) (eq. Gi) along the normals."""
    h = 1e-3
    c = np.array([1.0, -8.0, 8.0, -1.0]) / (12 * h)
    offs = np.array([-2, -1, 1, 2]) * h
    for _ in range(6):
        tx, ty, sx, sy = RNG.uniform(-1, 1, 4)
        a, b = RNG.uniform(0, 2 * math.pi, 2)
        tn = (math.cos(a), math.sin(a))
        sn = (math.cos(b), math.sin(b))
        g = O.green_kernels(k, tx, ty, tn[0], tn[1], sx, sy, sn[0], sn[1])
        d_src = sum(ci * G(k, tx, ty, sx + o * sn[0], sy + o * sn[1]) for ci, o in zip(c, offs))
        d_tgt = sum(ci * G(k, tx + o * tn[0], ty + o * tn[1], sx, sy) for ci, o in zip(c, offs))
        d2 = sum(ci * sum(cj * G(k, tx + oi * tn[0], ty + oi * tn[1], sx + oj * sn[0], sy + oj * sn[1])
                          for cj, oj in zip(c, offs)) for ci, oi in zip(c, offs))
        scale = abs(g["S"]) + 1
        assert abs(g["S"] - G(k, tx, ty, sx, sy)) < 1e-15 * scale
        assert abs(g["D"] - d_src) < 1e-8 * (abs(k) ** 1 + 1) * scale
        assert abs(g["Ds"] - d_tgt) < 1e-8 * (abs(k) ** 1 + 1) * scale
        assert abs(g["T"] - d2) < 1e-6 * (abs(k) ** 2 + 1) * scale


def test_kress_weight_moments():
    """sum_q R_q e^{i m s_q} = -(2 pi/|m|) for 0 < |m| < n and 0 for m = 0: the
    rule integrates log(4 sin^2(s/2)) e^{ims} exactly on trigonometric
    polynomials (int_0^{2pi} log(4 sin^2(s/2)) e^{ims} ds = -2pi/|m|)."""
    for N in (16, 64, 120):
        R = O.kress_weights(N)
        s = 2 * math.pi * np.arange(N) / N
        n = N // 2
        for m in range(-(n - 1), n):
            val = np.sum(R * np.exp(1j * m * s))
            exact = 0.0 if m == 0 else -2 * math.pi / abs(m)
            assert abs(val - exact) < 1e-12, (N, m, val)
    # the identity itself, by adaptive quadrature, for one m
    f = lambda s: math.log(4 * math.sin(s / 2) ** 2) * math.cos(3 * s)
    v, _ = integrate.quad(f, 0, 2 * math.pi, points=[0.0, 2 * math.pi], limit=200)
    assert abs(v + 2 * math.pi / 3) < 1e-9


def test_cutoff_window():
    a, b = 0.4, 2.5
    d = np.linspace(-3.2, 3.2, 2001)
    chi = O.cutoff(d, a, b)
    assert np.all(chi[np.abs(d) <= a] == 1.0)
    assert np.all(chi[np.abs(d) >= b] == 0.0)
    assert np.all(np.diff(chi[d >= 0]) <= 1e-15)       # non-increasing in |d|
    assert np.allclose(chi, chi[::-1])                  # even
    # psi(u) + psi(1-u) = 1 (symmetric transition)
    u = np.linspace(0.01, 0.99, 50)
    x = b - u * (b - a)
    assert np.allclose(O.cutoff(x, a, b) + O.cutoff(b - (1 - u) * (b - a), a, b), 1.0)


def test_vertical_wavenumber_branch():
    kap = np.array([0.0, 3.0, 5.0 - 1e-9, 7.0, -9.0])
    w = O.vertical_wavenumber(5.0, kap)
    assert np.all(w.imag >= 0)
    assert w[0] == 5.0 and abs(w[1] - 4.0) < 1e-15
    assert abs(w[3] - 1j * math.sqrt(24)) < 1e-14
    wc = O.vertical_wavenumber(12 + 0.5j, kap)
    assert np.all(wc.imag > 0)
    assert np.allclose(wc ** 2, (12 + 0.5j) ** 2 - kap ** 2)


@pytest.mark.parametrize("kk", [(5.0, 10.0), (9.3, 12.0 + 0.5j)])
def test_diagonal_limits_by_richardson(kk):
    """K2 = K - K1 log(4 sin^2((t-s)/2)) is smooth; its value at s = t
    (series limits) matches polynomial extrapolation of off-diagonal K2."""
    k1, k2 = kk
    prob = config1()
    nd = O.interface_nodes(prob.ifaces[0], prob.d)
    m = 17
    t = nd.s[m]
    d = prob.d
    m_arr = np.arange(1, len(prob.ifaces[0].a) + 1)
    f = prob.ifaces[0]

    def Z(s):
        x = -d / 2 + s * d / (2 * math.pi)
        ph = 2 * math.pi * m_arr * x / d
        y = f.y0 + np.cos(ph) @ f.a + np.sin(ph) @ f.b
        fp = (np.sin(ph) * (-2 * math.pi * m_arr / d)) @ f.a + (np.cos(ph) * (2 * math.pi * m_arr / d)) @ f.b
        hh = math.sqrt(1 + fp * fp)
        return x, y, fp / hh, -1 / hh, d / (2 * math.pi) * hh

    tx, ty, tnx, tny, _ = Z(t)
    hs = np.array([1, 2, 3, 4, 5, 6]) * 2e-3
    vals = {key: [] for key in ("S", "D", "Ds", "T")}
    for h in hs:
        sx, sy, snx, sny, sp = Z(t + h)
        g1 = O.green_kernels(k1, tx, ty, tnx, tny, sx, sy, snx, sny, log_parts=True)
        g2 = O.green_kernels(k2, tx, ty, tnx, tny, sx, sy, snx, sny, log_parts=True)
        lg = math.log(4 * math.sin(h / 2) ** 2)
        for key in vals:
            K = (g1[key] - g2[key]) * sp
            K1 = (g1["K1" + key] - g2["K1" + key]) * sp
            vals[key].append(K - K1 * lg)
    lim = O.self_diag_limits(k1, k2, nd.speed[m])
    for key in vals:
        v = np.array(vals[key])
        # K2 is smooth in h: fit a polynomial in h and evaluate at 0
        cr = np.polyfit(hs, v.real, 5)[-1]
        ci = np.polyfit(hs, v.imag, 5)[-1]
        ext = cr + 1j * ci
        assert abs(ext - lim[key + "2"]) < 1e-7 * (1 + abs(lim[key + "2"])), (key, ext, lim[key + "2"])


def _bump_density(prob, kappa0, s, t0):
    """Quasi-periodic density e^{i kappa0 x(s)} beta(s) whose periodic factor
    beta is a narrow bump around t0, negligible (< 1e-13) at the seam s = 0,
    so the unwrapped three-copy density vanishes at the dangling ends."""
    d = prob.d
    x = -d / 2 + s * d / (2 * math.pi)
    return np.exp(1j * kappa0 * x) * np.exp(-20 * (1 - np.cos(s - t0))) * (1 + 0.3 * np.sin(s))


@pytest.mark.parametrize("block", ["S", "D", "Ds", "T"])
def test_self_block_applies_three_copy_operator(block):
    """Rows of A_{1,1} (eq. Ablocks) times a quasi-periodic density equal the
    three-copy, Bloch-phased layer potentials (eqs. SDopsum, DtTopsum) of the
    kernel differences plus the jump terms -tau, +sigma, computed by adaptive
    quadrature with the singularity at s = t given to the integrator.  This
    pins the periodic log-split (Kress weights, cut-off window, diagonal
    limits, alpha phases).  The density vanishes at the ends of the unwrapped
    interval: there the plain rule is not accurate by design (the dangling
    ends are absorbed by the proxies, Sec. 2.5)."""
    prob = config1(N=120)
    d = prob.d
    th = float(prob.theta[0])
    k1, k2 = prob.k[0], prob.k[1]
    bl = O.bloch(prob, th)
    al = bl["alpha"]
    kappa0 = prob.k[0].real * math.cos(th)
    nd = O.interface_nodes(prob.ifaces[0], d)
    N = len(nd.x)
    A = O.assemble(O.self_block_terms(prob, 1), al)
    rows = {"D": (slice(0, N), slice(0, N)), "S": (slice(0, N), slice(N, 2 * N)),
            "T": (slice(N, 2 * N), slice(0, N)), "Ds": (slice(N, 2 * N), slice(N, 2 * N))}[block]
    Ablk = A[rows]
    ident = {"D": -1.0, "Ds": 1.0, "S": 0.0, "T": 0.0}[block]
    f = prob.ifaces[0]
    m_arr = np.arange(1, len(f.a) + 1)

    def Z(s):
        x = -d / 2 + s * d / (2 * math.pi)
        ph = 2 * math.pi * m_arr * x / d
        y = f.y0 + np.cos(ph) @ f.a + np.sin(ph) @ f.b
        fp = (np.sin(ph) * (-2 * math.pi * m_arr / d)) @ f.a + (np.cos(ph) * (2 * math.pi * m_arr / d)) @ f.b
        hh = math.sqrt(1 + fp * fp)
        return x, y, fp / hh, -1 / hh, d / (2 * math.pi) * hh

    for m in (40, 55, 60, 71, 80):
        t = nd.s[m]
        t0 = t + 0.05 * (m % 3 - 1)
        sig = _bump_density(prob, kappa0, nd.s, t0)
        tx, ty, tnx, tny, _ = Z(t)
        total = 0
        for l in (-1, 0, 1):
            def integrand(s, part):
                sx, sy, snx, sny, sp = Z(s)
                g1 = O.green_kernels(k1, tx, ty, tnx, tny, sx + l * d, sy, snx, sny)[block]
                g2 = O.green_kernels(k2, tx, ty, tnx, tny, sx + l * d, sy, snx, sny)[block]
                v = (g1 - g2) * sp * _bump_density(prob, kappa0, np.array([s]), t0)[0]
                return v.real if part == 0 else v.imag
            pts = [t] if l == 0 else None
            vr, _ = integrate.quad(integrand, 0, 2 * math.pi, args=(0,), points=pts, limit=400, epsabs=1e-14, epsrel=1e-13)
            vi, _ = integrate.quad(integrand, 0, 2 * math.pi, args=(1,), points=pts, limit=400, epsabs=1e-14, epsrel=1e-13)
            total += al ** l * (vr + 1j * vi)
        total += ident * sig[m]
        nys = Ablk[m] @ sig
        assert abs(nys - total) < 1e-10 * max(1.0, abs(total)), (block, m, nys, total)


def test_gauss_legendre_wall_nodes():
    prob = small_stack(I=2)
    for j in (1, 2, 3):
        x, y = O.wall_nodes(prob, j)
        bot, top = O.wall_extent(prob, j)
        assert np.all(x == -prob.d / 2)
        assert bot < y.min() and y.max() < top
        assert np.all(np.diff(y) > 0)
