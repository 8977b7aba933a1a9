"""Pins of the oracle's corner (polyline) discretisation: graded
Gauss-Legendre panels with product integration of the log-singular kernel
parts.

- The Legendre log moments and the product-integration weights are checked
  against 30-digit adaptive quadrature (mpmath).
- A flat polyline (the same graded panels, corners of angle pi) reproduces
  the Fresnel closed form.
- The trapezoid conserves flux (Remark r:flux), with the error falling as
  the corner grading deepens.
"""
import math

import numpy as np
import pytest

from oracle import mlqp_oracle as O
from workloads import corner_stack, trapezoid
from tests.closed_forms import fresnel

mp = pytest.importorskip("mpmath")
mp.mp.dps = 30


def test_legendre_log_moments_exact():
    for t in (-0.93, -0.2, 0.41, 0.999):
        L = O.legendre_log_moments(t, 15)
        ref = [float(mp.quad(lambda s: mp.legendre(n, s) * mp.log(abs(s - t)), [-1, t, 1])) for n in range(16)]
        assert np.max(np.abs(L - np.array(ref))) < 1e-14


def _f(s):  # a smooth density sample, with its mpmath twin
    return np.exp(0.7 * s) * np.cos(2.0 * s)


def _fm(s):
    return mp.exp(0.7 * s) * mp.cos(2 * s)


def test_own_panel_weights_integrate_log_singularity():
    g, w = np.polynomial.legendre.leggauss(16)
    half = 0.037
    for j in (0, 5, 15):
        t = g[j]
        W = O.own_panel_log_weights(t, half, g, w)
        ref = half * mp.quad(lambda s: _fm(s) * mp.log(half * abs(s - t)), [-1, t, 1])
        assert abs(W @ _f(g) - float(ref)) < 1e-13 * max(1.0, abs(float(ref)))


@pytest.mark.parametrize("target", [(1.0021, 0.0), (0.97, 0.013), (1.003, 0.05), (0.2, 0.5)])
def test_near_panel_weights_against_adaptive_quadrature(target):
    """Panel from (-1, 0) to (1, 0) scaled by 0.05; targets just beyond its
    end on the same line, above it, across a corner, and further away."""
    sc = 0.05
    xa, ya, xb, yb = -sc, 0.0, sc, 0.0
    px, py = target[0] * sc, target[1] * sc
    g, w = np.polynomial.legendre.leggauss(16)
    W = O.near_panel_log_weights(px, py, xa, ya, xb, yb, g, w)
    ref = sc * mp.quad(lambda s: _fm(s) * mp.log(mp.sqrt((px - sc * s) ** 2 + py ** 2)), [-1, 0, 1])
    assert abs(W @ _f(g) - float(ref)) < 1e-12 * max(1.0, abs(float(ref)))


def test_panel_geometry():
    L = 3
    f = trapezoid(-1.0, L)
    P = O.polyline_panels(f, 1.0)
    assert len(P.h) == 2 * len(f.vx) * L
    assert P.nodes.x.size == f.N
    xs, ys = O.polyline_breaks(f, 1.0)
    perim = np.sum(np.hypot(np.diff(xs), np.diff(ys)))
    assert abs(np.sum(P.h) - perim) < 1e-14
    assert abs(np.sum(P.nodes.w) - perim) < 1e-13
    assert np.allclose(np.hypot(P.nodes.nx, P.nodes.ny), 1.0)
    assert np.all(P.nodes.ny <= 0)  # normals point down, into the layer below
    # dyadic grading toward every corner: on each side the panel touching the
    # corner and its neighbour have size l/2^(L-1), the next ones double
    ends = np.concatenate([[P.xa[0]], P.xb])
    for c in f.vx:
        q = np.argmin(np.abs(ends - c))
        assert abs(ends[q] - c) < 1e-15
        left, right = P.h[q - 3:q][::-1], P.h[q:q + 3]
        for side in (left, right):
            assert abs(side[0] - side[1]) < 1e-14 and abs(side[2] - 2 * side[1]) < 1e-14


def test_flat_polyline_matches_fresnel():
    p = corner_stack(I=1, levels=2, flat=True, kvals=(5.0, 10.0), theta=-math.pi / 5, K=10, M=30)
    p.ifaces[0] = trapezoid(0.0, 2, height=0.0)
    r = O.solve(p, 0)
    rr, tt, q1, q2 = fresnel(5.0, 10.0, -math.pi / 5)
    K = p.params.K
    assert abs(r["aU"][K] - rr * np.exp(1j * q1 * O.y_upper(p))) < 1e-10
    assert abs(r["aD"][K] - tt * np.exp(-1j * q2 * O.y_lower(p))) < 1e-10
    assert abs(r["flux"]) < 1e-10


def test_trapezoid_flux_falls_with_corner_grading():
    flux = []
    for L in (2, 4):
        p = corner_stack(I=1, levels=L, kvals=(10.0, 20.0), theta=-math.pi / 4, K=12, M=30)
        flux.append(abs(O.solve(p, 0)["flux"]))
    assert flux[0] < 2e-6 and flux[1] < 1e-7
    assert flux[1] < flux[0] / 8  # about 4x per level of grading
