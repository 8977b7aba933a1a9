"""Closed-form references used to pin the oracle (independent of its code).

* Planar multilayer: the 1D problem of plane-wave scattering by flat layers
  (the transfer / scattering-matrix setting the paper contrasts with its
  method, Sec. 1).  In layer j the total field is
      u_j = A_j exp(i kappa x - i q_j (y - h)) + B_j exp(i kappa x + i q_j (y - h))
  with q_j = sqrt(k_j^2 - kappa^2) (Im >= 0); u and du/dy are continuous at
  every interface y = h_i.  A_1 = 1 (incident), B_{I+1} = 0 (radiation).
  For one interface this is Fresnel's r = (q1-q2)/(q1+q2), t = 2 q1/(q1+q2).
"""
import cmath
import math

import numpy as np


def _q(k, kappa):
    w = cmath.sqrt(complex(k) ** 2 - kappa ** 2)
    return -w if w.imag < 0 else w


def fresnel(k1, k2, theta):
    kappa = k1 * math.cos(theta)
    q1, q2 = _q(k1, kappa), _q(k2, kappa)
    return (q1 - q2) / (q1 + q2), 2 * q1 / (q1 + q2), q1, q2


def flat_multilayer(heights, k, theta):
    """Reflection coefficient B_1 and transmission A_{I+1} of the planar stack
    (fields referenced to y = 0: u_1 = e^{-i q1 y} + B_1 e^{i q1 y},
    u_{I+1} = A_{I+1} e^{-i q_{I+1} y}).  Returns (B1, A_last, q_first, q_last)."""
    I = len(heights)
    k1 = float(np.real(k[0]))
    kappa = k1 * math.cos(theta)
    q = [_q(kk, kappa) for kk in k]
    # unknowns: B_1, (A_j, B_j) j=2..I, A_{I+1}  -> 2I unknowns
    n = 2 * I
    M = np.zeros((n, n), complex)
    rhs = np.zeros(n, complex)

    def col(j, which):
        # column index of A_j ('A') or B_j ('B'), j 1-based
        if j == 1:
            assert which == "B"
            return 0
        if j == I + 1:
            assert which == "A"
            return n - 1
        return 1 + 2 * (j - 2) + (0 if which == "A" else 1)

    for i in range(1, I + 1):
        h = heights[i - 1]
        r0, r1 = 2 * (i - 1), 2 * (i - 1) + 1
        # layer i (above) minus layer i+1 (below): value and y-derivative
        for j, sgn in ((i, 1.0), (i + 1, -1.0)):
            ea, eb = cmath.exp(-1j * q[j - 1] * h), cmath.exp(1j * q[j - 1] * h)
            if j == 1:
                rhs[r0] -= sgn * ea
                rhs[r1] -= sgn * (-1j * q[0]) * ea
            else:
                M[r0, col(j, "A")] += sgn * ea
                M[r1, col(j, "A")] += sgn * (-1j * q[j - 1]) * ea
            if j != I + 1:
                M[r0, col(j, "B")] += sgn * eb
                M[r1, col(j, "B")] += sgn * (1j * q[j - 1]) * eb
    x = np.linalg.solve(M, rhs)
    return x[0], x[-1], q[0], q[-1]
