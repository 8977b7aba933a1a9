"""Problem descriptions (geometry, wavenumbers, angles, sizes) and the seeded
recipes for the synthetic gratings used by tests and benchmarks.

Conventions (the problem statement of Cho & Barnett, Sec. 1):
  * I interfaces Gamma_1..Gamma_I separate I+1 layers; layer i lies above
    Gamma_i and below Gamma_{i-1}; layer 1 and layer I+1 are semi-infinite.
  * Every interface is one period, x in [-d/2, d/2), of a d-periodic graph
        y(x) = y0 + sum_{m=1}^{n_modes} a_m cos(2 pi m x / d) + b_m sin(2 pi m x / d).
  * k[i-1] is the (complex, Im >= 0) wavenumber of layer i; k[0] must be real.
  * theta are incidence angles in (-pi, 0).

Nothing in this module evaluates the method: the oracle and the CUDA library
both consume these plain records.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace
from typing import List, Optional, Union

import numpy as np

SEED_BASE = 14105003


@dataclass
class Interface:
    """One d-periodic Fourier interface y(x) = y0 + sum a_m cos + b_m sin."""
    y0: float
    a: np.ndarray
    b: np.ndarray
    N: int  # quadrature nodes (even: the periodic log-split rule uses N = 2n)

    def __post_init__(self):
        self.a = np.asarray(self.a, dtype=np.float64).ravel()
        self.b = np.asarray(self.b, dtype=np.float64).ravel()
        if self.a.shape != self.b.shape:
            raise ValueError("a and b must have the same length")


@dataclass
class PolyInterface:
    """One d-periodic polyline interface: from (-d/2, y0) through the corners
    (vx[c], vy[c]) (vx increasing inside (-d/2, d/2)) to (d/2, y0).  It is
    discretised by Gauss-Legendre panels of `order` nodes, `levels` panels on
    each side of every corner, graded dyadically toward the corner."""
    y0: float
    vx: np.ndarray
    vy: np.ndarray
    levels: int = 2
    order: int = 16

    def __post_init__(self):
        self.vx = np.asarray(self.vx, dtype=np.float64).ravel()
        self.vy = np.asarray(self.vy, dtype=np.float64).ravel()
        if self.vx.shape != self.vy.shape or len(self.vx) == 0:
            raise ValueError("vx and vy must be non-empty and of equal length")

    @property
    def N(self) -> int:
        return 2 * len(self.vx) * self.levels * self.order


@dataclass
class Params:
    """Discretisation sizes of the periodizing scheme.

    P      proxy points per layer           M_w  Gauss-Legendre nodes per wall
    R      proxy circle radius              M    trapezoid nodes on U and on D
    K      Rayleigh-Bloch orders -K..K      gap_U / gap_D  clearance of U above
                                            max Gamma_1 / of D below min Gamma_I
    cut_a, cut_b  the smooth window of the periodic log-split: 1 for |t-s|<=a,
                  0 for |t-s| >= b (parameter units, 0 <= a < b <= pi)
    lsq_rcond     regularisation of the per-layer least-squares solves,
                  relative to the largest column norm of Q'_j
    """
    P: int = 60
    R: float = 1.5 * 2 * math.pi
    Mw: int = 40
    M: int = 60
    K: int = 20
    gap_U: float = 0.15 * 2 * math.pi
    gap_D: float = 0.15 * 2 * math.pi
    cut_a: float = 0.0
    cut_b: float = math.pi
    lsq_rcond: float = 1e-10


@dataclass
class Problem:
    d: float
    k: np.ndarray            # complex, length I+1
    theta: np.ndarray        # float, n_theta angles in (-pi, 0)
    ifaces: List[Union[Interface, PolyInterface]]
    params: Params
    name: str = ""

    def __post_init__(self):
        self.k = np.asarray(self.k, dtype=np.complex128).ravel()
        self.theta = np.atleast_1d(np.asarray(self.theta, dtype=np.float64))
        if len(self.k) != len(self.ifaces) + 1:
            raise ValueError("need I+1 wavenumbers for I interfaces")

    @property
    def I(self) -> int:
        return len(self.ifaces)

    @property
    def n_theta(self) -> int:
        return len(self.theta)

    def with_angles(self, theta) -> "Problem":
        return replace(self, theta=np.atleast_1d(np.asarray(theta, float)))


def wood_angle(k1: float, d: float, order: int = 1) -> float:
    """Incidence angle in (-pi, 0) at which Rayleigh order `order` of the
    upper layer grazes (kappa_order = k1): cos(theta) = 1 - 2 pi order/(d k1).
    Used only to place test angles (Sec. 1 definition of a Wood anomaly)."""
    c = 1.0 - 2.0 * math.pi * order / (d * k1)
    return -math.acos(c)


def _random_fourier(rng, n_modes, scale=0.05):
    m = np.arange(1, n_modes + 1)
    a = rng.normal(0.0, scale / m)
    b = rng.normal(0.0, scale / m)
    return a, b


def config1(flat: bool = False, R: Optional[float] = None, N: int = 100,
            P: int = 60, Mw: int = 40, K: int = 20, M: int = 60) -> Problem:
    """Single interface y = 0.5 sin x (or y = 0), period 2 pi, k = (5, 10),
    theta = -pi/5; 100 Kress nodes, 40 wall nodes, 60 proxies on a circle of
    radius 1.5 pi, K = 20."""
    d = 2 * math.pi
    b = np.array([0.0 if flat else 0.5])
    iface = Interface(0.0, np.zeros(1), b, N)
    p = Params(P=P, R=1.5 * math.pi if R is None else R, Mw=Mw, M=M, K=K,
               gap_U=0.15 * d, gap_D=0.15 * d)
    return Problem(d, [5.0, 10.0], [-math.pi / 5], [iface], p,
                   name="config1-flat" if flat else "config1")


def config2(N: int = 120, P: int = 60, Mw: int = 30, K: int = 25, M: int = 60,
            R: Optional[float] = None, I: int = 20) -> Problem:
    """I = 20 random 5-mode Fourier interfaces 1.5 apart, period 2 pi, layer
    wavenumbers U[5, 20] except a lossy layer 11 with k = 12 + 0.5i; three
    angles: one 1e-8 past the first Wood anomaly of layer 1, -pi/5, -pi/3."""
    rng = np.random.default_rng(SEED_BASE + 2)
    d = 2 * math.pi
    ifaces = []
    for i in range(1, I + 1):
        a, b = _random_fourier(rng, 5)
        ifaces.append(Interface(-1.5 * i, a, b, N))
    k = rng.uniform(5.0, 20.0, size=I + 1).astype(np.complex128)
    if I + 1 >= 11:
        k[10] = 12.0 + 0.5j
    th_w = wood_angle(float(k[0].real), d, 1) + 1e-8
    p = Params(P=P, R=1.5 * d if R is None else R, Mw=Mw, M=M, K=K,
               gap_U=0.15 * d, gap_D=0.15 * d)
    return Problem(d, k, [th_w, -math.pi / 5, -math.pi / 3], ifaces, p,
                   name="config2")


def trapezoid(y0: float, levels: int = 2, order: int = 16, height: float = 0.4,
              x_outer: float = 0.3, x_inner: float = 0.1) -> PolyInterface:
    """Trapezoidal profile of a unit-period corner grating: flat at y0 for
    |x| >= x_outer, flat top y0 + height for |x| <= x_inner, straight flanks."""
    return PolyInterface(y0, [-x_outer, -x_inner, x_inner, x_outer],
                         [y0, y0 + height, y0 + height, y0], levels, order)


def config3(I: int = 1000, levels: int = 2, P: int = 60, Mw: int = 30, K: int = 20,
            M: int = 60, theta: float = -math.pi / 4) -> Problem:
    """Paper-scale corner stack: I trapezoidal interfaces 1 apart (d = 1,
    height 0.4, corners at x = +-0.3, +-0.1), graded Gauss-Legendre panels;
    k_i alternating 10 and 20 with a uniform +-5 % jitter; one angle."""
    rng = np.random.default_rng(SEED_BASE + 3)
    d = 1.0
    ifaces = [trapezoid(-1.0 * i, levels) for i in range(1, I + 1)]
    base = np.where(np.arange(I + 1) % 2 == 0, 10.0, 20.0)
    k = (base * (1.0 + rng.uniform(-0.05, 0.05, size=I + 1))).astype(np.complex128)
    p = Params(P=P, R=1.5 * d, Mw=Mw, M=M, K=K, gap_U=0.15 * d, gap_D=0.15 * d)
    return Problem(d, k, [theta], ifaces, p, name="config3")


def corner_stack(I: int = 2, levels: int = 2, P: int = 60, Mw: int = 30, K: int = 12,
                 M: int = 30, kvals=(10.0, 20.0), theta: float = -math.pi / 4,
                 lossy: bool = False, flat: bool = False) -> Problem:
    """A few interfaces of the corner grating (d = 1), small enough for the
    oracle; `flat` replaces the trapezoids by flat polylines with the same
    panels (corners of angle pi), `lossy` gives the middle layer Im k = 0.5."""
    d = 1.0
    ifaces = []
    for i in range(1, I + 1):
        t = trapezoid(-1.0 * i, levels, height=0.0 if flat else 0.4)
        ifaces.append(t)
    k = np.array([kvals[j % 2] for j in range(I + 1)], dtype=np.complex128)
    if lossy and I >= 2:
        k[1] += 0.5j
    p = Params(P=P, R=1.5 * d, Mw=Mw, M=M, K=K, gap_U=0.15 * d, gap_D=0.15 * d)
    return Problem(d, k, [theta], ifaces, p, name="corner_stack")


def config4(I: int = 100, n_angles: int = 256, P: int = 60, Mw: int = 30,
            K: int = 25, M: int = 60, resolved: bool = False) -> Problem:
    """Angle sweep: I = 100 random Fourier interfaces (as config 2) with node
    counts drawn from {80, 120, 160, 240, 320}, k_i ~ U[5, 20] (all real),
    256 angles uniform in [-pi + 0.1, -0.1].

    resolved=True keeps every draw (profiles, wavenumbers, angles) and raises
    the discretisation to where a 3-interface window of the stack conserves
    flux to 1e-10 at every angle: node counts doubled (at most 512, so
    {160, 240, 320, 480, 512}), P = 100 proxies, 50 wall nodes, K = 40
    orders (near grazing incidence, kappa_0 = k_1 cos theta is close to
    +-k_1, and the bottom layer propagates orders up to |n| = k_1 + k_101
    ~ 29 with d = 2 pi), M = 90 nodes on U and D."""
    if resolved:
        P, Mw, K, M = 100, 50, 40, 90
    rng = np.random.default_rng(SEED_BASE + 4)
    d = 2 * math.pi
    ifaces = []
    for i in range(1, I + 1):
        a, b = _random_fourier(rng, 5)
        N = int(rng.choice([80, 120, 160, 240, 320]))
        if resolved:
            N = min(512, 2 * N)
        ifaces.append(Interface(-1.5 * i, a, b, N))
    k = rng.uniform(5.0, 20.0, size=I + 1)
    th = np.linspace(-math.pi + 0.1, -0.1, n_angles)
    p = Params(P=P, R=1.5 * d, Mw=Mw, M=M, K=K, gap_U=0.15 * d, gap_D=0.15 * d)
    return Problem(d, k, th, ifaces, p, name="config4-resolved" if resolved else "config4")


def config5(I: int = 50, n_angles: int = 16, N: int = 120, P: int = 60,
            Mw: int = 30, K: int = 25, M: int = 60) -> Problem:
    """Design-gradient stack: I = 50 interfaces with 4 Fourier modes each,
    k_i ~ U[5, 15], 16 angles in [-pi + 0.3, -0.3] nudged off Wood anomalies."""
    rng = np.random.default_rng(SEED_BASE + 5)
    d = 2 * math.pi
    ifaces = []
    for i in range(1, I + 1):
        a, b = _random_fourier(rng, 4)
        ifaces.append(Interface(-1.5 * i, a, b, N))
    k = rng.uniform(5.0, 15.0, size=I + 1)
    th = np.linspace(-math.pi + 0.3, -0.3, n_angles)
    k1 = float(k[0])
    # nudge any angle within 1e-3 of an upper-layer grazing order
    orders = 2 * math.pi * np.arange(-40, 41) / d
    for it in range(len(th)):
        kap = k1 * math.cos(th[it]) + orders
        if np.min(np.abs(np.abs(kap) - k1)) < 1e-3 * k1:
            th[it] += 1e-3
    p = Params(P=P, R=1.5 * d, Mw=Mw, M=M, K=K, gap_U=0.15 * d, gap_D=0.15 * d)
    return Problem(d, k, th, ifaces, p, name="config5")


def flat_stack(heights, k, theta, N=60, d=2 * math.pi, P=60, Mw=40, K=10,
               M=40, R=None) -> Problem:
    """Planar multilayer (all Fourier coefficients zero) at the given heights;
    the transfer-matrix closed form applies to it."""
    ifaces = [Interface(h, np.zeros(1), np.zeros(1), N) for h in heights]
    p = Params(P=P, R=1.5 * d if R is None else R, Mw=Mw, M=M, K=K,
               gap_U=0.15 * d, gap_D=0.15 * d)
    return Problem(d, k, theta, ifaces, p, name="flat")


def small_stack(I=3, N=64, P=50, Mw=30, K=10, M=40, seed=7, kmin=3.0,
                kmax=6.0, lossy=False, n_angles=1, d=2 * math.pi, amp=0.05,
                spacing=1.5, R=None) -> Problem:
    """A few gently curved random Fourier interfaces at modest wavenumbers:
    the size the oracle solves in about a second."""
    rng = np.random.default_rng(SEED_BASE + 1000 + seed)
    ifaces = []
    for i in range(1, I + 1):
        a, b = _random_fourier(rng, 3, amp)
        ifaces.append(Interface(-spacing * i, a, b, N))
    k = rng.uniform(kmin, kmax, size=I + 1).astype(np.complex128)
    if lossy and I >= 2:
        k[I // 2 + 1] += 0.3j
    th = np.linspace(-0.7 * math.pi, -0.3 * math.pi, n_angles) if n_angles > 1 \
        else np.array([-math.pi / 3])
    p = Params(P=P, R=1.5 * d if R is None else R, Mw=Mw, M=M, K=K,
               gap_U=0.15 * d, gap_D=0.15 * d)
    return Problem(d, k, th, ifaces, p, name=f"small{I}")


CONFIGS = {"config1": config1, "config2": config2, "config3": config3, "config4": config4,
           "config5": config5}
