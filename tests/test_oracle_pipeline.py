"""Whole-pipeline pins of the oracle: closed forms for flat layers, flux
conservation (Remark r:flux), brute-force dense solves for small I, the
system-size arithmetic of Sec. 4.2, LSQ semantics and self-convergence."""
import math

import numpy as np
import pytest
import scipy.linalg as sla

from oracle import mlqp_oracle as O
from workloads import config1, flat_stack, small_stack, wood_angle
from tests.closed_forms import flat_multilayer, fresnel


def _amps(r):
    return np.concatenate([r["aU"], r["aD"]])


def test_fresnel_single_flat_interface():
    """Config 1 with y = 0: a^U_0 = r e^{i q1 y_U}, a^D_0 = t e^{-i q2 y_D},
    every other order 0 (Fresnel; amplitude convention of eqs. RB1, RB3)."""
    for prob in (config1(flat=True), config1(flat=True, N=140, P=80, Mw=60)):
        r = O.solve(prob, 0)
        th = float(prob.theta[0])
        rr, tt, q1, q2 = fresnel(5.0, 10.0, th)
        K = prob.params.K
        aU0 = rr * np.exp(1j * q1 * O.y_upper(prob))
        aD0 = tt * np.exp(-1j * q2 * O.y_lower(prob))
        tol = 5e-10
        assert abs(r["aU"][K] - aU0) < tol
        assert abs(r["aD"][K] - aD0) < tol
        others = np.concatenate([np.delete(r["aU"], K), np.delete(r["aD"], K)])
        assert np.max(np.abs(others)) < tol
        assert abs(r["flux"]) < 1e-9


@pytest.mark.parametrize("lossy", [False, True])
def test_flat_multilayer_transfer_matrix(lossy):
    """Three flat interfaces (four layers, optionally one lossy): the block
    Schur / tridiagonal route reproduces the 1D transfer-matrix solution."""
    heights = [0.0, -1.3, -2.9]
    k = [4.0, 6.5 + (0.4j if lossy else 0), 5.2, 7.1]
    th = -1.1
    prob = flat_stack(heights, k, [th], N=80, P=70, Mw=40, K=10, M=40)
    r = O.solve(prob, 0)
    B1, Alast, q1, ql = flat_multilayer(heights, prob.k, th)
    K = prob.params.K
    assert abs(r["aU"][K] - B1 * np.exp(1j * q1 * O.y_upper(prob))) < 1e-9
    assert abs(r["aD"][K] - Alast * np.exp(-1j * ql * O.y_lower(prob))) < 1e-9
    others = np.concatenate([np.delete(r["aU"], K), np.delete(r["aD"], K)])
    assert np.max(np.abs(others)) < 1e-9
    if lossy:
        assert math.isnan(r["flux"])
        # absorption: outgoing flux strictly below the incident flux
        q1r = q1.real
        out = q1r * abs(B1) ** 2 + ql.real * abs(Alast) ** 2
        assert out < q1r


def test_flux_conservation_config1():
    """Remark r:flux: reflected + transmitted efficiencies sum to 1.  Literal
    config 1 reaches 1e-9; the resolved parameters (N = 140, P = 80,
    M_w = 60) reach 1e-11."""
    assert abs(O.solve(config1(), 0)["flux"]) < 1e-9
    assert abs(O.solve(config1(R=3 * math.pi), 0)["flux"]) < 1e-9
    assert abs(O.solve(config1(N=140, P=80, Mw=60), 0)["flux"]) < 1e-11


def test_flux_conservation_stack_and_wood_anomaly():
    """Three curved interfaces: flux to 1e-9 at a generic angle and to a few
    1e-9 when 1e-8 past a Wood anomaly of the top layer (Sec. 4.2: the flux
    error is no worse at Wood anomalies)."""
    prob = small_stack(I=3, N=80, P=60, Mw=40, K=10, M=40)
    k1 = prob.k[0].real
    thw = wood_angle(k1, prob.d, 1) + 1e-8
    p2 = prob.with_angles([-math.pi / 3, thw])
    asm = O.Assembler(p2)
    f0 = O.solve(p2, 0, asm)["flux"]
    f1 = O.solve(p2, 1, asm)["flux"]
    assert abs(f0) < 1e-9
    assert abs(f1) < 5e-9


def test_block_thomas_matches_dense_solve():
    """The forward/backward block sweep (Sec. 3.3) solves the assembled
    block-tridiagonal A' (eq. Aschur) to backward error ~1e-14 and gives the
    same Bragg amplitudes as one dense LU solve.  (A' has end blocks of
    condition ~1e9-1e12: its near-null directions come from the upgoing
    quasi-periodic waves that make the end layers' periodized Green's
    functions non-unique, so eta itself is compared through its residual.)"""
    prob = small_stack(I=3, N=80, P=60, Mw=40, K=10, M=40)
    r = O.solve(prob, 0, keep=True)
    A, f = O.dense_reduced_system(prob, r["schur"])
    eta = sla.solve(A, f)
    back = np.linalg.norm(A @ r["eta"] - f) / (np.linalg.norm(A, 2) * np.linalg.norm(r["eta"]))
    assert back < 1e-14
    n1 = 2 * prob.ifaces[0].N
    nI = 2 * prob.ifaces[-1].N
    X = r["schur"]["X"]
    P = prob.params.P
    aU = -(X[1][P:] @ eta[:n1])
    aD = -(X[prob.I + 1][P:] @ eta[-nI:])
    scale = np.max(np.abs(_amps(r)))
    assert np.max(np.abs(np.concatenate([aU, aD]) - _amps(r))) < 1e-11 * scale


def test_schur_route_matches_global_least_squares():
    """Eliminating x_j by per-layer least squares (Sec. 3.2) and solving the
    full rectangular system of eq. linsys by one global least-squares solve
    give the same Bragg amplitudes to discretisation accuracy."""
    prob = small_stack(I=2, N=64, P=50, Mw=32, K=8, M=32)
    th = float(prob.theta[0])
    r = O.solve(prob, 0)
    A, f, off = O.full_linsys(prob, th)
    x = sla.lstsq(A, f, cond=1e-13)[0]
    P = prob.params.P
    nK = 2 * prob.params.K + 1
    aU = x[off["xoff"][0] + P: off["xoff"][0] + P + nK]
    aD = x[off["xoff"][prob.I] + P: off["xoff"][prob.I] + P + nK]
    scale = np.max(np.abs(_amps(r)))
    assert np.max(np.abs(np.concatenate([aU, aD]) - _amps(r))) < 1e-8 * scale
    # shape of eq. linsys follows the size formula
    assert A.shape == O.system_size([f_.N for f_ in prob.ifaces], prob.I,
                                    prob.params.Mw, prob.params.M, P, prob.params.K)


def test_system_size_arithmetic_tables_1_2():
    """The printed sizes of the I = 1000 systems (tests/golden/
    system_sizes_tables_1_2.json, with its citation: Sec. 4.2, Tables 1-2)
    follow from the size formula of eq. linsys with the interface layout the
    fixture states."""
    import json
    import os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "system_sizes_tables_1_2.json")))
    for run in g["runs"]:
        I = run["I"]
        tri = set(range(4, I + 1, 8))
        rec = set(range(4, I + 1, 15))
        tri -= rec
        Ns = [run["N_rectangle"] if i in rec else run["N_triangle"] if i in tri else run["N_sine"]
              for i in range(1, I + 1)]
        assert O.system_size(Ns, I, run["Mw"], run["M"], run["P"], run["K"]) == (run["rows"], run["cols"])


def test_pivoted_qr_semantics():
    """Column-pivoted Householder QR: |diag R| equals LAPACK geqp3's on a
    generic matrix; full-rank LSQ matches lstsq; on a rank-deficient matrix
    the basic solution attains the minimal residual with zeros in the
    non-pivot columns."""
    rng = np.random.default_rng(5)
    A = rng.standard_normal((40, 25)) + 1j * rng.standard_normal((40, 25))
    B = rng.standard_normal((40, 7)) + 1j * rng.standard_normal((40, 7))
    _, R, piv, r = O.pivoted_qr(A, 1e-10)
    R2, P2 = sla.qr(A, mode="r", pivoting=True)
    assert r == 25
    assert np.allclose(np.abs(np.diag(R)), np.abs(np.diag(R2[0] if isinstance(R2, tuple) else R2)), rtol=1e-12)
    X = O.lsq_pivoted(A, B, 1e-10)
    assert np.allclose(X, np.linalg.lstsq(A, B, rcond=None)[0], atol=1e-12)
    # rank 10 matrix
    L = rng.standard_normal((40, 10)) + 1j * rng.standard_normal((40, 10))
    Rr = rng.standard_normal((10, 25))
    A2 = L @ Rr
    X2 = O.lsq_pivoted(A2, B, 1e-10)
    _, _, piv2, r2 = O.pivoted_qr(A2, 1e-10)
    assert r2 == 10
    assert np.all(X2[piv2[10:]] == 0)
    res_min = np.linalg.norm(B - A2 @ np.linalg.lstsq(A2, B, rcond=1e-10)[0])
    assert abs(np.linalg.norm(B - A2 @ X2) - res_min) < 1e-10 * res_min


def test_self_convergence_in_N():
    """Successive refinements of the interface quadrature converge (P3)."""
    vals = []
    for N in (60, 80, 100, 120):
        r = O.solve(config1(N=N, P=80, Mw=60), 0)
        vals.append(_amps(r))
    d1 = np.max(np.abs(vals[1] - vals[0]))
    d2 = np.max(np.abs(vals[2] - vals[1]))
    d3 = np.max(np.abs(vals[3] - vals[2]))
    assert d2 < 0.3 * d1 and d3 < 0.3 * d2 and d3 < 1e-9


def test_regularised_lsq_definition():
    """lsq() is the minimiser of ||Q X - C||^2 + lam^2 ||X||^2 with
    lam = rcond * max column norm: it satisfies the normal equations
    (Q^H Q + lam^2 I) X = Q^H C, and for a well-conditioned full-rank Q with
    rcond -> 0 it tends to the least-squares solution."""
    rng = np.random.default_rng(9)
    Q = rng.standard_normal((50, 20)) + 1j * rng.standard_normal((50, 20))
    C = rng.standard_normal((50, 6)) + 1j * rng.standard_normal((50, 6))
    rc = 1e-3
    lam = rc * np.max(np.linalg.norm(Q, axis=0))
    X = O.lsq(Q, C, rc)
    lhs = (Q.conj().T @ Q + lam ** 2 * np.eye(20)) @ X
    assert np.allclose(lhs, Q.conj().T @ C, atol=1e-11)
    X0 = O.lsq(Q, C, 1e-14)
    assert np.allclose(X0, np.linalg.lstsq(Q, C, rcond=None)[0], atol=1e-11)


def test_regularised_and_pivoted_lsq_agree_on_amplitudes():
    """The two readings of the per-layer 'backslash' (Sec. 3.2) give the same
    Bragg amplitudes to discretisation accuracy on resolved problems."""
    for prob in (config1(N=140, P=80, Mw=60), small_stack(I=3, N=80, P=60, Mw=40, K=10, M=40)):
        asm = O.Assembler(prob)
        r = O.solve(prob, 0, asm)
        orig = O.lsq
        O.lsq = O.lsq_pivoted
        try:
            rp = O.solve(prob, 0, asm)
        finally:
            O.lsq = orig
        scale = np.max(np.abs(_amps(r)))
        assert np.max(np.abs(_amps(r) - _amps(rp))) < 1e-9 * scale


def test_streaming_solve_is_the_plain_solve():
    """solve_streaming (blocks formed when the forward sweep needs them and
    dropped after) gives bitwise the amplitudes and densities of solve() on a
    smooth stack and on a corner stack with a lossy layer."""
    from workloads import corner_stack
    for prob in (small_stack(I=4, N=40, P=40, Mw=24, K=6, M=20),
                 corner_stack(I=3, levels=1, K=6, M=20, lossy=True)):
        a = O.solve(prob, 0)
        b = O.solve_streaming(prob, 0)
        assert np.array_equal(a["aU"], b["aU"]) and np.array_equal(a["aD"], b["aD"])
        assert np.array_equal(a["eta"], b["eta"])
        assert (math.isnan(a["flux"]) and math.isnan(b["flux"])) or a["flux"] == b["flux"]
