"""Pins of the oracle's adjoint block solve (the transposed system
A'^H mu = h of Sec. 3.3's reduced block-tridiagonal system):
- brute force: mu solves the dense conjugate-transposed system;
- duality: with h = -X_1[P:]^H e_n on Gamma_1, mu^H f = h^H eta is the upper
  Bragg amplitude a^U_n of the oracle's own solve (the identity the GPU
  adjoint is tested by), to 1e-8 of the largest amplitude (the end-layer
  near-null space of A' limits the adjoint route, see the test).  A random h is not used for duality: it excites
  the near-null directions of the end blocks (condition 1e8 and more), where
  mu is large and the identity holds only to kappa * eps; the Bragg rows do
  not radiate into those directions.
"""
import numpy as np

from oracle import mlqp_oracle as O
from tests.adjoint_forms import forms_gradient
from workloads import small_stack


def _setup(I):
    p = small_stack(I=I, N=40, P=40, Mw=24, K=8, M=30, lossy=(I == 3))
    sc = O.schur(p, float(p.theta[0]))
    eta = O.block_thomas(sc["Ad"], sc["Al"], sc["Au"], sc["f"], p.I)
    return p, sc, eta


def _flat(d, I):
    return np.concatenate([d[i] for i in range(1, I + 1)])


def test_adjoint_solves_the_dense_transposed_system():
    for I in (1, 2, 3):
        p, sc, _ = _setup(I)
        A, f = O.dense_reduced_system(p, sc)
        rng = np.random.default_rng(5 + I)
        n = [2 * q.N for q in p.ifaces]
        h = {i: rng.standard_normal(n[i - 1]) + 1j * rng.standard_normal(n[i - 1]) for i in range(1, I + 1)}
        mu = _flat(O.adjoint_block_thomas(sc["Ad"], sc["Al"], sc["Au"], h, I), I)
        hv = _flat(h, I)
        r = A.conj().T @ mu - hv
        assert np.linalg.norm(r) / (np.linalg.norm(A, 2) * np.linalg.norm(mu) + np.linalg.norm(hv)) < 1e-14
        # against a dense solve, where the system is well enough conditioned to compare elementwise
        if np.linalg.cond(A) < 1e8:
            ref = np.linalg.solve(A.conj().T, hv)
            assert np.max(np.abs(mu - ref)) / np.max(np.abs(ref)) < 1e-8


def test_adjoint_gives_the_bragg_amplitudes():
    for I in (2, 3):
        p, sc, eta = _setup(I)
        P = p.params.P
        f = _flat(sc["f"], I)
        ev = _flat(eta, I)
        aU, _ = O.recover_amplitudes(p, sc["X"], eta)
        n1 = 2 * p.ifaces[0].N
        nd = ev.size
        offs = np.concatenate([[0], np.cumsum([2 * q.N for q in p.ifaces])])
        split = lambda v: {i: v[offs[i - 1]:offs[i]] for i in range(1, I + 1)}
        # A' has a near-null direction at the end layers (condition 1e12 to
        # 1e15 here) that does not radiate: the forward route's amplitudes do
        # not see it, but mu picks up a large multiple of the left null
        # vector u, and u^H f vanishes only to rounding.  The two routes agree
        # to a few 1e-9 of the largest amplitude on these stacks; a wrong
        # transpose, conjugation or pivot order is off by O(1).
        tol = 1e-8
        for order in (0, p.params.K, 2 * p.params.K):
            h = np.zeros(nd, np.complex128)
            h[:n1] = -np.conj(sc["X"][1][P + order, :])
            mu = _flat(O.adjoint_block_thomas(sc["Ad"], sc["Al"], sc["Au"], split(h), I), I)
            assert abs(np.vdot(mu, f) - aU[order]) < tol * np.max(np.abs(aU)), (I, order, tol)


def test_lsq_adjoint_solves_the_regularised_normal_equations_and_gives_dC():
    """Y = (Q^H Q + lam^2)^{-1} G: small backward error; and for the
    functional Phi(C) = Re<S, X(C)> (linear in C), central differences along
    a random dC equal Re<Q Y, dC> with Y from G = S."""
    p = small_stack(I=2, N=40, P=40, Mw=24, K=8, M=30)
    al = O.bloch(p, float(p.theta[0]))
    asm = O.Assembler(p)
    rng = np.random.default_rng(4)
    for j in (1, 2, 3):
        Q = asm.Qp(j, al["alpha"], al)
        Cm = asm.Cp(j, al["alpha"])
        rc = p.params.lsq_rcond
        lam = rc * np.max(np.linalg.norm(Q, axis=0))
        S = rng.standard_normal((Q.shape[1], Cm.shape[1])) + 1j * rng.standard_normal((Q.shape[1], Cm.shape[1]))
        Y = O.lsq_adjoint(Q, S, rc)
        Mx = Q.conj().T @ Q + lam ** 2 * np.eye(Q.shape[1])
        nQ = np.linalg.norm(Q, 2)
        assert np.linalg.norm(Mx @ Y - S) / ((nQ ** 2 + lam ** 2) * np.linalg.norm(Y) + np.linalg.norm(S)) < 1e-13
        dC = rng.standard_normal(Cm.shape) + 1j * rng.standard_normal(Cm.shape)
        eps = 1e-3
        phi = lambda Cx: np.real(np.vdot(S, O.lsq(Q, Cx, rc)))
        fd = (phi(Cm + eps * dC) - phi(Cm - eps * dC)) / (2 * eps)
        an = np.real(np.vdot(Q @ Y, dC))
        # [Q; lam I] has condition about 1/rcond = 1e10, so X(C) itself carries
        # rounding errors of about 1e-6 relative in its near-null directions,
        # where a random S makes Phi large: the differences agree to that
        assert abs(fd - an) < 1e-4 * max(1.0, abs(an)), (j, fd, an)


def test_adjoint_gradient_matches_central_differences():
    """Gradient of J = sum over angles of the reflected 0th and -1st order
    efficiencies, with respect to layer wavenumbers and interface Fourier
    coefficients: the oracle's adjoint (transposed block solve, least-squares
    adjoint, block sensitivities contracted with block derivatives by central
    differences of the assembly) against central differences of J itself
    (h = 1e-6), to 1e-6 relative.  The stack uses lsq_rcond = 1e-6: the
    per-block terms of the end layers are of order 0.3 and cancel to 1e-2,
    and at the default 1e-10 the regularisation's 1/lam ~ 1e10 amplifies the
    1e-13 error of difference-quotient block derivatives past that (the
    adjoint then misses by O(1); at 1e-8 it agrees to 2e-6, at 1e-6 to 1e-9)."""
    from dataclasses import replace
    from workloads.problems import Interface
    base = small_stack(I=2, N=40, P=40, Mw=24, K=8, M=30, n_angles=2)
    prob = replace(base, params=replace(base.params, lsq_rcond=1e-6)).with_angles([-0.9, -2.1])

    def shift_k(j):
        def make(t):
            k = prob.k.copy()
            k[j] += t
            return replace(prob, k=k)
        return make

    def shift_shape(i, which, m):
        def make(t):
            ifs = list(prob.ifaces)
            f = ifs[i]
            a, b = f.a.copy(), f.b.copy()
            (a if which == "a" else b)[m] += t
            ifs[i] = Interface(f.y0, a, b, f.N)
            return replace(prob, ifaces=ifs)
        return make

    shifted = {"k1": shift_k(0), "k2": shift_k(1), "k3": shift_k(2),
               "a1[1]": shift_shape(0, "a", 0), "b2[2]": shift_shape(1, "b", 1)}
    grad = O.adjoint_gradient(prob, shifted, {p: 1e-3 for p in shifted})
    for p, make in shifted.items():
        hfd = 1e-6
        fd = (O.bragg_objective(make(hfd)) - O.bragg_objective(make(-hfd))) / (2 * hfd)
        assert abs(grad[p] - fd) < 1e-6 * max(abs(fd), 1e-3), (p, grad[p], fd)


def test_block_sensitivities_are_rank_one_forms():
    """The contraction of the oracle's block sensitivities with central
    differences of the blocks (its adjoint_gradient) equals the same
    difference of one scalar F(M) = mu^H (f - A eta + B zeta) +
    sum_j [(Q'y)_j^H (C'_j eta^_j - Q'_j xi_j) + r_j^H Q'_j y_j] over the
    moved blocks (xi = X eta^, zeta = xi[:P], y = (Q'^H Q' + lam^2)^{-1} Psi,
    r = C' eta^ - Q' xi): the sensitivities mu eta^H, mu zeta^H, Q'Y and
    (C' - Q'X) Y^H - Q'Y X^H all have rank one, and F is linear in the
    blocks.  This is the form the GPU gradient evaluates; a transposed or
    conjugated factor in either side fails it."""
    from dataclasses import replace
    base = small_stack(I=2, N=40, P=40, Mw=24, K=8, M=30, n_angles=2)
    prob = replace(base, params=replace(base.params, lsq_rcond=1e-6)).with_angles([-0.9, -2.1])

    def shift_k(j):
        def make(t):
            k = prob.k.copy()
            k[j] += t
            return replace(prob, k=k)
        return make

    shifted = {"k2": shift_k(1), "k3": shift_k(2)}
    t = 1e-3
    ref = O.adjoint_gradient(prob, shifted, {p: t for p in shifted})
    mine = {p: 0.0 for p in shifted}
    for a in range(prob.n_theta):
        th = float(prob.theta[a])
        sc = O.schur(prob, th)
        eta1 = O.block_thomas(sc["Ad"], sc["Al"], sc["Au"], sc["f"], prob.I)[1]
        g = O.reflected_weights(prob, th, sc["bloch"]) * -(sc["X"][1][prob.params.P:, :] @ eta1)
        for p, make in shifted.items():
            mine[p] += forms_gradient(prob, a, g, [make(s_ * t) for s_ in (-2, -1, 1, 2)], t)
    for p in shifted:
        assert abs(mine[p] - ref[p]) < 1e-9 * max(abs(ref[p]), 1e-3), (p, mine[p], ref[p])


def test_parameter_blocks_are_local():
    """Which blocks a parameter moves (the locality a restricted gradient
    fill would use), on a 4-interface stack: a Fourier coefficient of
    interface 2 moves the A blocks that touch interface 2, B_{i,j} (layer j's
    proxies to interface i) with i = 2 or j in {2, 3} (the proxy circles of
    layers 2 and 3 sit at their walls' mid-height) and Q', C' of layers 2
    and 3; the wavenumber of layer 3 moves
    the A blocks of interfaces 2 and 3, B_{2,3}, B_{3,3} and Q', C' of layer
    3.  Every other block is bitwise unchanged."""
    from dataclasses import replace
    from workloads.problems import Interface
    prob = small_stack(I=4, N=40, P=40, Mw=24, K=8, M=30)
    th = float(prob.theta[0])

    def shape(t):
        ifs = list(prob.ifaces)
        f = ifs[1]
        a = f.a.copy()
        a[0] += t
        ifs[1] = Interface(f.y0, a, f.b.copy(), f.N)
        return replace(prob, ifaces=ifs)

    def wavenumber(t):
        k = prob.k.copy()
        k[2] += t
        return replace(prob, k=k)

    cases = {
        "shape": (shape, {"A": {(i, j) for (i, j) in [(1, 2), (2, 1), (2, 2), (2, 3), (3, 2)]},
                          "B": {(1, 2), (2, 2), (2, 3), (3, 3)},
                          "Qp": {2, 3}, "Cp": {2, 3}}),
        "wavenumber": (wavenumber, {"A": {(2, 2), (2, 3), (3, 2), (3, 3)},
                                    "B": {(2, 3), (3, 3)}, "Qp": {3}, "Cp": {3}}),
    }
    for name, (make, moved) in cases.items():
        lo, hi = O._blocks(make(-1e-3), th), O._blocks(make(1e-3), th)
        for kind in ("A", "B", "Qp", "Cp"):
            for key in lo[kind]:
                same = np.array_equal(lo[kind][key], hi[kind][key])
                assert same == (key not in moved[kind]), (name, kind, key, same)


def test_gradient_forms_restricted_to_the_moved_blocks():
    """The difference of F over only the blocks a parameter moves equals the
    difference over every block (the others' terms are identical in the four
    moved problems and cancel), to 1e-9 of the gradient: a shape coefficient
    of interface 2 and the wavenumber of layer 3 on a 4-interface stack."""
    from dataclasses import replace
    from workloads.problems import Interface
    base = small_stack(I=4, N=40, P=40, Mw=24, K=8, M=30)
    prob = replace(base, params=replace(base.params, lsq_rcond=1e-6))
    P, t, a = prob.params.P, 1e-3, 0
    th = float(prob.theta[a])

    def shape(s_):
        ifs = list(prob.ifaces)
        f = ifs[1]
        av = f.a.copy()
        av[0] += s_
        ifs[1] = Interface(f.y0, av, f.b.copy(), f.N)
        return replace(prob, ifaces=ifs)

    def wavenumber(s_):
        k = prob.k.copy()
        k[2] += s_
        return replace(prob, k=k)

    cases = [(shape, {"f": False, "A": {(1, 2), (2, 1), (2, 2), (2, 3), (3, 2)},
                      "B": {(1, 2), (2, 2), (2, 3), (3, 3)}, "layers": {2, 3}}),
             (wavenumber, {"f": False, "A": {(2, 2), (2, 3), (3, 2), (3, 3)},
                           "B": {(2, 3), (3, 3)}, "layers": {3}})]
    sc = O.schur(prob, th)
    eta1 = O.block_thomas(sc["Ad"], sc["Al"], sc["Au"], sc["f"], prob.I)[1]
    g = O.reflected_weights(prob, th, sc["bloch"]) * -(sc["X"][1][P:, :] @ eta1)
    for make, only in cases:
        probs = [make(s_ * t) for s_ in (-2, -1, 1, 2)]
        full = forms_gradient(prob, a, g, probs, t)
        local = forms_gradient(prob, a, g, probs, t, only=only)
        assert abs(local - full) < 1e-9 * max(abs(full), 1e-3), (local, full)
