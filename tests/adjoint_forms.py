"""Test infrastructure: the rank-one form of the adjoint gradient's block
sensitivities, evaluated on the oracle's blocks, and an oracle-backed
stand-in for a solver context (solve_host, fd_gradient, close) that runs the
same steps the GPU gradient takes."""
import numpy as np

from oracle import mlqp_oracle as O


def forms_gradient(prob, a, g, moved_probs, t, only=None):
    """2 Re[(F(-2t) - 8 F(-t) + 8 F(t) - F(2t)) / (12 t)] for angle a: the
    sensitivities of prob's solve with g = w a^U of that angle (mu from
    A'^H mu = -X_1[P:]^H g; xi = X eta^; y = (Q'^H Q' + lam^2)^{-1} Psi;
    Q'y and r = C' eta^ - Q' xi), and F(M) = mu^H (f - A eta + B xi[:P]) +
    sum_j [(Q'y)_j^H (C'_j eta^_j - Q'_j xi_j) + r_j^H Q'_j y_j] over the
    oracle blocks of each moved problem.  only: None (every block) or
    {"f": bool, "A": keys, "B": keys, "layers": layers}, the terms kept."""
    I, P, rc = prob.I, prob.params.P, prob.params.lsq_rcond
    th = float(prob.theta[a])
    sc = O.schur(prob, th)
    eta = O.block_thomas(sc["Ad"], sc["Al"], sc["Au"], sc["f"], I)
    X = sc["X"]
    h = {i: np.zeros_like(eta[i]) for i in range(1, I + 1)}
    h[1] = -(X[1][P:, :].conj().T @ g)
    mu = O.adjoint_block_thomas(sc["Ad"], sc["Al"], sc["Au"], h, I)
    etaL = {j: np.concatenate([eta[i] for i in O.layer_columns(prob, j)]) for j in range(1, I + 2)}
    asm = O.Assembler(prob)
    xi, y, qy, rv = {}, {}, {}, {}
    for j in range(1, I + 2):
        psi = np.zeros(X[j].shape[0], np.complex128)
        for i in (j - 1, j):
            if 1 <= i <= I:
                psi[:P] += asm.B(i, j).conj().T @ mu[i]
        if j == 1:
            psi[P:] = -g
        y[j] = O.lsq_adjoint(sc["Qp"][j], psi[:, None], rc)[:, 0]
        xi[j] = X[j] @ etaL[j]
        qy[j] = sc["Qp"][j] @ y[j]
        rv[j] = sc["Cp"][j] @ etaL[j] - sc["Qp"][j] @ xi[j]

    keep = (lambda kind, key: True) if only is None else (lambda kind, key: key in only[kind])

    def F(b):
        s = np.vdot(mu[1], b["f"]) if only is None or only["f"] else 0.0
        for (i, j), A in b["A"].items():
            if keep("A", (i, j)):
                s -= np.vdot(mu[i], A @ eta[j])
        for (i, j), B in b["B"].items():
            if keep("B", (i, j)):
                s += np.vdot(mu[i], B @ xi[j][:P])
        for j in range(1, I + 2):
            if keep("layers", j):
                s += np.vdot(qy[j], b["Cp"][j] @ etaL[j] - b["Qp"][j] @ xi[j]) + np.vdot(rv[j], b["Qp"][j] @ y[j])
        return s

    Fs = [F(O._blocks(mp, th)) for mp in moved_probs]
    return 2.0 * ((Fs[0] - 8 * Fs[1] + 8 * Fs[2] - Fs[3]) / (12 * t)).real


class OracleContext:
    """Oracle-backed stand-in for a solver context: a solve leaves
    'factors', a gradient uses them up (as the library's does)."""

    def __init__(self, prob):
        self.prob = prob
        self.factored = False
        self.closed = False

    def solve_host(self):
        asm = O.Assembler(self.prob)
        aU = np.array([O.solve(self.prob, a, asm)["aU"] for a in range(self.prob.n_theta)])
        self.factored = True
        self.aU = aU
        return {"aU": aU}

    def efficiency_weights(self, orders=(0, -1)):
        pr = self.prob
        return np.array([O.reflected_weights(pr, float(th), O.bloch(pr, float(th)), tuple(orders))
                         for th in pr.theta])

    def efficiency_weight_gradient(self, moved, t, orders=(0, -1)):
        wm = [m.efficiency_weights(orders) for m in moved]
        dw = ((wm[0] - wm[3]) + 8.0 * (wm[2] - wm[1])) / (12.0 * t)
        return np.sum(dw * np.abs(self.aU) ** 2, axis=1)

    def fd_gradient(self, moved, t, g):
        if not self.factored:
            raise RuntimeError("no factors: solve first")
        self.factored = False
        probs = [m.prob for m in moved]
        return np.array([forms_gradient(self.prob, a, g[a], probs, t) for a in range(self.prob.n_theta)])

    def gradient_prepare(self, g):
        if not self.factored:
            raise RuntimeError("no factors: solve first")
        self.factored = False
        self.prepares = getattr(self, "prepares", 0) + 1
        return np.array(g)

    def gradient_eval(self, moved, t, work):
        self.evals = getattr(self, "evals", 0) + 1
        probs = [m.prob for m in moved]
        return np.array([forms_gradient(self.prob, a, work[a], probs, t) for a in range(self.prob.n_theta)])

    def gradient_eval_local(self, moved, t, work, kind, index):
        self.local_evals = getattr(self, "local_evals", 0) + 1
        return self.gradient_eval(moved, t, work)

    def set_problem(self, prob):
        self.prob = prob
        self.factored = False
        self.moves = getattr(self, "moves", 0) + 1

    def close(self):
        self.closed = True


def gradient_family():
    """The oracle's gradient pin stack (2 interfaces, 2 angles, lsq_rcond
    1e-6) as a family in five parameters p = (dk_1, dk_2, dk_3, da_1[1],
    db_2[2]): make_problem(p) and, for the oracle, the same five one-parameter
    shifts by name."""
    from dataclasses import replace
    from workloads import small_stack
    from workloads.problems import Interface
    base = small_stack(I=2, N=40, P=40, Mw=24, K=8, M=30, n_angles=2)
    prob = replace(base, params=replace(base.params, lsq_rcond=1e-6)).with_angles([-0.9, -2.1])

    def make_problem(p):
        k = prob.k.copy()
        k[:3] += p[:3]
        ifs = list(prob.ifaces)
        f0, f1 = ifs[0], ifs[1]
        a0 = f0.a.copy()
        a0[0] += p[3]
        b1 = f1.b.copy()
        b1[1] += p[4]
        ifs[0] = Interface(f0.y0, a0, f0.b.copy(), f0.N)
        ifs[1] = Interface(f1.y0, f1.a.copy(), b1, f1.N)
        return replace(prob, k=k, ifaces=ifs)

    def unit(q):
        def make(t):
            p = np.zeros(5)
            p[q] = t
            return make_problem(p)
        return make

    names = ["k1", "k2", "k3", "a1[1]", "b2[2]"]
    return prob, make_problem, {nm: unit(q) for q, nm in enumerate(names)}, names
