"""Host logic of paper_1410_5003_gb300.diff.bragg_efficiency (the torch
autograd function over the parameter gradient), driven through an
oracle-backed stand-in context: the forward value is the oracle's objective
and the backward gradient the oracle's adjoint gradient, including the
weights' own term for the top layer's wavenumber."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import mlqp_oracle as O  # noqa: E402
from paper_1410_5003_gb300.diff import bragg_efficiency  # noqa: E402
from tests.adjoint_forms import OracleContext, gradient_family  # noqa: E402


def test_bragg_efficiency_value_and_gradient_on_the_oracle():
    prob, make_problem, shifted, names = gradient_family()
    made = []

    def new_context(pr):
        made.append(OracleContext(pr))
        return made[-1]

    p = torch.zeros(5, dtype=torch.float64, requires_grad=True)
    J = bragg_efficiency(p, make_problem, new_context=new_context)
    assert abs(J.item() - O.bragg_objective(prob)) < 1e-13 * abs(J.item())
    J.backward()
    ref = O.adjoint_gradient(prob, shifted, {nm: 1e-3 for nm in names})
    for q, nm in enumerate(names):
        assert abs(p.grad[q].item() - ref[nm]) < 1e-9 * max(abs(ref[nm]), 1e-3), (nm, p.grad[q].item(), ref[nm])
    # the base context and four moved ones, moved on to each later parameter
    assert len(made) == 5 and all(c.closed for c in made)
    assert all(getattr(c, "moves", 0) == len(names) - 1 for c in made[1:])
    assert made[0].prepares == 1  # one solve and one set of sensitivities for all five parameters
    # each of the five moves one layer wavenumber or one interface: all evaluated locally
    assert made[0].local_evals == len(names)
    # a forward pass that needs no gradient releases its context at once
    made.clear()
    with torch.no_grad():
        bragg_efficiency(torch.zeros(5, dtype=torch.float64), make_problem, new_context=new_context)
    assert len(made) == 1 and made[0].closed


def test_bragg_efficiency_edge_cases_on_the_oracle():
    """No parameters: an empty gradient (one solve, the sensitivities still
    formed); a second backward through the same graph is refused (the
    solver context was released by the first)."""
    from workloads import small_stack
    prob = small_stack(I=1, N=40, P=40, Mw=24, K=8, M=30)

    def make_problem(pv):
        return prob

    p = torch.zeros(0, dtype=torch.float64, requires_grad=True)
    J = bragg_efficiency(p, make_problem, new_context=OracleContext)
    J.backward()
    assert p.grad.shape == (0,)
    p = torch.zeros(1, dtype=torch.float64, requires_grad=True)
    J = bragg_efficiency(p, make_problem, new_context=OracleContext)
    J.backward(retain_graph=True)
    assert abs(p.grad.item()) < 1e-9  # make_problem ignores p: dJ/dp = 0 up to the difference's rounding
    with pytest.raises(RuntimeError):
        J.backward()


def weight_cases():
    """A grazing angle of order +1 (kappa_1 = k_1, a Wood anomaly) and an
    ordinary one, on a one-interface stack with K = 8."""
    import math
    from dataclasses import replace
    from workloads import small_stack
    prob = small_stack(I=1, N=40, P=40, Mw=24, K=8, M=30)
    k1, d = float(np.real(prob.k[0])), prob.d
    th_w = -math.acos(1.0 - 2.0 * math.pi / (d * k1))
    return replace(prob).with_angles([th_w, -0.9]), k1, d, th_w


def check_weight_cases(w, K, k1, d, th_w):
    """w_n = 0 where k^U_n is imaginary or zero, and the specular weight is 1
    (k^U_0 = k_1 |sin theta|)."""
    import math
    assert abs(w[0, K] - 1.0) < 1e-14 and abs(w[1, K] - 1.0) < 1e-14
    kap = k1 * math.cos(th_w) + 2 * math.pi / d
    assert w[0, K + 1] == 0.0 or k1 * k1 - kap * kap <= 1e-12 * k1 * k1
    assert w[1, K + 8] == 0.0 and w[1, K - 8] == 0.0  # evanescent at |n| = 8
    for n in range(-K, K + 1):  # orders not asked for weigh nothing
        if n not in (0, 1, -8, 8):
            assert w[0, K + n] == 0.0 and w[1, K + n] == 0.0


def test_reflected_weights_vanish_for_evanescent_and_grazing_orders():
    """The oracle's weights on the special cases: the specular weight is 1
    whatever the angle, evanescent and grazing orders weigh 0."""
    pr, k1, d, th_w = weight_cases()
    w = OracleContext(pr).efficiency_weights(orders=(0, 1, -8, 8))
    check_weight_cases(w, pr.params.K, k1, d, th_w)


def test_parameter_locality_is_read_from_the_moved_problems():
    """The autograd path evaluates a parameter locally (only the blocks near
    it) when its moved problems differ from the base in one layer wavenumber
    or one interface, and over the whole stack otherwise."""
    from paper_1410_5003_gb300.diff import _locality
    from paper_1410_5003_gb300.mlqp import PARAM_INTERFACE, PARAM_LAYER
    prob, make_problem, _, _ = gradient_family()

    def moved(q):
        out = []
        for s_ in (-2, -1, 1, 2):
            if q == 5:  # two parameters at once
                pv = np.array([0, 0, s_ * 1e-3, s_ * 1e-3, 0])
            else:
                pv = np.zeros(5)
                pv[q] = s_ * 1e-3
            out.append(make_problem(pv))
        return out

    assert _locality(prob, moved(0)) == (PARAM_LAYER, 1)
    assert _locality(prob, moved(2)) == (PARAM_LAYER, 3)
    assert _locality(prob, moved(3)) == (PARAM_INTERFACE, 1)
    assert _locality(prob, moved(4)) == (PARAM_INTERFACE, 2)
    assert _locality(prob, moved(5)) is None
