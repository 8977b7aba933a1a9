"""Host logic of paper_1410_5003_gb300.diff.bragg_efficiency (the torch
autograd function over the parameter gradient), driven through an
oracle-backed stand-in context: the forward value is the oracle's objective
and the backward gradient the oracle's adjoint gradient, including the
weights' own term for the top layer's wavenumber."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import mlqp_oracle as O  # noqa: E402
from paper_1410_5003_gb300.diff import bragg_efficiency, reflected_weights  # noqa: E402
from tests.adjoint_forms import OracleContext, gradient_family  # noqa: E402


def test_reflected_weights_match_the_oracle():
    prob, make_problem, _, _ = gradient_family()
    for pv in (np.zeros(5), np.array([0.3, 0, 0, 0, 0])):
        pr = make_problem(pv)
        w = reflected_weights(pr, (0, -1, 1))
        for a in range(pr.n_theta):
            th = float(pr.theta[a])
            ref = O.reflected_weights(pr, th, O.bloch(pr, th), (0, -1, 1))
            assert np.allclose(w[a], ref, rtol=1e-14, atol=0.0)


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
    # a forward pass that needs no gradient releases its context at once
    made.clear()
    with torch.no_grad():
        bragg_efficiency(torch.zeros(5, dtype=torch.float64), make_problem, new_context=new_context)
    assert len(made) == 1 and made[0].closed
