"""One ADI sub-step of the oracle equals a dense solve of the full system
assembled by 3D quadrature from the weak form (meshes of at most 4^3 elements)."""
import numpy as np
import pytest

from oracle import maxwell_adi as ma
from oracle import bspline
from paper_2103_06998_gb300 import inputs
from bruteforce import Dense3D

CASES = [((3, 3, 3), 2, "uniform"), ((4, 3, 2), 2, "random"), ((2, 3, 4), 3, "random"),
         ((4, 4, 4), 2, "head"), ((3, 2, 3), 1, "random")]


def _problem(n, p, kind, tau=0.07):
    if kind == "uniform":
        return ma.make_problem(n, p, tau)
    if kind == "head":
        eps, mu, sigma, _ = inputs.head_map(n, 2103)
    else:
        eps, mu, sigma = inputs.random_material(n, 7, mu_range=(1.0, 3.0))
    return ma.make_problem(n, p, tau, eps, mu, sigma)


def _rel(a, b):
    return np.sqrt(sum(np.sum((x - y) ** 2) for x, y in zip(a, b)) / sum(np.sum(y ** 2) for y in b))


@pytest.mark.parametrize("n,p,kind", CASES)
@pytest.mark.parametrize("half", [1, 2])
def test_e_substep_equals_dense_solve(n, p, kind, half):
    prob = _problem(n, p, kind)
    state = ma.apply_dirichlet(inputs.random_fields(prob.shape, 3))
    D = Dense3D(n, p)
    ref = __import__("bruteforce").e_substep(D, half, state[:3], state[3:], prob.a, prob.b, prob.c)
    got = ma.solve_E(prob, half, ma.rhs_E(prob, half, state[:3], state[3:], 0.0))
    assert _rel(got, ref) < 1e-12


@pytest.mark.parametrize("n,p,kind", CASES)
def test_h_substep_equals_dense_solve(n, p, kind):
    prob = _problem(n, p, kind)
    s1 = ma.apply_dirichlet(inputs.random_fields(prob.shape, 4))
    s2 = ma.apply_dirichlet(inputs.random_fields(prob.shape, 5))
    D = Dense3D(n, p)
    ref = __import__("bruteforce").h_substep(D, s1[3:], s1[:3], s2[:3], prob.d)
    got = ma.solve_H(prob, ma.rhs_H(prob, s1[3:], s1[:3], s2[:3]))
    assert _rel(got, ref) < 1e-12


def test_source_row_equals_dense():
    n, p = (3, 4, 3), 2
    prob = _problem(n, p, "random")
    src = inputs.dipole(2103)
    ma.set_source(prob, src["x0"], src["comp"], src["amp"], src["f0"], src["t0"], src["s"])
    state = ma.apply_dirichlet(inputs.random_fields(prob.shape, 8))
    D = Dense3D(n, p)
    t_mid = 1.3
    g = np.sin(2 * np.pi * src["f0"] * (t_mid - src["t0"])) * np.exp(-((t_mid - src["t0"]) / src["s"]) ** 2)
    J = [np.zeros(D.phi.shape[1]) for _ in range(3)]
    J[src["comp"]] = src["amp"] * g * D.point_row(src["x0"])
    ref = __import__("bruteforce").e_substep(D, 1, state[:3], state[3:], prob.a, prob.b, prob.c, J=J)
    got = ma.solve_E(prob, 1, ma.rhs_E(prob, 1, state[:3], state[3:], t_mid))
    assert _rel(got, ref) < 1e-12


def test_x_first_order_is_not_exact_for_heterogeneous_material():
    # The Appendix order (material direction first) is exact; solving the mass
    # direction first is not when the row coefficients vary.  This guards the
    # ordering itself.
    n, p = (3, 3, 3), 2
    prob = _problem(n, p, "random")
    state = ma.apply_dirichlet(inputs.random_fields(prob.shape, 9))
    rhs = ma.rhs_E(prob, 1, state[:3], state[3:], 0.0)
    from oracle.banded import solve_lines
    M, S, _, _ = prob.mats["x"]
    u = solve_lines(M, rhs[0], "x", p, False)
    u = solve_lines(M, u, "z", p, True)
    u = solve_lines(prob.mats["y"][0], u, "y", p, True, stiff=prob.mats["y"][1], coef=prob.c)
    D = Dense3D(n, p)
    ref = __import__("bruteforce").e_substep(D, 1, state[:3], state[3:], prob.a, prob.b, prob.c)
    assert _rel([u], [ref[0]]) > 1e-6
