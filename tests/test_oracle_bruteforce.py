"""One ADI sub-step of the oracle equals a dense solve of the full system
assembled by 3D quadrature from the weak form (meshes of at most 4^3 elements)."""
import numpy as np
import pytest

from oracle import maxwell_adi as ma
from oracle import bspline
from paper_2103_06998_gb300 import inputs
from bruteforce import Dense3D

CASES = [((3, 3, 3), 2, "uniform"), ((4, 3, 2), 2, "random"), ((2, 3, 4), 3, "random"),
         ((4, 4, 4), 2, "head"), ((3, 2, 3), 1, "random"), ((2, 3, 2), 4, "random")]


def _problem(n, p, kind, tau=0.07):
    if kind == "uniform":
        return ma.make_problem(n, p, tau)
    if kind == "head":
        eps, mu, sigma, _ = inputs.head_map(n, 2103)
    else:
        eps, mu, sigma = inputs.random_material(n, 7, mu_range=(1.0, 3.0))
    return ma.make_problem(n, p, tau, eps, mu, sigma)


def _bound(p):
    """1e-12; for p = 4 the dense solve's own rounding (the condition number of
    the 3D system grows with p) sits near 5e-12, so 2e-11."""
    return 1e-12 if p <= 3 else 2e-11


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
    assert _rel(got, ref) < _bound(p)


@pytest.mark.parametrize("n,p,kind", CASES)
def test_h_substep_equals_dense_solve(n, p, kind):
    prob = _problem(n, p, kind)
    s1 = ma.apply_dirichlet(inputs.random_fields(prob.shape, 4))
    s2 = ma.apply_dirichlet(inputs.random_fields(prob.shape, 5))
    D = Dense3D(n, p)
    ref = __import__("bruteforce").h_substep(D, s1[3:], s1[:3], s2[:3], prob.d)
    got = ma.solve_H(prob, ma.rhs_H(prob, s1[3:], s1[:3], s2[:3]))
    assert _rel(got, ref) < _bound(p)


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


# ---- the "quad" reading: per-element coefficients inside the right-hand side integrals

def _quad_problem(n, p, kind, tau=0.07):
    if kind == "head":
        eps, mu, sigma, _ = inputs.head_map(n, 2103)
    else:
        eps, mu, sigma = inputs.random_material(n, 7, mu_range=(1.0, 3.0))
    return ma.make_problem(n, p, tau, eps, mu, sigma, rhs_material="quad")


QUAD_CASES = [((4, 3, 2), 2, "random"), ((2, 3, 4), 3, "random"), ((4, 4, 4), 2, "head"), ((3, 2, 3), 1, "random")]


@pytest.mark.parametrize("n,p,kind", QUAD_CASES)
@pytest.mark.parametrize("half", [1, 2])
def test_quad_e_substep_equals_dense_solve(n, p, kind, half):
    # the dense assembler weights every Gauss point of its own 3D grid (scipy basis)
    # with the coefficient of the element that holds it
    prob = _quad_problem(n, p, kind)
    src = inputs.dipole(2103)
    ma.set_source(prob, src["x0"], src["comp"], src["amp"], src["f0"], src["t0"], src["s"])
    state = ma.apply_dirichlet(inputs.random_fields(prob.shape, 3))
    D = Dense3D(n, p)
    t_mid = 1.3
    g = np.sin(2 * np.pi * src["f0"] * (t_mid - src["t0"])) * np.exp(-((t_mid - src["t0"]) / src["s"]) ** 2)
    J = [np.zeros(D.phi.shape[1]) for _ in range(3)]
    J[src["comp"]] = src["amp"] * g * D.point_row(src["x0"])
    e = [min(int(np.floor(src["x0"][a] * n[a])), n[a] - 1) for a in range(3)]
    el = prob.elem
    ref = __import__("bruteforce").e_substep(D, half, state[:3], state[3:], prob.a, prob.b, prob.c, J=J,
                                             elem=(el["a"], el["b"], el["c"], el["b"][e[2], e[1], e[0]]))
    got = ma.solve_E(prob, half, ma.rhs_E(prob, half, state[:3], state[3:], t_mid))
    assert _rel(got, ref) < 1e-12
    # and it is not the row reading on this heterogeneous material
    row = ma.make_problem(n, p, prob.tau, *(_material(n, kind)))
    ma.set_source(row, src["x0"], src["comp"], src["amp"], src["f0"], src["t0"], src["s"])
    assert _rel(ma.solve_E(row, half, ma.rhs_E(row, half, state[:3], state[3:], t_mid)), ref) > 1e-4


def _material(n, kind):
    if kind == "head":
        return inputs.head_map(n, 2103)[:3]
    return inputs.random_material(n, 7, mu_range=(1.0, 3.0))


@pytest.mark.parametrize("n,p,kind", QUAD_CASES)
def test_quad_h_substep_equals_dense_solve(n, p, kind):
    prob = _quad_problem(n, p, kind)
    s1 = ma.apply_dirichlet(inputs.random_fields(prob.shape, 4))
    s2 = ma.apply_dirichlet(inputs.random_fields(prob.shape, 5))
    D = Dense3D(n, p)
    ref = __import__("bruteforce").h_substep(D, s1[3:], s1[:3], s2[:3], prob.d, d_elem=prob.elem["d"])
    got = ma.solve_H(prob, ma.rhs_H(prob, s1[3:], s1[:3], s2[:3]))
    assert _rel(got, ref) < 1e-12


@pytest.mark.parametrize("p", [1, 2, 3])
def test_quad_equals_row_for_uniform_material(p):
    n = (4, 3, 5)
    shp = (n[2], n[1], n[0])
    eps, mu, sigma = np.full(shp, 3.0), np.full(shp, 1.5), np.full(shp, 20.0)
    pr = ma.make_problem(n, p, 0.05, eps, mu, sigma)
    pq = ma.make_problem(n, p, 0.05, eps, mu, sigma, rhs_material="quad")
    for pp in (pr, pq):
        ma.set_source(pp, (0.31, 0.62, 0.45), 1, 2.0, 2.0, 0.5, 0.5)
    st = ma.apply_dirichlet(inputs.random_fields(pr.shape, 6))
    a, _ = ma.run(pr, st, 0.4, 2)
    b, _ = ma.run(pq, st, 0.4, 2)
    assert _rel(b, a) < 1e-13
