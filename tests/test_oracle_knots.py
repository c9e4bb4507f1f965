"""Pins of the oracle on non-uniform elements (open knot vectors with arbitrary
interior knots): basis = scipy.interpolate.BSpline, the closed-form integrals
int B_i = (t_{i+p+1} - t_i) / (p + 1), the identities that hold for any knots,
and one ADI sub-step = the dense solve of the full system assembled from the
weak form on the same elements."""
import numpy as np
import pytest
from scipy.interpolate import BSpline

from oracle import bspline, material
from oracle import maxwell_adi as ma
from paper_2103_06998_gb300 import inputs
from bruteforce import Dense3D
import bruteforce


def graded(n, r=1.35):
    """Element boundaries refined geometrically towards both ends."""
    h = np.array([r ** min(e, n - 1 - e) for e in range(n)], dtype=np.float64)
    b = np.concatenate([[0.0], np.cumsum(h)])
    b /= b[-1]
    b[-1] = 1.0
    return b


def jittered(n, seed):
    rng = np.random.default_rng(seed)
    h = 1.0 + 0.6 * (rng.random(n) - 0.5)
    b = np.concatenate([[0.0], np.cumsum(h)])
    b /= b[-1]
    b[-1] = 1.0
    return b


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_basis_and_matrices_on_nonuniform_knots(p):
    n = 7
    br = jittered(n, p)
    x, w, e = bspline.gauss_points(n, p + 2, br)
    v, d = bspline.eval_basis(n, p, x, e, br)
    t = bspline.knot_vector(n, p, br)
    for i in range(n + p):
        c = np.zeros(n + p)
        c[i] = 1
        s = BSpline(t, c, p)
        np.testing.assert_allclose(v[:, i], s(x), atol=1e-14)
        np.testing.assert_allclose(d[:, i], s.derivative()(x), atol=1e-11)
    M, S, A, B = bspline.matrices_1d(n, p, breaks=br)
    # int B_i = (t_{i+p+1} - t_i) / (p + 1) for every B-spline
    np.testing.assert_allclose(M.sum(axis=0), (t[p + 1:] - t[:n + p]) / (p + 1), rtol=1e-13)
    one = np.ones(n + p)
    np.testing.assert_allclose(S @ one, 0, atol=1e-11)
    np.testing.assert_allclose(A @ one, 0, atol=1e-12)
    E = np.zeros((n + p, n + p))
    E[-1, -1], E[0, 0] = 1.0, -1.0
    np.testing.assert_allclose(A + A.T, E, atol=1e-12)
    np.testing.assert_allclose(B, A.T, atol=1e-15)
    # points on element boundaries belong to the element on the right
    assert bspline.element_of(n, br[3], br) == 3 and bspline.element_of(n, 1.0, br) == n - 1


def test_uniform_breaks_equal_the_uniform_path():
    n, p = (5, 4, 3), 2
    br = tuple(np.linspace(0, 1, k + 1) for k in n)
    eps, mu, sigma, _ = inputs.head_map(n, 2103)
    a = ma.make_problem(n, p, 0.05, eps, mu, sigma)
    b = ma.make_problem(n, p, 0.05, eps, mu, sigma, breaks=br)
    st = ma.apply_dirichlet(list(inputs.random_fields(a.shape, 2)))
    ra, _ = ma.run(a, st, 0.0, 1)
    rb, _ = ma.run(b, st, 0.0, 1)
    for x, y in zip(ra, rb):
        np.testing.assert_allclose(y, x, rtol=1e-13, atol=1e-14)


def _rel(a, b):
    return np.sqrt(sum(np.sum((x - y) ** 2) for x, y in zip(a, b)) / sum(np.sum(y ** 2) for y in b))


@pytest.mark.parametrize("n,p", [((4, 3, 3), 2), ((3, 4, 2), 3), ((4, 3, 4), 1)])
@pytest.mark.parametrize("half", [1, 2])
def test_substeps_equal_dense_solve_on_nonuniform_knots(n, p, half):
    br = (graded(n[0]), jittered(n[1], 5), jittered(n[2], 6))
    eps, mu, sigma = inputs.random_material(n, 7, mu_range=(1.0, 3.0))
    prob = ma.make_problem(n, p, 0.07, eps, mu, sigma, breaks=br)
    src = inputs.dipole(2103)
    ma.set_source(prob, src["x0"], src["comp"], src["amp"], src["f0"], src["t0"], src["s"])
    st = ma.apply_dirichlet(list(inputs.random_fields(prob.shape, 3)))
    D = Dense3D(n, p, breaks=br)
    # the hats from the dense grid, independent of the oracle's element integrals
    np.testing.assert_allclose(material.row_hats(eps, n, p, br), D.hat(eps), rtol=1e-12)
    t_mid = 1.3
    g = np.sin(2 * np.pi * src["f0"] * (t_mid - src["t0"])) * np.exp(-((t_mid - src["t0"]) / src["s"]) ** 2)
    J = [np.zeros(D.phi.shape[1]) for _ in range(3)]
    J[src["comp"]] = src["amp"] * g * D.point_row(src["x0"])
    ref = bruteforce.e_substep(D, half, st[:3], st[3:], prob.a, prob.b, prob.c, J=J)
    got = ma.solve_E(prob, half, ma.rhs_E(prob, half, st[:3], st[3:], t_mid))
    assert _rel(got, ref) < 1e-12
    s2 = ma.apply_dirichlet(list(inputs.random_fields(prob.shape, 4)))
    refh = bruteforce.h_substep(D, st[3:], st[:3], s2[:3], prob.d)
    goth = ma.solve_H(prob, ma.rhs_H(prob, st[3:], st[:3], s2[:3]))
    assert _rel(goth, refh) < 1e-12
