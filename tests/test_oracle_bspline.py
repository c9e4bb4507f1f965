"""Pins of oracle.bspline against closed forms and scipy (no GPU)."""
import numpy as np
import pytest
from scipy.interpolate import BSpline

from oracle import bspline


def test_p2_interior_stencils_closed_form():
    # Uniform quadratic B-splines: int B_i B_{i+k} = h [66, 26, 1]/120 (the
    # quintic B-spline at the integers); stiffness h^-1 [1, -1/3, -1/6];
    # advection int B_i' B_l for i - l = 0, 1, 2: [0, 5/12, 1/24] (antisymmetric).
    n, p = 12, 2
    h = 1.0 / n
    M, S, A, B = bspline.matrices_1d(n, p)
    for l in range(4, 9):
        np.testing.assert_allclose(M[l, l - 2:l + 3] * 120 / h, [1, 26, 66, 26, 1], atol=1e-12)
        np.testing.assert_allclose(S[l, l - 2:l + 3] * h, [-1 / 6, -1 / 3, 1, -1 / 3, -1 / 6], atol=1e-12)
        np.testing.assert_allclose(A[l, l - 2:l + 3], [-1 / 24, -5 / 12, 0, 5 / 12, 1 / 24], atol=1e-12)


def test_p1_closed_form():
    # linear hat functions: M interior h [1/6, 2/3, 1/6], S h^-1 [-1, 2, -1]
    n, p = 10, 1
    h = 1.0 / n
    M, S, A, _ = bspline.matrices_1d(n, p)
    np.testing.assert_allclose(M[5, 4:7] / h, [1 / 6, 2 / 3, 1 / 6], atol=1e-13)
    np.testing.assert_allclose(S[5, 4:7] * h, [-1, 2, -1], atol=1e-12)
    np.testing.assert_allclose(A[5, 4:7], [-0.5, 0, 0.5], atol=1e-13)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
@pytest.mark.parametrize("n", [1, 3, 7])
def test_invariants(n, p):
    M, S, A, B = bspline.matrices_1d(n, p)
    N = n + p
    # partition of unity: sum over all trial functions of M = int B_l
    G = bspline.element_integrals(n, p).sum(axis=1)
    np.testing.assert_allclose(M.sum(axis=1), G, atol=1e-13)
    np.testing.assert_allclose(G.sum(), 1.0, atol=1e-13)
    # constants are in the kernel of S and of A (derivative of 1 is 0)
    np.testing.assert_allclose(S @ np.ones(N), 0, atol=1e-11)
    np.testing.assert_allclose(A @ np.ones(N), 0, atol=1e-12)
    # integration by parts: A + A^T = e_N e_N^T - e_1 e_1^T, B = A^T
    E = np.zeros((N, N))
    E[-1, -1], E[0, 0] = 1.0, -1.0
    np.testing.assert_allclose(A + A.T, E, atol=1e-12)
    np.testing.assert_allclose(B, A.T, atol=1e-14)
    np.testing.assert_allclose(M, M.T, atol=1e-15)
    np.testing.assert_allclose(S, S.T, atol=1e-12)
    assert np.all(np.linalg.eigvalsh(M) > 0)
    # bandwidth p
    i, j = np.nonzero(np.abs(M) + np.abs(S) + np.abs(A) > 0)
    assert np.max(np.abs(i - j)) <= p


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_basis_against_scipy(p):
    n = 5
    x, w, e = bspline.gauss_points(n, p + 2)
    v, d = bspline.eval_basis(n, p, x, e)
    t = bspline.knot_vector(n, p)
    for i in range(n + p):
        c = np.zeros(n + p)
        c[i] = 1
        s = BSpline(t, c, p)
        np.testing.assert_allclose(v[:, i], s(x), atol=1e-14)
        np.testing.assert_allclose(d[:, i], s.derivative()(x), atol=1e-12)


def test_point_values_partition_of_unity():
    for x0 in (0.0, 0.13, 0.5, 0.77, 1.0 - 1e-12):
        np.testing.assert_allclose(bspline.point_values(9, 2, x0).sum(), 1.0, atol=1e-14)
