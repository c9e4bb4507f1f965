"""Host logic of one axis as the library runs it (no GPU), on uniform and
non-uniform elements:
* adi_axis_bands: the band form of the mass, stiffness and mixed matrices
  defined after eq. discrete4 (section "Variational formulation") against the
  oracle's dense matrices, the closed-form interior stencils of cardinal
  B-splines, the symmetry B = A^T, and the interior rows the kernels replace by
  one constant stencil;
* adi_axis_tables: the element integrals of the basis (material weights)
  against the oracle, and the largest Dirichlet-reduced eigenvalue of M^{-1} S
  against the oracle's generalised eigensolver and the closed form for linear
  elements;
* adi_axis_element_matrices: the per-element blocks of the quad right-hand
  side against the oracle's quadrature on each element, summing to the bands;
* adi_axis_mass_lu: the mass LU factors (full and Dirichlet-reduced) multiply
  back to M, are symmetric (U = L^T) with positive pivots, and solve like a
  dense solver;
* adi_axis_point_basis: the dipole's basis values against the oracle, with the
  element rule at element boundaries and the partition of unity.
"""
from fractions import Fraction

import numpy as np
import pytest

from oracle import bspline


def _adi():
    from paper_2103_06998_gb300 import adi
    return adi


def graded(n, r=1.25):
    h = np.array([r ** min(e, n - 1 - e) for e in range(n)], dtype=np.float64)
    b = np.concatenate([[0.0], np.cumsum(h)])
    b /= b[-1]
    b[-1] = 1.0
    return b


def core(n, layers=4, r=1.3):
    """Uniform elements in the middle, geometrically refined towards both ends."""
    h = np.array([r ** (min(e, n - 1 - e) - layers) if min(e, n - 1 - e) < layers else 1.0 for e in range(n)])
    b = np.concatenate([[0.0], np.cumsum(h)])
    b /= b[-1]
    b[-1] = 1.0
    return b


def _dense_to_band(X, p):
    N = X.shape[0]
    out = np.zeros((N, 2 * p + 1))
    for k in range(N):
        for d in range(2 * p + 1):
            i = k + d - p
            if 0 <= i < N:
                out[k, d] = X[k, i]
    return out


def _cardinal(p, deriv):
    """Interior stencil of the uniform-mesh matrices for h = 1, exact: the
    integrals of products of cardinal B-splines (and of their derivatives) are
    values of the cardinal B-spline of degree 2p+1 (and of its second
    derivative) at the integers."""
    from math import comb, factorial

    def bspline_value(m, x, order):  # order-th derivative of the cardinal B-spline of degree m at x
        s = Fraction(0)
        for j in range(m + 2):
            t = x - j
            if t > 0 and m - order >= 0:
                s += (-1) ** j * comb(m + 1, j) * Fraction(t) ** (m - order) * factorial(m) / factorial(m - order)
        return s / factorial(m)

    m = 2 * p + 1
    # int B(x) B(x - k) dx = B_{2p+1}(p + 1 + k); int B'(x) B'(x - k) dx = -B''_{2p+1}(p + 1 + k)
    return [float(bspline_value(m, p + 1 + k, 0) if deriv == 0 else -bspline_value(m, p + 1 + k, 2))
            for k in range(-p, p + 1)]


@pytest.mark.parametrize("p", [1, 2, 3, 4])
@pytest.mark.parametrize("kind", ["uniform", "graded", "core"])
@pytest.mark.parametrize("n", [1, 3, 7, 16])
def test_bands_equal_the_oracle_matrices(n, p, kind):
    br = None if kind == "uniform" else (graded(n) if kind == "graded" else core(n))
    bands, inner = _adi().axis_bands(n, p, br)
    M, S, A, B = bspline.matrices_1d(n, p, breaks=br)
    for name, X in zip("MSAB", (M, S, A, B)):
        ref = _dense_to_band(X, p)
        scale = np.max(np.abs(ref))
        assert np.max(np.abs(bands[name] - ref)) <= 1e-13 * scale, name
    # B = A^T in band form: B[k][d] = A[k + d - p][2p - d]
    N, W = n + p, 2 * p + 1
    for k in range(N):
        for d in range(W):
            i = k + d - p
            if 0 <= i < N:
                assert bands["B"][k, d] == pytest.approx(bands["A"][i, W - 1 - d], rel=1e-13, abs=1e-15)
            else:
                assert bands["B"][k, d] == 0.0 and bands["M"][k, d] == 0.0


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_uniform_interior_stencils_are_the_cardinal_values(p):
    n = 24
    h = 1.0 / n
    bands, (lo, hi) = _adi().axis_bands(n, p)
    N = n + p
    # uniform elements: every row inside 2p .. N-1-2p carries the interior stencil
    assert (lo, hi) == (2 * p, N - 1 - 2 * p)
    m, s = _cardinal(p, 0), _cardinal(p, 1)
    for k in range(lo, hi + 1):
        # rounding bounds: the host compiler may contract a*b+c into one FMA (it does on Arm)
        np.testing.assert_allclose(bands["M"][k], np.array(m) * h, rtol=1e-12, atol=0)
        np.testing.assert_allclose(bands["S"][k], np.array(s) / h, rtol=1e-11, atol=1e-11 / h)
        # A is antisymmetric in the interior (int B_i' B_l = -int B_i B_l'), rows sum to zero
        a_scale = np.max(np.abs(bands["A"][k]))
        np.testing.assert_allclose(bands["A"][k], -bands["A"][k][::-1], rtol=0, atol=1e-13 * a_scale)
        assert abs(bands["A"][k].sum()) < 1e-13 * a_scale and abs(bands["S"][k].sum()) < 1e-10 / h
    # partition of unity: the rows of M sum to the integral of each basis function
    G = bspline.element_integrals(n, p).sum(axis=1)
    np.testing.assert_allclose(bands["M"].sum(axis=1), G, rtol=1e-12)


@pytest.mark.parametrize("p", [1, 2, 3])
@pytest.mark.parametrize("kind", ["graded", "core"])
def test_interior_rows_carry_the_middle_row(p, kind):
    n = 30
    br = graded(n) if kind == "graded" else core(n)
    bands, (lo, hi) = _adi().axis_bands(n, p, br)
    N = n + p
    # the interior rows lie inside 2p .. N-1-2p, hold the middle row's bands,
    # and the rows just outside them do not
    assert 2 * p <= lo <= hi <= N - 1 - 2 * p
    mid = (2 * p + N - 1 - 2 * p) // 2
    # the B-splines nonzero on element e depend only on the knots of elements
    # e-p+1 .. e+p-1, so band row k (an integral over elements k-p .. k) is fixed
    # by the sizes of elements k-2p+1 .. k+p-1
    if kind == "graded":  # sizes change from element to element: the middle row alone
        assert lo == hi == mid
    else:  # uniform elements 4 .. 25: rows k with 4 <= k-2p+1 and k+p-1 <= 25
        assert (lo, hi) == (3 + 2 * p, 26 - p)
    for name in "MSAB":
        X = bands[name]
        scale = np.max(np.abs(X[mid]))
        for k in range(lo, hi + 1):
            assert np.max(np.abs(X[k] - X[mid])) <= 1e-12 * scale
    differs = lambda k: any(np.max(np.abs(bands[x][k] - bands[x][mid])) > 1e-12 * np.max(np.abs(bands[x][mid]))
                            for x in "MSAB")
    assert lo == 2 * p or differs(lo - 1)
    assert hi == N - 1 - 2 * p or differs(hi + 1)


def test_small_axes_have_no_interior_rows():
    for n, p in [(1, 1), (2, 2), (4, 3), (3, 4)]:
        _, (lo, hi) = _adi().axis_bands(n, p)
        assert lo > hi


def test_invalid_arguments_are_rejected():
    adi = _adi()
    for args in [(0, 2, None), (4, 0, None), (4, 5, None), (3, 2, np.array([0.0, 0.5, 0.4, 1.0])),
                 (3, 2, np.array([0.0, 0.2, 0.6, 0.9])), (3, 2, np.array([0.1, 0.2, 0.6, 1.0])),
                 (3, 2, np.array([0.0, np.nan, 0.6, 1.0]))]:
        with pytest.raises(adi.AdiError) as e:
            adi.axis_bands(*args)
        assert e.value.status == adi.ADI_EINVAL


@pytest.mark.parametrize("p", [1, 2, 3, 4])
@pytest.mark.parametrize("kind", ["uniform", "graded", "core"])
@pytest.mark.parametrize("reduced", [False, True])
def test_mass_lu_reproduces_the_mass_matrix(p, kind, reduced):
    n = 17
    br = None if kind == "uniform" else (graded(n) if kind == "graded" else core(n))
    Lb, inv_d, Ub = _adi().axis_mass_lu(n, p, br, reduced)
    N = n + p
    lo, hi = (1, N - 2) if reduced else (0, N - 1)
    M = bspline.matrices_1d(n, p, breaks=br)[0][lo:hi + 1, lo:hi + 1]
    m = hi - lo + 1
    L, U = np.eye(m), np.eye(m)
    for k in range(lo, hi + 1):
        for q in range(1, p + 1):
            if k - q >= lo:
                L[k - lo, k - q - lo] = Lb[k, q - 1]
            if k + q <= hi:
                U[k - lo, k + q - lo] = Ub[k, q - 1]
    # M is symmetric positive definite: positive pivots, and U = L^T up to rounding
    assert np.all(inv_d[lo:hi + 1] > 0)
    np.testing.assert_allclose(U, L.T, rtol=1e-12, atol=1e-14)
    D = np.diag(1.0 / inv_d[lo:hi + 1])
    np.testing.assert_allclose(L @ D @ U, M, rtol=0, atol=1e-13 * np.max(np.abs(M)))
    # rows outside the factorised range stay zero; a solve with the factors matches a dense solve
    out = [k for k in range(N) if k < lo or k > hi]
    assert np.all(inv_d[out] == 0) and np.all(Lb[out] == 0) and np.all(Ub[out] == 0)
    b = np.random.default_rng(5).standard_normal(m)
    x = np.linalg.solve(U, np.linalg.solve(D, np.linalg.solve(L, b)))
    np.testing.assert_allclose(x, np.linalg.solve(M, b), rtol=1e-10, atol=1e-12 * np.max(np.abs(x)))


@pytest.mark.parametrize("p", [1, 2, 3, 4])
@pytest.mark.parametrize("kind", ["uniform", "graded"])
def test_point_basis_equals_the_oracle(p, kind):
    n = 9 if kind == "graded" else 8  # uniform: dyadic boundaries, exact in binary
    br = graded(n) if kind == "graded" else None
    edges = br if br is not None else np.linspace(0.0, 1.0, n + 1)
    xs = list(np.random.default_rng(11).random(20)) + [0.0, 1.0] + list(edges[1:-1])
    for x0 in xs:
        e, vals = _adi().axis_point_basis(n, p, x0, br)
        ref = bspline.point_values(n, p, x0, breaks=br)
        full = np.zeros(n + p)
        full[e:e + p + 1] = vals
        np.testing.assert_allclose(full, ref, rtol=1e-13, atol=1e-15)
        # the element holding x0; a boundary point belongs to the element on its right, 1 to the last
        assert edges[e] <= x0 <= edges[e + 1] and (x0 < edges[e + 1] or e == n - 1)
        # partition of unity, non-negative values
        assert abs(vals.sum() - 1.0) < 1e-14 and np.all(vals >= 0)


def test_host_axis_calls_reject_invalid_arguments():
    adi = _adi()
    for call in (lambda: adi.axis_mass_lu(0, 2), lambda: adi.axis_mass_lu(4, 5),
                 lambda: adi.axis_mass_lu(3, 2, np.array([0.0, 0.6, 0.5, 1.0])),
                 lambda: adi.axis_point_basis(4, 2, -0.1), lambda: adi.axis_point_basis(4, 2, 1.5),
                 lambda: adi.axis_point_basis(4, 2, float("nan")), lambda: adi.axis_point_basis(4, 0, 0.5)):
        with pytest.raises(adi.AdiError) as e:
            call()
        assert e.value.status == adi.ADI_EINVAL
    L = adi.load_library()
    z = np.zeros(64)
    assert L.adi_axis_mass_lu(4, 2, None, 2, adi._dptr(z), adi._dptr(z), adi._dptr(z)) == adi.ADI_EINVAL
    assert L.adi_axis_mass_lu(4, 2, None, 0, None, adi._dptr(z), adi._dptr(z)) == adi.ADI_EINVAL


@pytest.mark.parametrize("p", [1, 2, 3, 4])
@pytest.mark.parametrize("kind", ["uniform", "graded", "core"])
def test_element_integrals_and_lambda_max_equal_the_oracle(p, kind):
    from oracle import material
    n = 14
    br = None if kind == "uniform" else (graded(n) if kind == "graded" else core(n))
    G, lam = _adi().axis_tables(n, p, br)
    ref = bspline.element_integrals(n, p, breaks=br)  # (N, n): integral of B_r over element e
    N = n + p
    for r in range(N):
        for a in range(p + 1):
            e = r - p + a
            assert G[r, a] == pytest.approx(ref[r, e] if 0 <= e < n else 0.0, rel=1e-13, abs=1e-16)
    # each basis function's integrals over its elements sum to its integral, and all of them to 1
    assert G.sum() == pytest.approx(1.0, rel=1e-13)
    assert lam == pytest.approx(material.lambda_max(n, p, br), rel=1e-10)


def test_lambda_max_of_linear_elements_is_the_closed_form():
    # p = 1, uniform: M_D^{-1} S_D has the eigenvalues (6/h^2)(1 - cos t)/(2 + cos t),
    # t = k pi / n, k = 1 .. n-1 (the tridiagonal stencils h/6 [1 4 1] and 1/h [-1 2 -1])
    for n in (4, 9, 20):
        h = 1.0 / n
        t = np.arange(1, n) * np.pi / n
        exact = np.max(6.0 / h ** 2 * (1 - np.cos(t)) / (2 + np.cos(t)))
        assert _adi().axis_tables(n, 1)[1] == pytest.approx(exact, rel=1e-12)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
@pytest.mark.parametrize("kind", ["uniform", "graded"])
def test_element_blocks_equal_the_oracle_and_sum_to_the_bands(p, kind):
    n = 11
    br = graded(n) if kind == "graded" else None
    loc = _adi().axis_element_matrices(n, p, br)
    x, w, elem = bspline.gauss_points(n, p + 1, br)
    v, d = bspline.eval_basis(n, p, x, elem, br)
    N = n + p
    dense = np.zeros((4, N, N))
    for e in range(n):
        q = elem == e
        fa = {0: v, 1: d, 2: v, 3: d}  # test-function factor of M, S, A, B
        fb = {0: v, 1: d, 2: d, 3: v}  # trial-function factor
        for op in range(4):
            ref = (fa[op][q][:, e:e + p + 1] * w[q][:, None]).T @ fb[op][q][:, e:e + p + 1]
            np.testing.assert_allclose(loc[e, op], ref, rtol=1e-13, atol=1e-14 * np.max(np.abs(ref)))
            dense[op, e:e + p + 1, e:e + p + 1] += loc[e, op]
    # summed over the elements the blocks give the matrices of the bands
    for op, X in enumerate(bspline.matrices_1d(n, p, breaks=br)):
        np.testing.assert_allclose(dense[op], X, rtol=0, atol=1e-13 * np.max(np.abs(X)))
