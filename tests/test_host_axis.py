"""The 1D matrices of one axis as the library builds them on the host
(adi_axis_bands; no GPU): the band form of the mass, stiffness and mixed
matrices defined after eq. discrete4 (section "Variational formulation"),
against the oracle's dense matrices, the closed-form interior stencils of
cardinal B-splines, the symmetry B = A^T, and the interior rows the kernels
replace by one constant stencil, on uniform and non-uniform elements.
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
