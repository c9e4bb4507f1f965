"""1D B-spline basis and the 1D matrices of the Kronecker factorisation (FP64).

Test infrastructure only (see ``oracle/__init__.py``).

Paper: section "Variational formulation", the definitions that follow eq.
(discrete4): M is the 1D mass matrix, S the 1D stiffness matrix, A the 1D
advection matrix with the derivative on the trial function and B the one with
the derivative on the test function.  Rows are test functions, columns trial
functions.  The paper states both A and B with the derivative on the trial
function; the integrands of eq. (dupa1abcd) put the derivative of B on the test
function, which is the reading used here, so B = A^T.  The basis is the open
knot vector of degree p with C^{p-1} continuity on (0, 1) ("quadratic C^1" in
the head experiment; linear example in the Appendix) on uniform elements, or
on the element boundaries given by ``breaks`` (the formulation admits any
knots: the matrices keep bandwidth p).

Pins (tests/test_oracle_bspline.py): closed-form interior stencils of the
uniform p = 2 matrices, partition of unity, S.1 = 0, A + A^T = e_N e_N^T -
e_1 e_1^T, symmetry of M and S, agreement of basis values with
scipy.interpolate.BSpline, and the Fourier symbol limit of the largest
eigenvalue of M^{-1} S.
"""
import numpy as np


def _breaks(n, breaks):
    """Element boundaries 0 = x_0 < x_1 < ... < x_n = 1 (uniform if None)."""
    if breaks is None:
        return np.linspace(0.0, 1.0, n + 1)
    b = np.asarray(breaks, dtype=np.float64)
    assert b.shape == (n + 1,) and b[0] == 0.0 and b[-1] == 1.0 and np.all(np.diff(b) > 0)
    return b


def knot_vector(n, p, breaks=None):
    """Open knot vector on [0, 1] with ``n`` elements, degree ``p``: the element
    boundaries (uniform unless ``breaks`` is given) with the end knots repeated
    p + 1 times."""
    return np.concatenate([np.zeros(p), _breaks(n, breaks), np.ones(p)])


def element_of(n, x0, breaks=None):
    """The element (knot span 0..n-1) that holds x0; a point on an element
    boundary belongs to the element on its right, x0 = 1 to the last one."""
    b = _breaks(n, breaks)
    return int(min(max(np.searchsorted(b, x0, side="right") - 1, 0), n - 1))


def n_basis(n, p):
    """Number of B-splines N = n + p."""
    return n + p


def eval_basis(n, p, x, elem, breaks=None):
    """Values and first derivatives of all N B-splines at points ``x``.

    ``elem[q]`` is the element (knot span 0..n-1) that contains ``x[q]``; it
    fixes the half-open span convention at knots.  Cox-de Boor recursion:
    N_{i,0} = 1 on span i, N_{i,k} = w1 N_{i,k-1} + w2 N_{i+1,k-1} with the
    usual 0/0 = 0 convention; the derivative of N_{i,p} is
    p/(U_{i+p}-U_i) N_{i,p-1} - p/(U_{i+p+1}-U_{i+1}) N_{i+1,p-1}.
    Returns (vals, ders), each of shape (len(x), N).
    """
    U = knot_vector(n, p, breaks)
    x = np.asarray(x, dtype=np.float64)
    elem = np.asarray(elem)
    nq = x.shape[0]
    nfun0 = len(U) - 1
    # degree 0: the span index of element e is e + p
    Nk = np.zeros((nq, nfun0))
    Nk[np.arange(nq), elem + p] = 1.0
    lower = None
    for k in range(1, p + 1):
        nf = len(U) - 1 - k
        new = np.zeros((nq, nf))
        for i in range(nf):
            d1 = U[i + k] - U[i]
            d2 = U[i + k + 1] - U[i + 1]
            if d1 > 0:
                new[:, i] += (x - U[i]) / d1 * Nk[:, i]
            if d2 > 0:
                new[:, i] += (U[i + k + 1] - x) / d2 * Nk[:, i + 1]
        lower = Nk
        Nk = new
    vals = Nk
    N = vals.shape[1]
    ders = np.zeros_like(vals)
    if p >= 1:
        for i in range(N):
            d1 = U[i + p] - U[i]
            d2 = U[i + p + 1] - U[i + 1]
            if d1 > 0:
                ders[:, i] += p / d1 * lower[:, i]
            if d2 > 0:
                ders[:, i] -= p / d2 * lower[:, i + 1]
    return vals, ders


def gauss_points(n, q, breaks=None):
    """Gauss-Legendre points and weights, ``q`` per element, on [0, 1].

    Returns (x, w, elem) for all n*q points.
    """
    g, gw = np.polynomial.legendre.leggauss(q)
    b = _breaks(n, breaks)
    h = np.diff(b)
    x = np.concatenate([0.5 * (b[e] + b[e + 1]) + 0.5 * h[e] * g for e in range(n)])
    w = np.concatenate([0.5 * h[e] * gw for e in range(n)])
    elem = np.repeat(np.arange(n), q)
    return x, w, elem


def matrices_1d(n, p, q=None, breaks=None):
    """The 1D matrices M, S, A, B (dense N x N, FP64).

    M[l, i] = int B_i B_l, S[l, i] = int B_i' B_l', A[l, i] = int B_i' B_l,
    B[l, i] = int B_i B_l' (= A[i, l]).  Row l is the test function.
    Gauss-Legendre with q = p + 1 points per element integrates the degree-2p
    integrands exactly.
    """
    if q is None:
        q = p + 1
    x, w, elem = gauss_points(n, q, breaks)
    v, d = eval_basis(n, p, x, elem, breaks)
    M = (v * w[:, None]).T @ v
    S = (d * w[:, None]).T @ d
    A = (v * w[:, None]).T @ d  # A[l, i] = sum_q w B_l B_i'
    B = (d * w[:, None]).T @ v  # B[l, i] = sum_q w B_l' B_i
    return M, S, A, B


def element_integrals(n, p, breaks=None):
    """G[r, e] = integral over element e of B_r (used by the material hats)."""
    x, w, elem = gauss_points(n, p + 1, breaks)
    v, _ = eval_basis(n, p, x, elem, breaks)
    G = np.zeros((v.shape[1], n))
    for e in range(n):
        sel = elem == e
        G[:, e] = (v[sel] * w[sel, None]).sum(axis=0)
    return G


def point_values(n, p, x0, breaks=None):
    """Values of all N B-splines at one point x0 in [0, 1]."""
    e = element_of(n, x0, breaks)
    v, _ = eval_basis(n, p, np.array([x0]), np.array([e]), breaks)
    return v[0]
