"""1D B-spline basis and the 1D matrices of the Kronecker factorisation (FP64).

Test infrastructure only (see ``oracle/__init__.py``).

Paper: section "Variational formulation", the definitions that follow eq.
(discrete4): M is the 1D mass matrix, S the 1D stiffness matrix, A the 1D
advection matrix with the derivative on the trial function and B the one with
the derivative on the test function.  Rows are test functions, columns trial
functions.  The paper states both A and B with the derivative on the trial
function; the integrands of eq. (dupa1abcd) put the derivative of B on the test
function, which is the reading used here, so B = A^T.  The basis is the open
uniform knot vector of degree p with C^{p-1} continuity on (0, 1) ("quadratic
C^1" in the head experiment; linear example in the Appendix).

Pins (tests/test_oracle_bspline.py): closed-form interior stencils of the
uniform p = 2 matrices, partition of unity, S.1 = 0, A + A^T = e_N e_N^T -
e_1 e_1^T, symmetry of M and S, agreement of basis values with
scipy.interpolate.BSpline, and the Fourier symbol limit of the largest
eigenvalue of M^{-1} S.
"""
import numpy as np


def knot_vector(n, p):
    """Open uniform knot vector on [0, 1] with ``n`` elements, degree ``p``."""
    return np.concatenate([np.zeros(p), np.linspace(0.0, 1.0, n + 1), np.ones(p)])


def n_basis(n, p):
    """Number of B-splines N = n + p."""
    return n + p


def eval_basis(n, p, x, elem):
    """Values and first derivatives of all N B-splines at points ``x``.

    ``elem[q]`` is the element (knot span 0..n-1) that contains ``x[q]``; it
    fixes the half-open span convention at knots.  Cox-de Boor recursion:
    N_{i,0} = 1 on span i, N_{i,k} = w1 N_{i,k-1} + w2 N_{i+1,k-1} with the
    usual 0/0 = 0 convention; the derivative of N_{i,p} is
    p/(U_{i+p}-U_i) N_{i,p-1} - p/(U_{i+p+1}-U_{i+1}) N_{i+1,p-1}.
    Returns (vals, ders), each of shape (len(x), N).
    """
    U = knot_vector(n, p)
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


def gauss_points(n, q):
    """Gauss-Legendre points and weights, ``q`` per element, on [0, 1].

    Returns (x, w, elem) for all n*q points.
    """
    g, gw = np.polynomial.legendre.leggauss(q)
    h = 1.0 / n
    x = np.concatenate([(e + 0.5) * h + 0.5 * h * g for e in range(n)])
    w = np.concatenate([0.5 * h * gw for _ in range(n)])
    elem = np.repeat(np.arange(n), q)
    return x, w, elem


def matrices_1d(n, p, q=None):
    """The 1D matrices M, S, A, B (dense N x N, FP64).

    M[l, i] = int B_i B_l, S[l, i] = int B_i' B_l', A[l, i] = int B_i' B_l,
    B[l, i] = int B_i B_l' (= A[i, l]).  Row l is the test function.
    Gauss-Legendre with q = p + 1 points per element integrates the degree-2p
    integrands exactly.
    """
    if q is None:
        q = p + 1
    x, w, elem = gauss_points(n, q)
    v, d = eval_basis(n, p, x, elem)
    M = (v * w[:, None]).T @ v
    S = (d * w[:, None]).T @ d
    A = (v * w[:, None]).T @ d  # A[l, i] = sum_q w B_l B_i'
    B = (d * w[:, None]).T @ v  # B[l, i] = sum_q w B_l' B_i
    return M, S, A, B


def element_integrals(n, p):
    """G[r, e] = integral over element e of B_r (used by the material hats)."""
    x, w, elem = gauss_points(n, p + 1)
    v, _ = eval_basis(n, p, x, elem)
    G = np.zeros((v.shape[1], n))
    for e in range(n):
        sel = elem == e
        G[:, e] = (v[sel] * w[sel, None]).sum(axis=0)
    return G


def point_values(n, p, x0):
    """Values of all N B-splines at one point x0 in [0, 1]."""
    e = min(int(np.floor(x0 * n)), n - 1)
    v, _ = eval_basis(n, p, np.array([x0]), np.array([e]))
    return v[0]
