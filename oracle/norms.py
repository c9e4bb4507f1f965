"""Function norms of the discrete fields and point evaluation on a plane (FP64).

Test infrastructure only (see ``oracle/__init__.py``).

The paper reports, for the head simulation, the L2 and H1 norms of the
electric and magnetic fields over time (section "Incorporating non-regular
material data", Figure head_norms) and, for the manufactured solution, errors in
the L2 and H(curl) norms (section "Numerical code verification with
manufactured solution"); its field pictures are cross sections along an OYZ
plane (Figures head2, head3).  Here the three norms of a vector field
u = (u1, u2, u3) given by B-spline coefficients are their definitions written
as integrals over the unit cube, evaluated by Gauss quadrature with p + 3
points per element and axis (exact for these polynomial integrands):

    ||u||_L2^2     = sum_i int u_i^2
    ||u||_H1^2     = ||u||_L2^2 + sum_i int |grad u_i|^2
    ||u||_Hcurl^2  = ||u||_L2^2 + int |curl u|^2

``plane`` evaluates one coefficient array at the points of a uniform grid on the
plane {x_axis = pos}: u_j = j / (nu - 1), v_k = k / (nv - 1) over the two other
axes in x, y, z order, returned as out[k, j].

Pins (tests/test_oracle_norms.py): coefficients all ones give u = 1 (partition
of unity): L2 = 1, no gradient, no curl; the Greville-abscissa coefficients give
u(x) = x exactly: int x^2 = 1/3, |grad| = 1, and the curl of (0, x, 0) is
(0, 0, 1); the L2 norm equals the mass-matrix quadratic form c^T (M(x)M(x)M) c
and the gradient part c^T (S(x)M(x)M + M(x)S(x)M + M(x)M(x)S) c (matrices from
oracle.bspline, a different route than the pointwise evaluation here); the
projected manufactured solution u_A at t = 0 has norm 1 up to the projection
error (the paper normalises ||u_A(., 0)|| = 1); point values on a plane equal
scipy.interpolate.BSpline.
"""
import numpy as np

from . import bspline
from .banded import apply_1d
from .manufactured import evaluate, quad_grid


def _weights(grid):
    gx, gy, gz = grid
    return np.einsum("k,j,i->kji", gz[1], gy[1], gx[1])


def field_norms(u, n, p):
    """(L2, H1, H(curl)) norms of the vector field with coefficients u[0..2]."""
    grid = quad_grid(n, p)
    W = _weights(grid)
    val = [evaluate(u[i], grid) for i in range(3)]
    # d[i][a] = d u_i / d x_a
    d = [[evaluate(u[i], grid, tuple(int(a == k) for k in range(3))) for a in range(3)] for i in range(3)]
    l2 = sum(np.sum(W * v * v) for v in val)
    grad = sum(np.sum(W * d[i][a] ** 2) for i in range(3) for a in range(3))
    curl = (d[2][1] - d[1][2], d[0][2] - d[2][0], d[1][0] - d[0][1])
    c2 = sum(np.sum(W * c * c) for c in curl)
    return np.sqrt(l2), np.sqrt(l2 + grad), np.sqrt(l2 + c2)


def norms(state, n, p):
    """[L2(E), L2(H), H1(E), H1(H), Hcurl(E), Hcurl(H)] of a 6-component state."""
    e = field_norms(state[:3], n, p)
    h = field_norms(state[3:], n, p)
    return np.array([e[0], h[0], e[1], h[1], e[2], h[2]])


def _basis_at(ne, p, pts):
    elem = np.minimum(np.floor(np.asarray(pts) * ne).astype(int), ne - 1)
    v, _ = bspline.eval_basis(ne, p, np.asarray(pts, dtype=np.float64), elem)
    return v   # (len(pts), N)


def plane(u, n, p, axis, pos, nu, nv):
    """Values of the coefficient array u (Nz, Ny, Nx) on the plane x_axis = pos."""
    others = [a for a in range(3) if a != axis]
    pts = {axis: np.array([pos]), others[0]: np.linspace(0.0, 1.0, nu), others[1]: np.linspace(0.0, 1.0, nv)}
    Bx = _basis_at(n[0], p, pts[0])
    By = _basis_at(n[1], p, pts[1])
    Bz = _basis_at(n[2], p, pts[2])
    vals = apply_1d(Bx, apply_1d(By, apply_1d(Bz, u, "z"), "y"), "x")   # (pz, py, px)
    if axis == 0:
        return vals[:, :, 0]          # [z][y]: v = z, u = y
    if axis == 1:
        return vals[:, 0, :]          # [z][x]
    return vals[0, :, :]              # [y][x]
