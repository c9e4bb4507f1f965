"""Pins of oracle.banded: Kronecker application and banded line solves."""
import numpy as np
import scipy.linalg

from oracle import banded, bspline
from paper_2103_06998_gb300 import inputs


def test_kron3_equals_numpy_kron():
    rng = np.random.default_rng(0)
    X, Y, Z = rng.standard_normal((5, 5)), rng.standard_normal((4, 4)), rng.standard_normal((3, 3))
    u = rng.standard_normal((3, 4, 5))          # (Nz, Ny, Nx)
    ref = np.kron(np.kron(Z, Y), X) @ u.ravel()  # x fastest in the flat index
    np.testing.assert_allclose(banded.kron3(X, Y, Z, u).ravel(), ref, atol=1e-13)


def _dense_line(base, stiff, c):
    return base + c[:, None] * stiff


def test_solve_lines_against_dense_and_scipy():
    n, p = 6, 2
    M, S, _, _ = bspline.matrices_1d(n, p)
    N = n + p
    shp = (5, 4, N)
    r = inputs.random_fields(shp, 11)[0]
    c = 0.01 + inputs.random_fields(shp, 12)[1] ** 2
    for dirichlet in (False, True):
        x = banded.solve_lines(M, r, "x", p, dirichlet, stiff=S, coef=c)
        for k in range(shp[0]):
            for j in range(shp[1]):
                A = _dense_line(M, S, c[k, j])
                if dirichlet:
                    ref = np.zeros(N)
                    ref[1:-1] = np.linalg.solve(A[1:-1, 1:-1], r[k, j, 1:-1])
                else:
                    ref = np.linalg.solve(A, r[k, j])
                np.testing.assert_allclose(x[k, j], ref, rtol=1e-11, atol=1e-12)
    # constant matrix: scipy.linalg.solve_banded on every line along z
    rz = inputs.random_fields((N, 3, 4), 13)[2]
    xz = banded.solve_lines(M, rz, "z", p, False)
    ab = np.zeros((2 * p + 1, N))
    for d in range(-p, p + 1):
        diag = np.diagonal(M, d)
        if d >= 0:
            ab[p - d, d:] = diag
        else:
            ab[p - d, :d] = diag
    ref = scipy.linalg.solve_banded((p, p), ab, rz.reshape(N, -1)).reshape(rz.shape)
    np.testing.assert_allclose(xz, ref, rtol=1e-11, atol=1e-12)


def test_apply_along_each_axis():
    rng = np.random.default_rng(1)
    u = rng.standard_normal((3, 4, 5))
    for ax, L in (("x", 5), ("y", 4), ("z", 3)):
        Mt = rng.standard_normal((L, L))
        out = banded.apply_1d(Mt, u, ax)
        axis = banded.AXIS[ax]
        ref = np.moveaxis(np.einsum("li,...i->...l", Mt, np.moveaxis(u, axis, -1)), -1, axis)
        np.testing.assert_allclose(out, ref, atol=1e-13)
