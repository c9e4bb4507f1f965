"""Pins of oracle.norms (function norms and plane evaluation)."""
import json
import os

import numpy as np
import pytest
import scipy.interpolate

from oracle import bspline, norms
from oracle import manufactured as mf
from oracle.banded import kron3

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def _greville(ne, p):
    U = bspline.knot_vector(ne, p)
    return np.array([U[i + 1:i + p + 1].mean() for i in range(ne + p)])


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_constant_and_linear_fields(p):
    n = (4, 5, 3)
    shp = (n[2] + p, n[1] + p, n[0] + p)
    one = np.ones(shp)
    zero = np.zeros(shp)
    # partition of unity: u = (1, 1, 1)
    l2, h1, hc = norms.field_norms([one, one, one], n, p)
    np.testing.assert_allclose([l2, h1, hc], [np.sqrt(3)] * 3, rtol=1e-13)
    # Greville coefficients reproduce u(x) = x: E = (0, x, 0), curl E = (0, 0, 1)
    gx = _greville(n[0], p)
    lin = np.broadcast_to(gx[None, None, :], shp).copy()
    l2, h1, hc = norms.field_norms([zero, lin, zero], n, p)
    np.testing.assert_allclose(l2, np.sqrt(1.0 / 3.0), rtol=1e-13)
    np.testing.assert_allclose(h1, np.sqrt(1.0 / 3.0 + 1.0), rtol=1e-13)
    np.testing.assert_allclose(hc, np.sqrt(1.0 / 3.0 + 1.0), rtol=1e-13)
    # and u = (y, 0, 0): gradient 1, curl (0, 0, -1)
    gy = _greville(n[1], p)
    liny = np.broadcast_to(gy[None, :, None], shp).copy()
    l2, h1, hc = norms.field_norms([liny, zero, zero], n, p)
    np.testing.assert_allclose([l2, h1, hc], [np.sqrt(1 / 3), np.sqrt(4 / 3), np.sqrt(4 / 3)], rtol=1e-13)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_norms_equal_matrix_quadratic_forms(p):
    n = (3, 4, 5)
    rng = np.random.default_rng(p)
    u = [rng.standard_normal((n[2] + p, n[1] + p, n[0] + p)) for _ in range(3)]
    Mx, Sx, Ax, Bx = bspline.matrices_1d(n[0], p)
    My, Sy, Ay, By = bspline.matrices_1d(n[1], p)
    Mz, Sz, Az, Bz = bspline.matrices_1d(n[2], p)
    l2 = sum(np.sum(c * kron3(Mx, My, Mz, c)) for c in u)
    grad = sum(np.sum(c * (kron3(Sx, My, Mz, c) + kron3(Mx, Sy, Mz, c) + kron3(Mx, My, Sz, c))) for c in u)
    got = norms.field_norms(u, n, p)
    np.testing.assert_allclose(got[0], np.sqrt(l2), rtol=1e-12)
    np.testing.assert_allclose(got[1], np.sqrt(l2 + grad), rtol=1e-12)
    # curl: squares of the six partial derivatives minus twice the three cross products
    # int d2 u3 d3 u2 = u2^T (M (x) A (x) B) u3 etc. (A: derivative on the trial function)
    E1, E2, E3 = u
    sq = (np.sum(E1 * (kron3(Mx, My, Sz, E1) + kron3(Mx, Sy, Mz, E1)))
          + np.sum(E2 * (kron3(Mx, My, Sz, E2) + kron3(Sx, My, Mz, E2)))
          + np.sum(E3 * (kron3(Mx, Sy, Mz, E3) + kron3(Sx, My, Mz, E3))))
    cross = (np.sum(E2 * kron3(Mx, Ay, Bz, E3)) + np.sum(E3 * kron3(Bx, My, Az, E1))
             + np.sum(E1 * kron3(Ax, By, Mz, E2)))
    np.testing.assert_allclose(got[2], np.sqrt(l2 + sq - 2 * cross), rtol=1e-12)


def test_projected_manufactured_solution_has_unit_norm():
    n, p = (16, 16, 16), 2
    mats = {"x": bspline.matrices_1d(16, p), "y": bspline.matrices_1d(16, p), "z": bspline.matrices_1d(16, p)}
    st = mf.project(lambda a, b, c: mf.u_A(a, b, c, 0.0), n, p, mats)
    nv = norms.norms(st, n, p)
    # ||u_A(., 0)|| = 1 over all six components (the paper's normalisation)
    total = np.hypot(nv[0], nv[1])
    assert abs(total - GOLD["norm_uA_t0"]["value"]) < 1e-4


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_plane_values_equal_scipy_bspline(axis):
    n, p = (5, 4, 6), 2
    rng = np.random.default_rng(axis)
    u = rng.standard_normal((n[2] + p, n[1] + p, n[0] + p))
    pos = 0.37
    got = norms.plane(u, n, p, axis, pos, 7, 5)
    others = [a for a in range(3) if a != axis]
    pts = {axis: [pos], others[0]: np.linspace(0, 1, 7), others[1]: np.linspace(0, 1, 5)}
    D = []
    for a in range(3):
        x = np.clip(np.array(pts[a], dtype=np.float64), 0.0, 1.0 - 1e-15)
        D.append(scipy.interpolate.BSpline.design_matrix(x, bspline.knot_vector(n[a], p), p).toarray())
    # value at (x, y, z) = sum_ijk u[k, j, i] Bx_i By_j Bz_k
    ref = np.einsum("kji,ai,bj,ck->cba", u, D[0], D[1], D[2])   # (z, y, x)
    ref = ref[:, :, 0] if axis == 0 else (ref[:, 0, :] if axis == 1 else ref[0, :, :])
    # (the end point 1.0 is clipped just inside the last span for scipy)
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12)
