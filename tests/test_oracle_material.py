"""Pins of oracle.material: row hats, conductivity coefficients, CFL limit."""
import numpy as np
import pytest

from oracle import material
from paper_2103_06998_gb300 import inputs
from bruteforce import Dense3D


def test_uniform_material_gives_uniform_hat():
    n, p = (5, 4, 3), 2
    f = np.full((3, 4, 5), 7.25)
    np.testing.assert_allclose(material.row_hats(f, n, p), 7.25, rtol=1e-14)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_hat_equals_3d_quadrature(p):
    # eps^_rst = int eps B_rst / int B_rst, by a full 3D Gauss sum
    n = (3, 4, 2)
    eps, _, sigma = inputs.random_material(n, 5)
    D = Dense3D(n, p)
    np.testing.assert_allclose(material.row_hats(eps, n, p), D.hat(eps), rtol=1e-12)
    np.testing.assert_allclose(material.row_hats(sigma, n, p), D.hat(sigma), rtol=1e-12, atol=1e-15)


def test_sigma_zero_reduces_to_paper_constants():
    eps = np.array([1.0, 12.0, 50.0])
    mu = np.array([1.0, 2.0, 1.0])
    tau = 0.03
    a, b, c, d = material.coefficients(eps, mu, np.zeros(3), tau)
    np.testing.assert_array_equal(a, 1.0)
    np.testing.assert_allclose(b, tau / (2 * eps), rtol=1e-15)
    np.testing.assert_allclose(c, tau ** 2 / (4 * eps * mu), rtol=1e-15)
    np.testing.assert_allclose(d, tau / (2 * mu), rtol=1e-15)


def test_conductive_decay_is_second_order():
    # a = (1 - alpha)/(1 + alpha) approximates exp(-sigma tau / (2 eps)), the exact
    # decay of eps E' = -sigma E over a half step, with error O(alpha^3).
    eps, sig = 2.0, 0.7
    errs = []
    for tau in (0.1, 0.05, 0.025):
        a, _, _, _ = material.coefficients(np.array([eps]), np.array([1.0]), np.array([sig]), tau)
        errs.append(abs(a[0] - np.exp(-sig * tau / (2 * eps))))
    assert errs[0] / errs[1] > 7.5 and errs[1] / errs[2] > 7.5


def test_lambda_max_tends_to_symbol_limit():
    # Fourier symbol of S/M for uniform quadratic B-splines at theta = pi:
    # S = (1 + 2/3 - 1/3) / h^2-scale = 4/3, M = (66 - 52 + 2)/120 = 2/15 -> 10.
    n = 64
    lam = material.lambda_max(n, 2)
    assert abs(lam / n ** 2 - 10.0) < 0.05
    # and linear elements: 12 (= 4 / (1/3))
    assert abs(material.lambda_max(n, 1) / n ** 2 - 12.0) < 0.05


def test_cfl_dt_uniform():
    n = (16, 16, 16)
    eh = np.ones((18, 18, 18))
    dt = material.cfl_dt(n, 2, eh, eh)
    lam = material.lambda_max(16, 2)
    np.testing.assert_allclose(dt, 2.0 / np.sqrt(3 * lam), rtol=1e-14)
    assert 0.35 / 16 < dt < 0.38 / 16


@pytest.mark.parametrize("sig", [0.0, 40.0, 300.0])   # alpha = 0, 0.2, 1.5
def test_conductive_half_step_closed_form(sig):
    """One E half step (half step 1, component E1) in uniform eps, mu, sigma
    against the closed form of the time-discrete model, per eigenmode.

    Model (the conductivity reading): eps E1' + sigma E1 = d2 H3 - d3 H2 and
    mu H3' = d2 E1 - d1 E2.  The first split half step takes the sigma term by
    the trapezoidal rule and d2 H3 implicitly at the new level, with H3 at the
    new level from its own half step:
        eps (E+ - E0) / (tau/2) + sigma (E+ + E0) / 2 = d2 H3+,
        H3+ = H30 + tau / (2 mu) d2 E+            (E2 = 0, H2 = 0).
    On the y-eigenmodes v_k of the Dirichlet-reduced pencil S_D v = lam M_D v
    (d2 d2 -> -lam) with E0 = X (x) v_j (x) Z and d2 H30 -> M^-1 A Y this gives,
    with alpha = sigma tau / (4 eps) and beta = tau^2 / (4 eps mu),
        E+ = X (x) [ (1 - alpha) / (1 + alpha + beta lam_j) v_j
                     + sum_k (tau / (2 eps)) g_k / (1 + alpha + beta lam_k) v_k ] (x) Z,
    g_k = v_k^T (A Y)_interior (M_D-orthonormal v_k).  The eigenpairs come from
    scipy.linalg.eigh, independent of the oracle's line solves, and nothing
    here uses the oracle's a, b, c: dropping the factor (1 + alpha) from b or
    from c, or the sign of alpha in a, changes E+ by far more than the
    tolerance (checked below on the sigma > 0 cases).
    """
    import scipy.linalg
    from oracle import bspline
    from oracle import maxwell_adi as ma

    n, p, tau = (3, 7, 4), 2, 0.05
    eps_v, mu_v = 2.5, 1.7
    shp_e = (n[2], n[1], n[0])
    prob = ma.make_problem(n, p, tau, np.full(shp_e, eps_v), np.full(shp_e, mu_v), np.full(shp_e, sig))
    Nx, Ny, Nz = n[0] + p, n[1] + p, n[2] + p
    My, Sy, Ay, _ = bspline.matrices_1d(n[1], p)
    lam, V = scipy.linalg.eigh(Sy[1:-1, 1:-1], My[1:-1, 1:-1])   # V^T M_D V = I
    rng = np.random.default_rng(4)
    X = rng.standard_normal(Nx)                  # E1 and H3 free in x
    Z = rng.standard_normal(Nz)
    Z[0] = Z[-1] = 0.0                           # E1 tangential, H3 normal in z
    Y = rng.standard_normal(Ny)                  # H3 free in y
    j = 2
    vj = np.zeros(Ny)
    vj[1:-1] = V[:, j]
    E1 = np.einsum("k,j,i->kji", Z, vj, X)
    H3 = np.einsum("k,j,i->kji", Z, Y, X)
    zero = np.zeros_like(E1)
    alpha = sig * tau / (4 * eps_v)
    beta = tau * tau / (4 * eps_v * mu_v)
    g = V.T @ (Ay @ Y)[1:-1]

    def closed(alpha_a, alpha_b, alpha_c):
        # a (1 + alpha_a) = 1 - alpha, b = tau/(2 eps (1 + alpha_b)), c = beta / (1 + alpha_c)
        a = (1 - alpha) / (1 + alpha_a)
        b = tau / (2 * eps_v * (1 + alpha_b))
        c = beta / (1 + alpha_c)
        y = V @ ((a * (np.arange(len(lam)) == j) + b * g) / (1 + c * lam))
        out = np.zeros(Ny)
        out[1:-1] = y
        return np.einsum("k,j,i->kji", Z, out, X)

    expect = np.zeros(Ny)
    expect[1:-1] = V @ (((1 - alpha) * (np.arange(len(lam)) == j) + tau / (2 * eps_v) * g)
                        / (1 + alpha + beta * lam))
    expect = np.einsum("k,j,i->kji", Z, expect, X)
    # the closed form written with the paper-style factors agrees with the physical one
    np.testing.assert_allclose(closed(alpha, alpha, alpha), expect, rtol=1e-12, atol=1e-14)

    got = ma.solve_E(prob, 1, ma.rhs_E(prob, 1, [E1, zero, zero], [zero, zero, H3], 0.0))[0]
    scale = np.abs(expect).max()
    assert np.abs(got - expect).max() <= 1e-12 * scale
    if sig > 0:
        # the mistakes this pin exists for: (1 + alpha) missing in b, in c, or in a
        for wrong in (closed(alpha, 0.0, alpha), closed(alpha, alpha, 0.0), closed(0.0, alpha, alpha)):
            assert np.abs(wrong - expect).max() > 1e-3 * scale
