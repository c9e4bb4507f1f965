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


@pytest.mark.parametrize("p", [1, 2, 3])
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
