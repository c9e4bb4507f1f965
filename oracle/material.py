"""Per-test-function material, conductivity coefficients, explicit CFL (FP64).

Test infrastructure only (see ``oracle/__init__.py``).

Paper, section "Incorporating non-regular material data into isogeometric
alternating-direction solver": the material (tau^, eps^, mu^) is attached to the
test B-spline B_r(x) B_s(y) B_t(z); row rst of each of the three 1D systems and
of the right-hand side uses the hat values.  The paper does not say how voxel
(per-element) data become per-test-function values.  Reading used here: the
support-weighted mean

    eps^_rst = sum_e eps_e W_e / sum_e W_e,   W_e = prod_d int_{e_d} B_{r_d},

(exact for uniform data), the same rule for mu^ and sigma^, and tau^ = tau.

Conductivity is not in the paper's equations.  Reading: eps dE/dt + sigma E =
curl H - J, with sigma E taken trapezoidally over each half step.  With
alpha = sigma^ tau / (4 eps^) the E rows are divided by (1 + alpha):

    a = (1 - alpha) / (1 + alpha)      (weight of M E_old)
    b = tau / (2 eps^ (1 + alpha))     (weight of the curl and source terms)
    c = tau^2 / (4 eps^ mu^ (1 + alpha))  (weight of S on the left, R on the right)
    d = tau / (2 mu^)                  (weight of the curl terms in the H rows)

so that at sigma = 0 these are 1, tau/(2 eps), tau^2/(4 eps mu), tau/(2 mu) of
eqs. (discrete1)-(discrete4).

Explicit CFL limit (not in the paper; used only to choose tau):
dt_CFL = 2 / (c_max sqrt(lambda_x + lambda_y + lambda_z)), lambda_d the largest
eigenvalue of M_D^{-1} S_D on axis d (Dirichlet-reduced), c_max =
1/sqrt(min eps^ mu^).

Pins (tests/test_oracle_material.py): uniform data give the uniform value; the
hat equals a brute-force 3D quadrature of int eps B_rst / int B_rst; sigma = 0
reduces a, b, c, d to the paper's constants; for sigma > 0, one E half step in
uniform material reproduces, mode by mode, the closed-form amplification
(1 - alpha) / (1 + alpha + beta lam) and curl response (tau / 2 eps) /
(1 + alpha + beta lam) of the time-discrete model (a missing (1 + alpha) in a,
b or c fails it); lambda h^2 tends to 10 for p = 2 (the Fourier symbol of S / M
at theta = pi).
"""
import numpy as np
import scipy.linalg

from . import bspline
from .banded import apply_1d


def row_hats(field, n, p, breaks=None):
    """Support-weighted mean of per-element ``field`` (nz, ny, nx) per row;
    breaks: per-axis element boundaries (x, y, z) or None for uniform."""
    nx, ny, nz = n
    bx, by, bz = breaks if breaks is not None else (None, None, None)
    Gx = bspline.element_integrals(nx, p, bx)
    Gy = bspline.element_integrals(ny, p, by)
    Gz = bspline.element_integrals(nz, p, bz)
    num = apply_1d(Gx, apply_1d(Gy, apply_1d(Gz, field, "z"), "y"), "x")
    one = np.ones_like(field)
    den = apply_1d(Gx, apply_1d(Gy, apply_1d(Gz, one, "z"), "y"), "x")
    return num / den


def coefficients(eps_hat, mu_hat, sigma_hat, tau):
    """Row coefficients (a, b, c, d) of the E and H sub-steps."""
    alpha = sigma_hat * tau / (4.0 * eps_hat)
    a = (1.0 - alpha) / (1.0 + alpha)
    b = tau / (2.0 * eps_hat * (1.0 + alpha))
    c = tau * tau / (4.0 * eps_hat * mu_hat * (1.0 + alpha))
    d = tau / (2.0 * mu_hat) * np.ones_like(eps_hat)
    return a, b, c, d


def lambda_max(n, p, breaks=None):
    """Largest eigenvalue of M_D^{-1} S_D (Dirichlet-reduced) on one axis."""
    M, S, _, _ = bspline.matrices_1d(n, p, breaks=breaks)
    w = scipy.linalg.eigh(S[1:-1, 1:-1], M[1:-1, 1:-1], eigvals_only=True)
    return float(w.max())


def cfl_dt(n, p, eps_hat, mu_hat, breaks=None):
    nx, ny, nz = n
    bx, by, bz = breaks if breaks is not None else (None, None, None)
    lam = lambda_max(nx, p, bx) + lambda_max(ny, p, by) + lambda_max(nz, p, bz)
    cmax = 1.0 / np.sqrt(np.min(eps_hat * mu_hat))
    return 2.0 / (cmax * np.sqrt(lam))
