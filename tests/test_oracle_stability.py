"""Stability pins: unconditional stability for uniform material (spectral
radius of the one-step map), bounded energy at tau far above the explicit limit,
and the decay of the heterogeneous head-map workload at 4x the limit."""
import numpy as np
import pytest

from oracle import maxwell_adi as ma
from oracle import material
from oracle.banded import kron3
from paper_2103_06998_gb300 import inputs


def _amplification(prob):
    shp = prob.shape
    Nc = int(np.prod(shp))
    cols = []
    for k in range(6 * Nc):
        v = np.zeros(6 * Nc)
        v[k] = 1.0
        st = ma.apply_dirichlet([v[i * Nc:(i + 1) * Nc].reshape(shp) for i in range(6)])
        out = ma.step(prob, st, 0.0)
        cols.append(np.concatenate([u.ravel() for u in out]))
    return np.array(cols).T


@pytest.mark.parametrize("n,p", [((3, 3, 3), 2), ((2, 3, 2), 3)])
@pytest.mark.parametrize("fac", [1.0, 20.0, 1000.0])
def test_spectral_radius_at_most_one_uniform(n, p, fac):
    one = np.ones((n[2] + p, n[1] + p, n[0] + p))
    dt = material.cfl_dt(n, p, one, one)
    G = _amplification(ma.make_problem(n, p, fac * dt))
    rho = np.abs(np.linalg.eigvals(G)).max()
    assert rho < 1.0 + 1e-9


def _energy(prob, st):
    Mx, My, Mz = prob.mats["x"][0], prob.mats["y"][0], prob.mats["z"][0]
    return sum(np.sum(u * kron3(Mx, My, Mz, u)) for u in st)


@pytest.mark.parametrize("fac", [20.0, 100.0])
def test_no_growth_far_above_cfl_uniform(fac):
    n, p = (8, 8, 8), 2
    one = np.ones((10, 10, 10))
    prob = ma.make_problem(n, p, fac * material.cfl_dt(n, p, one, one))
    st = ma.apply_dirichlet(inputs.random_fields(prob.shape, 1))
    e = []
    for _ in range(300):
        st = ma.step(prob, st, 0.0)
        e.append(_energy(prob, st))
    e = np.array(e)
    assert np.all(np.isfinite(e))
    assert e[-100:].max() <= 1.05 * e[:100].max()


def test_head_map_decays_at_four_times_cfl():
    n, p = (8, 8, 8), 2
    eps, mu, sigma, _ = inputs.head_map(n, 2103)
    eh = material.row_hats(eps, n, p)
    dt = material.cfl_dt(n, p, eh, material.row_hats(mu, n, p))
    prob = ma.make_problem(n, p, 4.0 * dt, eps, mu, sigma)
    st = ma.apply_dirichlet(inputs.random_fields(prob.shape, 1))
    e0 = _energy(prob, st)
    for _ in range(300):
        st = ma.step(prob, st, 0.0)
    assert _energy(prob, st) < e0
