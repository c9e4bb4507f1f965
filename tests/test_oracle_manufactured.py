"""Manufactured-solution pins of the oracle: the paper's error bounds on 16^3,
second order in tau, and u_A itself (exact solution, unit norm)."""
import json
import os

import numpy as np
import pytest

from oracle import manufactured as mf
from oracle import maxwell_adi as ma

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def test_gamma_and_unit_norm():
    np.testing.assert_allclose(mf.GAMMA, GOLD["gamma"]["value"], rtol=1e-15)
    # ||u_A(.,0)||_L2 = 1 by a fine Gauss sum of the exact field
    g, w = np.polynomial.legendre.leggauss(12)
    x = 0.5 + 0.5 * g
    w = 0.5 * w
    X3, X2, X1 = np.meshgrid(x, x, x, indexing="ij")
    W = np.einsum("k,j,i->kji", w, w, w)
    u = mf.u_A(X1, X2, X3, 0.0)
    np.testing.assert_allclose(np.sqrt(sum(np.sum(W * c ** 2) for c in u)), GOLD["norm_uA_t0"]["value"], rtol=1e-12)


def test_uA_solves_maxwell_with_pec():
    # dE/dt = curl H, dH/dt = -curl E (eps = mu = 1), div E = div H = 0,
    # E x n = 0 and H . n = 0 on the faces -- checked by central differences.
    rng = np.random.default_rng(0)
    P = rng.uniform(0.05, 0.95, size=(3, 40))
    t = 0.37
    h = 1e-5
    f = lambda x1, x2, x3, tt: np.array(mf.u_A(x1, x2, x3, tt))
    x1, x2, x3 = P
    dt = (f(x1, x2, x3, t + h) - f(x1, x2, x3, t - h)) / (2 * h)
    def d(ax):
        e = np.zeros(3)
        e[ax] = h
        return (f(x1 + e[0], x2 + e[1], x3 + e[2], t) - f(x1 - e[0], x2 - e[1], x3 - e[2], t)) / (2 * h)
    D = [d(0), d(1), d(2)]
    curl = lambda o: np.array([D[1][o + 2] - D[2][o + 1], D[2][o] - D[0][o + 2], D[0][o + 1] - D[1][o]])
    np.testing.assert_allclose(dt[:3], curl(3), atol=1e-7)
    np.testing.assert_allclose(dt[3:], -curl(0), atol=1e-7)
    np.testing.assert_allclose(D[0][0] + D[1][1] + D[2][2], 0, atol=1e-7)
    np.testing.assert_allclose(D[0][3] + D[1][4] + D[2][5], 0, atol=1e-7)
    s = rng.uniform(0, 1, size=40)
    for face in (0.0, 1.0):
        u = f(face + 0 * s, s, s[::-1], t)    # x1 face: E2 = E3 = 0, H1 = 0
        np.testing.assert_allclose(u[[1, 2, 3]], 0, atol=1e-14)
        u = f(s, face + 0 * s, s[::-1], t)    # x2 face: E1 = E3 = 0, H2 = 0
        np.testing.assert_allclose(u[[0, 2, 4]], 0, atol=1e-14)
        u = f(s, s[::-1], face + 0 * s, t)    # x3 face: E1 = E2 = 0, H3 = 0
        np.testing.assert_allclose(u[[0, 1, 5]], 0, atol=1e-14)


def _run_errors(nsteps, n=(16, 16, 16), p=2, samples=10):
    tau = 1.0 / nsteps
    prob = ma.make_problem(n, p, tau)
    st = mf.project(lambda a, b, c: mf.u_A(a, b, c, 0.0), n, p, prob.mats)
    t = 0.0
    worst = np.zeros(4)
    every = max(1, nsteps // samples)
    for k in range(nsteps):
        st = ma.step(prob, st, t)
        t += tau
        if (k + 1) % every == 0:
            worst = np.maximum(worst, mf.errors(st, n, p, t))
    return worst   # (L2 E, L2 H, Hcurl E, Hcurl H), max over sampled t in (0, 1]


def test_paper_bounds_tau_one_tenth_and_order_two():
    e10 = _run_errors(10)
    assert e10[0] < GOLD["l2_error_bound"]["tau_1_10"] and e10[1] < GOLD["l2_error_bound"]["tau_1_10"]
    assert e10[2] < GOLD["hcurl_error_bound"]["tau_1_10"] and e10[3] < GOLD["hcurl_error_bound"]["tau_1_10"]
    e20 = _run_errors(20)
    e40 = _run_errors(40)
    for a, b in ((e10, e20), (e20, e40)):
        order = np.log2(a[:2] / b[:2])
        assert np.all((order > 1.8) & (order < 2.2)), order


def test_paper_bounds_tau_1_over_1280():
    e = _run_errors(1280)
    assert e[0] < GOLD["l2_error_bound"]["tau_1_1280"] and e[1] < GOLD["l2_error_bound"]["tau_1_1280"], e
    assert e[2] < GOLD["hcurl_error_bound"]["tau_1_1280"] and e[3] < GOLD["hcurl_error_bound"]["tau_1_1280"], e


def test_spatial_order_p_plus_one():
    # Projection error of u_A(., 0) decays like h^(p+1) in L2 (approximation theory).
    errs = []
    for ne in (4, 8, 16):
        n = (ne, ne, ne)
        prob = ma.make_problem(n, 2, 0.1)
        st = mf.project(lambda a, b, c: mf.u_A(a, b, c, 0.0), n, 2, prob.mats)
        errs.append(mf.errors(st, n, 2, 0.0)[0])
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all((rates > 2.6) & (rates < 3.4)), rates
