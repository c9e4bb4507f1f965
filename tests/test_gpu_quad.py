"""The quad reading of the material (ADI_RHS_QUAD: per-element coefficients
inside the right-hand side integrals, element-wise kernel) against the FP64
oracle's quad form, element by element; and equal to the row reading for
uniform material on the GPU as well.

Tolerances per step: those of the row reading (tests/test_gpu_parity.py); the
(p+1)^3 element contributions of each coefficient are summed in FP64."""
import numpy as np
import pytest

from oracle import maxwell_adi as ma
from oracle import material
from paper_2103_06998_gb300 import inputs
from parity_check import assert_parity
from test_gpu_parity import tol

pytestmark = pytest.mark.gpu


def _adi():
    from paper_2103_06998_gb300 import adi
    return adi


def _mat(n, kind):
    if kind == "head":
        return inputs.head_map(n, 2103)[:3]
    return inputs.random_material(n, 7, mu_range=(1.0, 2.0))


CASES = [((21, 13, 10), 2, "head"), ((9, 12, 7), 1, "random"), ((10, 9, 11), 3, "random"), ((17, 9, 12), 3, "head")]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("n,p,kind", CASES)
def test_quad_step_matches_oracle(n, p, kind, prec):
    eps, mu, sigma = _mat(n, kind)
    tau = 0.03
    prob = ma.make_problem(n, p, tau, eps, mu, sigma, rhs_material="quad")
    src = inputs.dipole(2103)
    ma.set_source(prob, src["x0"], src["comp"], src["amp"], src["f0"], src["t0"], src["s"])
    st = ma.apply_dirichlet(list(inputs.random_fields(prob.shape, 3)))
    ref, _ = ma.run(prob, st, 1.6, 1)
    s = _adi().Solver(n, p, tau, eps, mu, sigma, precision=prec, rhs_material="quad")
    s.factor()
    s.set_source(src["x0"], src["comp"], src["amp"], src["f0"], src["t0"], src["s"])
    s.set_fields(np.array(st), 1.6)
    s.step(1)
    got, t = s.fields()
    s.close()
    assert abs(t - (1.6 + tau)) < 1e-12
    # per step from an identical state
    assert_parity(got, ref, tol(prec, p, kind), what="quad %s p=%d %s" % (prec, p, kind))
    # the quad reading is a different discretisation than the row one on this material
    row = ma.make_problem(n, p, tau, eps, mu, sigma)
    ma.set_source(row, src["x0"], src["comp"], src["amp"], src["f0"], src["t0"], src["s"])
    ref_row, _ = ma.run(row, st, 1.6, 1)
    num = sum(np.sum((a - b) ** 2) for a, b in zip(ref_row, ref))
    assert np.sqrt(num / sum(np.sum(b ** 2) for b in ref)) > 1e-4


def test_quad_64_head_dipole():
    n, p = (64, 64, 64), 2
    eps, mu, sigma, _ = inputs.head_map(n, 2103)
    tau = 4.0 * material.cfl_dt(n, p, material.row_hats(eps, n, p), material.row_hats(mu, n, p))
    prob = ma.make_problem(n, p, tau, eps, mu, sigma, rhs_material="quad")
    src = inputs.dipole(2103)
    ma.set_source(prob, src["x0"], src["comp"], src["amp"], src["f0"], src["t0"], src["s"])
    st = ma.apply_dirichlet(list(inputs.random_fields(prob.shape, 5)))
    ref, _ = ma.run(prob, st, 1.6, 1)
    s = _adi().Solver(n, p, tau, eps, mu, sigma, rhs_material="quad")
    s.factor()
    s.set_source(src["x0"], src["comp"], src["amp"], src["f0"], src["t0"], src["s"])
    s.set_fields(np.array(st), 1.6)
    s.step(1)
    got, _ = s.fields()
    s.close()
    assert_parity(got, ref, tol("fp32", p), what="quad 64^3")


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_quad_equals_row_for_uniform_material(prec):
    adi = _adi()
    n, p = (14, 11, 9), 2
    shp = (n[2], n[1], n[0])
    eps, mu, sigma = np.full(shp, 3.0), np.full(shp, 1.5), np.full(shp, 20.0)
    st = np.array(ma.apply_dirichlet(list(inputs.random_fields((n[2] + p, n[1] + p, n[0] + p), 6))))
    out = []
    for rm in ("row", "quad"):
        s = adi.Solver(n, p, 0.05, eps, mu, sigma, precision=prec, rhs_material=rm)
        s.factor()
        s.set_source((0.31, 0.62, 0.45), 1, 2.0, 2.0, 0.5, 0.5)
        s.set_fields(st, 0.4)
        s.step(2)
        out.append(s.fields()[0])
        s.close()
    assert_parity(list(out[1]), list(out[0]), 1e-12 if prec == "fp64" else 1e-5, what="quad vs row, uniform")


def test_quad_rejected_with_mixed():
    adi = _adi()
    with pytest.raises(adi.AdiError) as e:
        adi.Solver((4, 4, 4), 2, 0.1, precision="mixed", rhs_material="quad")
    assert e.value.status == adi.ADI_EINVAL
