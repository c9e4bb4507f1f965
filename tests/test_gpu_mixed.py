"""Mixed precision (ADI_PREC_MIXED) against the FP64 oracle.

The E right-hand side is contracted from field tiles rounded to BF16 (FP32
accumulation), which alone leaves a relative error of order 2^-9 ~ 2e-3 in E*.
One refinement (residual in compensated float-float arithmetic, or in FP64;
correction solved in FP32) brings the step back to FP32 accuracy: relative l2 per step from an identical state within the
FP32 bound of tests/test_gpu_parity.py.  Without the refinement the error must
be at least ten times larger and still below 1e-2 (the BF16 rounding bound
with the 3D mass-matrix conditioning).
"""
import numpy as np
import pytest

from oracle import maxwell_adi as ma
from oracle import material
from paper_2103_06998_gb300 import inputs

from parity_check import errors
from test_gpu_parity import SMALL, tol

pytestmark = pytest.mark.gpu


def _adi():
    from paper_2103_06998_gb300 import adi
    return adi


def _step(n, p, tau, mat, refine, src, t0=1.37, steps=1, use_graph=True, residual="ff", want_state=False):
    adi = _adi()
    if mat == "uniform":
        eps = mu = sigma = None
    elif mat == "head":
        eps, mu, sigma, _ = inputs.head_map(n, 2103)
    else:
        eps, mu, sigma = inputs.random_material(n, 7, mu_range=(1.0, 2.0))
    prob = ma.make_problem(n, p, tau, eps, mu, sigma)
    ma.set_source(prob, src["x0"], src["comp"], src["amp"], src["f0"], src["t0"], src["s"])
    s = adi.Solver(n, p, tau, eps, mu, sigma, precision="mixed", refine=refine, use_graph=use_graph,
                   residual=residual)
    s.factor()
    s.set_source(src["x0"], src["comp"], src["amp"], src["f0"], src["t0"], src["s"])
    st = ma.apply_dirichlet(list(inputs.random_fields(prob.shape, 3)))
    s.set_fields(np.array(st), t0)
    ref, _ = ma.run(prob, st, t0, steps)
    s.step(steps)
    got, _ = s.fields()
    s.close()
    rel, elem = errors(got, ref)
    if want_state:
        return rel, max(elem), got
    return rel, max(elem)   # global relative l2, worst point of any component


@pytest.mark.parametrize("n,p,mat", SMALL)
def test_mixed_step_matches_oracle(n, p, mat):
    src = inputs.dipole(2103)
    e_ref, m_ref = _step(n, p, 0.03, mat, True, src)
    e_raw, _ = _step(n, p, 0.03, mat, False, src)
    assert e_ref < tol("fp32", p, mat) and m_ref < tol("fp32", p, mat), (e_ref, m_ref)
    # the BF16 error alone, amplified like the FP32 rounding (kappa_1D(p)^3)
    assert e_raw > 10 * e_ref and e_raw < (1e-2 if p <= 3 else 3e-2), (e_raw, e_ref)


def test_mixed_64_head_dipole():
    # the 64^3 head map at tau = 4 dt_CFL: one step and five steps
    n, p = (64, 64, 64), 2
    eps, mu, sigma, _ = inputs.head_map(n, 2103)
    tau = 4.0 * material.cfl_dt(n, p, material.row_hats(eps, n, p), material.row_hats(mu, n, p))
    src = inputs.dipole(2103)
    assert max(_step(n, p, tau, "head", True, src, t0=1.5)) < tol("fp32", p)
    assert max(_step(n, p, tau, "head", True, src, t0=1.5, steps=5)) < 5 * tol("fp32", p)


def test_mixed_graph_equals_substeps():
    adi = _adi()
    n, p, tau = (20, 17, 12), 2, 0.02
    eps, mu, sigma, _ = inputs.head_map(n, 2103)
    src = inputs.dipole(2103)
    st = np.array(ma.apply_dirichlet(list(inputs.random_fields((n[2] + p, n[1] + p, n[0] + p), 4))))
    out = []
    for graph in (True, False):
        s = adi.Solver(n, p, tau, eps, mu, sigma, precision="mixed", use_graph=graph)
        s.factor()
        s.set_source(src["x0"], src["comp"], src["amp"], src["f0"], src["t0"], src["s"])
        s.set_fields(st, 1.2)
        if graph:
            s.step(3)
        else:
            for _ in range(3):
                for w in range(4):
                    s.substep(w)
        out.append(s.fields()[0])
        s.close()
    assert np.array_equal(out[0], out[1])


@pytest.mark.parametrize("n,p,mat", SMALL)
def test_float_float_residual_matches_fp64_residual(n, p, mat):
    # the refinement's residual in compensated float-float arithmetic (the
    # default) against the same residual in FP64: both refined steps meet the
    # FP32 bound against the oracle, and they agree with each other to FP32
    # rounding of the state (E* is the same; only the correction can differ)
    src = inputs.dipole(2103)
    e_ff, m_ff, g_ff = _step(n, p, 0.03, mat, True, src, residual="ff", want_state=True)
    e_64, m_64, g_64 = _step(n, p, 0.03, mat, True, src, residual="fp64", want_state=True)
    assert max(e_ff, m_ff) < tol("fp32", p, mat) and max(e_64, m_64) < tol("fp32", p, mat)
    rel, elem = errors(g_ff, g_64)
    scale = tol("fp32", p, mat) / 1e-5   # the FP32 amplification of this case
    assert rel < 1e-6 * scale and max(elem) < 2e-6 * scale, (rel, elem)
