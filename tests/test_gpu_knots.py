"""Non-uniform elements (adi_create_knots) against the FP64 oracle on the same
element boundaries, element by element: graded meshes (no two band rows alike:
every row takes the band tables) and meshes with a uniform core and graded
ends (the kernels' constant-stencil path on the core rows, tables near the
ends), p = 1..3, head-like material with the dipole; one step from a white-noise
state.  Tolerances: those of the uniform case for p <= 2; for p = 3 the bound
of white-noise material, 3e-5 (measured 1.01e-5 at the worst point: the small
elements at the graded ends raise the mass matrices' condition number)."""
import numpy as np
import pytest

from oracle import maxwell_adi as ma
from paper_2103_06998_gb300 import inputs
from parity_check import assert_parity
from test_gpu_parity import tol

pytestmark = pytest.mark.gpu


def _adi():
    from paper_2103_06998_gb300 import adi
    return adi


def graded(n, r=1.25):
    h = np.array([r ** min(e, n - 1 - e) for e in range(n)], dtype=np.float64)
    b = np.concatenate([[0.0], np.cumsum(h)])
    b /= b[-1]
    b[-1] = 1.0
    return b


def core(n, layers=5, r=1.3):
    """Uniform elements in the middle, geometrically refined towards both ends."""
    h = np.array([r ** (min(e, n - 1 - e) - layers) if min(e, n - 1 - e) < layers else 1.0 for e in range(n)])
    b = np.concatenate([[0.0], np.cumsum(h)])
    b /= b[-1]
    b[-1] = 1.0
    return b


CASES = [((21, 17, 12), 2, "graded"), ((40, 24, 19), 2, "core"), ((14, 11, 16), 3, "core"), ((13, 10, 9), 1, "graded"),
         ((12, 13, 11), 3, "graded")]


def _breaks(n, kind):
    f = graded if kind == "graded" else core
    return tuple(f(k) for k in n)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("n,p,kind", CASES)
def test_nonuniform_step_matches_oracle(n, p, kind, prec):
    br = _breaks(n, kind)
    eps, mu, sigma, _ = inputs.head_map(n, 2103)
    tau = 0.02
    prob = ma.make_problem(n, p, tau, eps, mu, sigma, breaks=br)
    src = inputs.dipole(2103)
    ma.set_source(prob, src["x0"], src["comp"], src["amp"], src["f0"], 1.6, src["s"])
    st = ma.apply_dirichlet(list(inputs.random_fields(prob.shape, 3)))
    ref, _ = ma.run(prob, st, 1.7, 1)
    s = _adi().Solver(n, p, tau, eps, mu, sigma, precision=prec, breaks=br)
    s.factor()
    s.set_source(src["x0"], src["comp"], src["amp"], src["f0"], 1.6, src["s"])
    s.set_fields(np.array(st), 1.7)
    s.step(1)
    got, _ = s.fields()
    s.close()
    assert_parity(got, ref, tol(prec, p, "head" if p <= 2 else "random"), what="%s p=%d %s" % (prec, p, kind))


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_nonuniform_quad_reading(prec):
    n, p = (15, 12, 10), 2
    br = _breaks(n, "graded")
    eps, mu, sigma = inputs.random_material(n, 7, mu_range=(1.0, 2.0))
    prob = ma.make_problem(n, p, 0.03, eps, mu, sigma, rhs_material="quad", breaks=br)
    src = inputs.dipole(2103)
    ma.set_source(prob, src["x0"], src["comp"], src["amp"], src["f0"], 1.6, src["s"])
    st = ma.apply_dirichlet(list(inputs.random_fields(prob.shape, 4)))
    ref, _ = ma.run(prob, st, 1.7, 1)
    s = _adi().Solver(n, p, 0.03, eps, mu, sigma, precision=prec, rhs_material="quad", breaks=br)
    s.factor()
    s.set_source(src["x0"], src["comp"], src["amp"], src["f0"], 1.6, src["s"])
    s.set_fields(np.array(st), 1.7)
    s.step(1)
    got, _ = s.fields()
    s.close()
    assert_parity(got, ref, tol(prec, p, "random"), what="quad %s graded" % prec)


def test_uniform_breaks_reproduce_the_uniform_result():
    # the same mesh given as explicit boundaries (FP64: only the rounding of the
    # element points of the setup quadrature differs)
    adi = _adi()
    n, p = (19, 14, 11), 2
    eps, mu, sigma, _ = inputs.head_map(n, 2103)
    st = np.array(ma.apply_dirichlet(list(inputs.random_fields((n[2] + p, n[1] + p, n[0] + p), 5))))
    out = []
    for br in (None, tuple(np.arange(k + 1) / k for k in n)):
        s = adi.Solver(n, p, 0.02, eps, mu, sigma, precision="fp64", breaks=br)
        s.factor()
        s.set_fields(st, 0.0)
        s.step(2)
        out.append(s.fields()[0])
        s.close()
    assert_parity(list(out[1]), list(out[0]), 1e-12, what="explicit uniform boundaries")


def test_bad_breaks_rejected():
    adi = _adi()
    n = (4, 4, 4)
    bad = (np.array([0.0, 0.5, 0.4, 0.8, 1.0]), None, None)
    with pytest.raises(adi.AdiError) as e:
        adi.Solver(n, 2, 0.01, breaks=bad)
    assert e.value.status == adi.ADI_EINVAL
    with pytest.raises(adi.AdiError):
        adi.Solver(n, 2, 0.01, breaks=(None, np.array([0.0, 0.25, 0.5, 0.75, 0.99]), None))
