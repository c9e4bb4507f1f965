"""Device-side diagnostics against the oracle: the L2, H1 and H(curl) norms of E
and H (adi_norms, quadratic forms of the 1D matrices on the GPU; the oracle
integrates the fields pointwise by Gauss quadrature) and field values on a
coordinate plane (adi_plane).  FP64: 1e-11 relative; FP32: 1e-6 (the forms are
applied in FP32 and summed in FP64)."""
import numpy as np
import pytest

from oracle import maxwell_adi as ma
from oracle import norms as on
from paper_2103_06998_gb300 import inputs

pytestmark = pytest.mark.gpu


def _adi():
    from paper_2103_06998_gb300 import adi
    return adi


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-11), ("fp32", 1e-6)])
@pytest.mark.parametrize("n,p", [((11, 9, 13), 2), ((7, 10, 6), 3), ((12, 5, 8), 1), ((37, 35, 33), 2), ((8, 7, 9), 4)])
def test_norms_match_oracle(n, p, prec, tol):
    adi = _adi()
    eps, mu, sigma, _ = inputs.head_map(n, 2103)
    s = adi.Solver(n, p, 0.01, eps, mu, sigma, precision=prec)
    s.factor()
    st = ma.apply_dirichlet(list(inputs.random_fields((n[2] + p, n[1] + p, n[0] + p), 4)))
    s.set_fields(np.array(st), 0.0)
    got = s.norms()
    ref = on.norms(st, n, p)
    np.testing.assert_allclose(got, ref, rtol=tol)
    # after steps with the dipole the norms still agree with the state the GPU holds
    src = inputs.dipole(2103)
    s.set_source(src["x0"], src["comp"], src["amp"], src["f0"], src["t0"], src["s"])
    s.step(3)
    st3, _ = s.fields()
    np.testing.assert_allclose(s.norms(), on.norms(list(st3), n, p), rtol=tol)
    s.close()


def test_norms_of_zero_state_and_bad_args():
    adi = _adi()
    s = adi.Solver((6, 6, 6), 2, 0.01)
    s.factor()
    assert np.array_equal(s.norms(), np.zeros(6))
    with pytest.raises(adi.AdiError) as e:
        s.plane(6, 0, 0.5, 4, 4)
    assert e.value.status == adi.ADI_EINVAL
    with pytest.raises(adi.AdiError) as e:
        s.plane(0, 0, 1.5, 4, 4)
    assert e.value.status == adi.ADI_EINVAL
    s.close()


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 1e-6)])
@pytest.mark.parametrize("axis,pos", [(0, 0.5), (1, 0.0), (2, 1.0), (0, 0.3137)])
def test_plane_matches_oracle(axis, pos, prec, tol):
    adi = _adi()
    n, p = (13, 11, 9), 2
    s = adi.Solver(n, p, 0.01, precision=prec)
    s.factor()
    st = ma.apply_dirichlet(list(inputs.random_fields((n[2] + p, n[1] + p, n[0] + p), 8)))
    s.set_fields(np.array(st), 0.0)
    got, _ = s.fields()
    for comp in (0, 4):
        pl = s.plane(comp, axis, pos, 17, 12)
        ref = on.plane(got[comp], n, p, axis, pos, 17, 12)
        np.testing.assert_allclose(pl, ref, rtol=tol, atol=tol * np.abs(ref).max())
    s.close()
