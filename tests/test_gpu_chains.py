"""The concurrent schedule of a half step gives the same fields, bit for bit, as
the serial one and as the sub-steps run one by one.

The three E components of a half step are independent chains of line solves on
disjoint arrays (the material-direction solve, then the two mass solves).  By
default they run on three branch streams (parallel branches of the captured
step).  Every array sees the same operations in the same order as in the serial
schedule and as in adi_substep 0..3, so the test compares for equality: graph
and direct launches, FP32, FP64 and mixed, uniform and non-uniform mu, p = 1..4.
"""
import numpy as np
import pytest

from paper_2103_06998_gb300 import inputs

pytestmark = pytest.mark.gpu


def _solver(n, p, prec, mat, serial, use_graph):
    from paper_2103_06998_gb300 import adi
    if mat == "head":
        eps, mu, sigma, _ = inputs.head_map(n, 2103)
    else:
        eps, mu, sigma = inputs.random_material(n, 7, mu_range=(1.0, 3.0))
    s = adi.Solver(n, p, 0.01, eps, mu, sigma, precision=prec, use_graph=use_graph, serial_chains=serial)
    s.factor()
    src = inputs.dipole(2103)
    s.set_source(src["x0"], src["comp"], src["amp"], src["f0"], src["t0"], src["s"])
    s.set_fields(inputs.random_fields(s.shape, 11), 0.0)
    return s


def _run(n, p, prec, mat, serial, use_graph, nstep=3, substeps=False):
    s = _solver(n, p, prec, mat, serial, use_graph)
    if substeps:
        for _ in range(nstep):
            for w in range(4):
                s.substep(w)
    else:
        s.step(nstep)
    out, _ = s.fields()
    s.close()
    return out


CASES = [((37, 29, 41), 2, "fp32", "head"), ((33, 40, 27), 3, "fp32", "head"), ((21, 18, 25), 1, "fp32", "head"),
         ((19, 14, 23), 4, "fp32", "head"), ((30, 26, 22), 2, "fp64", "head"), ((30, 26, 22), 2, "mixed", "head"),
         ((25, 31, 20), 2, "fp32", "random")]


@pytest.mark.parametrize("n,p,prec,mat", CASES)
@pytest.mark.parametrize("use_graph", [True, False])
def test_concurrent_chains_equal_serial(n, p, prec, mat, use_graph):
    a = _run(n, p, prec, mat, serial=False, use_graph=use_graph)
    b = _run(n, p, prec, mat, serial=True, use_graph=use_graph)
    assert np.all(np.isfinite(a))
    assert np.array_equal(a, b)


@pytest.mark.parametrize("n,p,prec,mat", CASES)
def test_step_equals_substeps(n, p, prec, mat):
    a = _run(n, p, prec, mat, serial=False, use_graph=True)
    b = _run(n, p, prec, mat, serial=False, use_graph=False, substeps=True)
    assert np.array_equal(a, b)
