"""Element-wise and norm-wise comparison of GPU fields with the FP64 oracle.

A single relative l2 over all six components hides a wrong value at one point
of a large grid (one wrong dipole row of relative size 1e-2 moves the norm of a
256^3 state by about 1e-6), so every parity check also bounds the worst point:

    rel_l2  = ||got - ref|| / ||ref||                      over all components
    elem_c  = max |got_c - ref_c| / max |ref_c|            per component c

and both must stay within the stated tolerance.  A component whose reference
is zero everywhere is measured against the largest reference value of any
component.
"""
import numpy as np


def errors(got, ref):
    got = [np.asarray(g, np.float64) for g in got]
    ref = [np.asarray(r, np.float64) for r in ref]
    num = sum(float(np.sum((g - r) ** 2)) for g, r in zip(got, ref))
    den = sum(float(np.sum(r ** 2)) for r in ref)
    rel = float(np.sqrt(num / den)) if den > 0 else float(np.sqrt(num))
    top = max(float(np.abs(r).max()) for r in ref) if ref else 0.0
    elem = []
    for g, r in zip(got, ref):
        scale = float(np.abs(r).max())
        if scale == 0.0:
            scale = top if top > 0 else 1.0
        elem.append(float(np.abs(g - r).max()) / scale)
    return rel, elem


def assert_parity(got, ref, tol, elem_tol=None, what=""):
    """Both the global relative l2 and every component's worst point within tolerance."""
    elem_tol = tol if elem_tol is None else elem_tol
    rel, elem = errors(got, ref)
    assert rel < tol, "%s relative l2 %.3e >= %.1e" % (what, rel, tol)
    worst = int(np.argmax(elem))
    assert elem[worst] < elem_tol, "%s component %d: max|got-ref|/max|ref| = %.3e >= %.1e (all: %s)" % (
        what, worst, elem[worst], elem_tol, ", ".join("%.2e" % e for e in elem))
    return rel, elem
