"""Batched mode: every instance of a heterogeneous batch equals the same
instance stepped alone (bit for bit), one instance matches the oracle, and the
line-tile autotuner keeps results and state unchanged."""
import os
import tempfile

import numpy as np
import pytest

from oracle import maxwell_adi as ma
from paper_2103_06998_gb300 import inputs
from parity_check import assert_parity

pytestmark = pytest.mark.gpu

SIZES = [((12, 9, 14), 2), ((10, 13, 8), 3), ((16, 11, 9), 2), ((9, 9, 12), 3)]


def _instances():
    out = []
    for i, (n, p) in enumerate(SIZES):
        eps, mu, sigma, _ = inputs.head_map(n, 2103 + i)
        out.append(dict(n=n, p=p, dt=0.01 + 0.002 * i, eps=eps, mu=mu, sigma=sigma, source=inputs.dipole(2103 + i)))
    return out


def _prepare(solver, inst, seed):
    src = inst["source"]
    solver.set_source(src["x0"], src["comp"], src["amp"], src["f0"], src["t0"], src["s"])
    n, p = inst["n"], inst["p"]
    st = inputs.random_fields((n[2] + p, n[1] + p, n[0] + p), seed)
    solver.set_fields(st, 1.3)
    return st


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_batch_equals_instances_alone(prec):
    from paper_2103_06998_gb300 import adi
    insts = _instances()
    b = adi.Batch(insts, precision=prec)
    b.factor()
    states = [_prepare(s, inst, 10 + i) for i, (s, inst) in enumerate(zip(b.solvers, insts))]
    b.step(3)
    b.sync()
    got = [s.fields() for s in b.solvers]
    for i, inst in enumerate(insts):
        a = adi.Solver(inst["n"], inst["p"], inst["dt"], inst["eps"], inst["mu"], inst["sigma"], precision=prec)
        a.factor()
        _prepare(a, inst, 10 + i)
        a.step(3)
        ref, t = a.fields()
        a.close()
        assert np.array_equal(got[i][0], ref), i
        assert abs(got[i][1] - t) < 1e-12
    # every instance (p = 2 and p = 3) against the FP64 oracle, element by element
    from test_gpu_parity import tol
    for i, inst in enumerate(insts):
        prob = ma.make_problem(inst["n"], inst["p"], inst["dt"], inst["eps"], inst["mu"], inst["sigma"])
        src = inst["source"]
        ma.set_source(prob, src["x0"], src["comp"], src["amp"], src["f0"], src["t0"], src["s"])
        ref, _ = ma.run(prob, ma.apply_dirichlet(list(states[i])), 1.3, 3)
        assert_parity(list(got[i][0]), ref, 3 * tol(prec, inst["p"]), what="batch instance %d" % i)
    b.close()


def test_autotune_keeps_results():
    from paper_2103_06998_gb300 import adi
    insts = _instances()
    b = adi.Batch(insts)
    b.factor()
    for i, (s, inst) in enumerate(zip(b.solvers, insts)):
        _prepare(s, inst, 20 + i)
    before = [s.fields()[0] for s in b.solvers]
    with tempfile.TemporaryDirectory() as d:
        cache = os.path.join(d, "tiles.txt")
        b.autotune(cache)
        lines = open(cache).read().split()
        assert len(lines) == 2 * len(insts)
        assert all(int(v) in (8, 16, 32, 64) for v in lines[1::2])
        after = [s.fields()[0] for s in b.solvers]
        for x, y in zip(before, after):
            assert np.array_equal(x, y)
        b.step(2)
        b.sync()
        tuned = [s.fields()[0] for s in b.solvers]
        b2 = adi.Batch(insts)   # default tiles
        b2.factor()
        for i, (s, inst) in enumerate(zip(b2.solvers, insts)):
            _prepare(s, inst, 20 + i)
        b2.step(2)
        b2.sync()
        for i, s in enumerate(b2.solvers):
            assert np.array_equal(s.fields()[0], tuned[i])
        b2.autotune(cache)      # second batch reads the cache, appends nothing
        assert open(cache).read().split() == lines
        b2.close()
    b.close()
