"""Failure paths and restart, on the GPU, without faulting it.

* A bounded device wait that gives up is reported as ADI_ETIMEOUT by the next
  synchronising call, once, and the handle keeps working: the wait runs on a
  barrier that expects bytes no copy delivers (nothing is in flight).
* Device memory exhaustion is ADI_ENOMEM from adi_create (one state array
  larger than the GPU's memory: the first cudaMalloc fails, nothing leaks).
* Checkpoint and resume: 2n steps in one go equal n steps, adi_fields into host
  memory, a fresh handle, adi_set_fields and n more steps, bit for bit (tau a
  power of two so that the restart time t0 + n tau is exact).
"""
import numpy as np
import pytest

from paper_2103_06998_gb300 import inputs

pytestmark = pytest.mark.gpu


def _adi():
    from paper_2103_06998_gb300 import adi
    return adi


@pytest.mark.parametrize("which", [0, 1])
def test_bounded_wait_times_out_and_handle_recovers(which):
    adi = _adi()
    n, p = (10, 9, 8), 2
    s = adi.Solver(n, p, 0.01)
    s.factor()
    st = inputs.random_fields(s.shape, 2)
    s.set_fields(st, 0.0)
    s.sync()
    s.wait_selftest(which, 64)
    with pytest.raises(adi.AdiError) as e:
        s.sync()
    assert e.value.status == adi.ADI_ETIMEOUT
    s.sync()                         # reported once, then clear
    s.step(2)                        # the handle still steps and matches a fresh one
    got, _ = s.fields()
    s.close()
    r = adi.Solver(n, p, 0.01)
    r.factor()
    r.set_fields(st, 0.0)
    r.step(2)
    ref, _ = r.fields()
    r.close()
    assert np.array_equal(got, ref)
    with pytest.raises(adi.AdiError) as e:
        adi.Solver(n, p, 0.01).wait_selftest(2, 10)
    assert e.value.status == adi.ADI_EINVAL


def test_out_of_device_memory_is_enomem():
    adi = _adi()
    # 4302^3 coefficients x 4 bytes = 318 GB for one component: more than the GPU holds
    with pytest.raises(adi.AdiError) as e:
        adi.Solver((4300, 4300, 4300), 2, 0.01)
    assert e.value.status == adi.ADI_ENOMEM
    # and the library is still usable afterwards
    s = adi.Solver((4, 4, 4), 2, 0.01)
    s.factor()
    s.step(1)
    s.close()


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_checkpoint_resume_bitwise(prec):
    adi = _adi()
    n, p, tau, nstep = (18, 13, 11), 2, 2.0 ** -7, 4
    eps, mu, sigma, _ = inputs.head_map(n, 2103)
    src = dict(inputs.dipole(2103))

    def solver():
        s = adi.Solver(n, p, tau, eps, mu, sigma, precision=prec)
        s.factor()
        s.set_source(src["x0"], src["comp"], src["amp"], src["f0"], 1.25, src["s"])
        return s

    st = inputs.random_fields((n[2] + p, n[1] + p, n[0] + p), 6)
    a = solver()
    a.set_fields(st, 1.0)
    a.step(2 * nstep)
    ref, t_ref = a.fields()
    a.close()
    b = solver()
    b.set_fields(st, 1.0)
    b.step(nstep)
    ck, t_ck = b.fields()
    b.close()
    c = solver()
    c.set_fields(ck, t_ck)
    c.step(nstep)
    got, t_got = c.fields()
    c.close()
    assert t_ck == 1.0 + nstep * tau and t_got == t_ref
    assert np.array_equal(got, ref)
