"""Host transfers through the C-ABI: page-locked host buffers (read and written
by the kernels directly) and pageable ones (staged through a copy) give the
same state and the same read-back bit for bit; a NaN in a page-locked buffer is
rejected with ADI_ENUMERIC and leaves the state unchanged."""
import numpy as np
import pytest

from paper_2103_06998_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_pinned_and_pageable_agree(prec):
    import torch
    from paper_2103_06998_gb300 import adi
    n, p = (13, 10, 7), 2
    shape = (6, n[2] + p, n[1] + p, n[0] + p)
    st = inputs.random_fields(shape[1:], 21)
    s = adi.Solver(n, p, 0.02, precision=prec)
    s.factor()
    pin_in = torch.empty(st.size, dtype=torch.float64, pin_memory=True)
    pin_out = torch.empty(st.size, dtype=torch.float64, pin_memory=True)
    pin_in.numpy()[:] = st.ravel()

    s.set_fields(st, 0.5)                      # pageable: staged copy
    a0, _ = s.fields()
    s.set_fields_ptr(pin_in.data_ptr(), 0.5)   # page-locked: direct
    b0, _ = s.fields()
    t = s.fields_ptr(pin_out.data_ptr())       # direct write-back
    assert np.array_equal(a0, b0)
    assert np.array_equal(pin_out.numpy().reshape(shape), a0)
    assert t == 0.5

    s.step(2)
    a1, t1 = s.fields()
    s.fields_ptr(pin_out.data_ptr())
    assert np.array_equal(pin_out.numpy().reshape(shape), a1)

    pin_in.numpy()[123] = np.nan               # rejected; state and time unchanged
    with pytest.raises(adi.AdiError) as e:
        s.set_fields_ptr(pin_in.data_ptr(), 9.0)
    assert e.value.status == adi.ADI_ENUMERIC
    a2, t2 = s.fields()
    assert np.array_equal(a2, a1) and t2 == t1
    s.close()
