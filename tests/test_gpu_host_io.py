"""Host transfers through the C-ABI: page-locked host buffers (read and written
by the kernels directly) and pageable ones (staged through a copy) give the
same state and the same read-back bit for bit; a NaN in a page-locked buffer is
rejected with ADI_ENUMERIC and leaves the state unchanged.

The float forms (adi_set_fields_f32 / adi_fields_f32) against the double ones:
the FP32 state set from floats equals the state set from the same values as
doubles, reading back as floats returns exactly the FP32 state, the
coefficients fixed by the boundary conditions come back zero, 16-byte aligned
and unaligned host pointers take the vector and the scalar kernels with the same
result, pointers off their element alignment are refused on the host, and an
FP64 handle round-trips floats exactly.

The asynchronous forms (adi_set_fields_async / adi_fields_async: copy-engine
transfers through device staging arrays on the handle's input and output
streams) give the same states and read-backs as the synchronous calls, in a
loop without synchronisation, mixed with sub-steps and synchronous calls, and
across a change of the host element size on one handle; a NaN is refused on
the device and reported once by adi_sync.
"""
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


N, P = (37, 29, 23), 2  # 6 N_c is not a multiple of 4: the vector kernels' scalar tail runs


def _solver(prec):
    from paper_2103_06998_gb300 import adi
    s = adi.Solver(N, P, 0.01, precision=prec)
    s.factor()
    return s


def _pinned(nbytes):
    torch = pytest.importorskip("torch")
    return torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)


def _constrained(shape):
    """Mask of the coefficients the boundary conditions fix to zero (6, Nz, Ny, Nx)."""
    nz, ny, nx = shape
    m = np.zeros((6,) + shape, dtype=bool)
    for c in range(6):
        axes = [a for a in range(3) if a != c] if c < 3 else [c - 3]
        for a in axes:  # a = 0: x, 1: y, 2: z
            sl = [slice(None)] * 3
            for end in (0, -1):
                sl[2 - a] = end
                m[(c,) + tuple(sl)] = True
                sl[2 - a] = slice(None)
    return m


def _view(buf, dtype, count, offset=0):
    return np.frombuffer(buf.numpy(), dtype=np.uint8)[offset:offset + count * np.dtype(dtype).itemsize].view(dtype)


@pytest.mark.parametrize("offset", [0, 4])
def test_float_transfers_equal_double_transfers(offset):
    s = _solver("fp32")
    st = inputs.random_fields(s.shape, 21).astype(np.float32)
    n = st.size
    buf = _pinned(n * 4 + 16)
    a = _view(buf, np.float32, n, offset)  # offset 4: not 16-byte aligned (scalar kernels)
    a[:] = st.ravel()
    s.set_fields_f32_ptr(a.ctypes.data, 0.5)
    got64, t = s.fields()
    assert t == 0.5
    ref = st.astype(np.float64)
    ref[_constrained(s.shape)] = 0.0
    assert np.array_equal(got64, ref)
    # pageable floats, and doubles of the same values: the same state
    r = _solver("fp32")
    r.set_fields(st.astype(np.float64), 0.5)
    assert np.array_equal(r.fields()[0], got64)
    pg = np.ascontiguousarray(st.ravel())
    r.set_fields_f32_ptr(pg.ctypes.data, 0.5)
    assert np.array_equal(r.fields()[0], got64)
    # reading back as floats: pinned (aligned or not) and pageable
    out = _view(_pinned(n * 4 + 16), np.float32, n, offset)
    s.fields_f32_ptr(out.ctypes.data)
    assert np.array_equal(out.astype(np.float64), got64.ravel())
    out2 = np.empty(n, dtype=np.float32)
    s.fields_f32_ptr(out2.ctypes.data)
    assert np.array_equal(out2, out)
    # doubles into pinned memory, 16-byte aligned or only 8-byte aligned
    d = _view(_pinned(n * 8 + 16), np.float64, n, 2 * offset)
    s.fields_ptr(d.ctypes.data)
    assert np.array_equal(d, got64.ravel())
    s.close()
    r.close()


def test_misaligned_pointers_are_rejected_on_the_host():
    # a double* or float* off its element alignment is refused before any device
    # work (a device access through it would fault)
    from paper_2103_06998_gb300 import adi
    s = _solver("fp32")
    buf = np.zeros(6 * int(np.prod(s.shape)) * 8 + 16, dtype=np.uint8)
    base = buf.ctypes.data
    for call in (lambda p: s.set_fields_ptr(p, 0.0), lambda p: s.fields_ptr(p)):
        with pytest.raises(adi.AdiError) as e:
            call(base + (8 - base % 8) + 4)
        assert e.value.status == adi.ADI_EINVAL
    for call in (lambda p: s.set_fields_f32_ptr(p, 0.0), lambda p: s.fields_f32_ptr(p)):
        with pytest.raises(adi.AdiError) as e:
            call(base + (4 - base % 4) + 2)
        assert e.value.status == adi.ADI_EINVAL
    s.close()


def test_float_nan_is_rejected_and_state_kept():
    from paper_2103_06998_gb300 import adi
    s = _solver("fp32")
    st = inputs.random_fields(s.shape, 23).astype(np.float32)
    s.set_fields_f32_ptr(np.ascontiguousarray(st.ravel()).ctypes.data, 1.0)
    before, _ = s.fields()
    bad = st.copy().ravel()
    bad[bad.size // 2 + 1] = np.nan
    for ptr in (np.ascontiguousarray(bad).ctypes.data,):
        with pytest.raises(adi.AdiError) as e:
            s.set_fields_f32_ptr(ptr, 2.0)
        assert e.value.status == adi.ADI_ENUMERIC
    buf = _pinned(bad.size * 4)
    a = _view(buf, np.float32, bad.size)
    a[:] = bad
    with pytest.raises(adi.AdiError) as e:
        s.set_fields_f32_ptr(a.ctypes.data, 2.0)
    assert e.value.status == adi.ADI_ENUMERIC
    after, t = s.fields()
    assert t == 1.0 and np.array_equal(after, before)
    s.close()


def test_fp64_handle_round_trips_floats():
    s = _solver("fp64")
    st = inputs.random_fields(s.shape, 24).astype(np.float32)
    s.set_fields_f32_ptr(np.ascontiguousarray(st.ravel()).ctypes.data, 0.0)
    out = np.empty(st.size, dtype=np.float32)
    s.fields_f32_ptr(out.ctypes.data)
    ref = st.copy()
    ref[_constrained(s.shape)] = 0.0
    assert np.array_equal(out, ref.ravel())
    s.close()


# ---- asynchronous transfers: set, step, read, set, step, read, ... without waiting
@pytest.mark.parametrize("prec,elem", [("fp32", 4), ("fp32", 8), ("fp64", 8)])
def test_async_pipeline_equals_synchronous_calls(prec, elem):
    dt = np.float32 if elem == 4 else np.float64
    a, b = _solver(prec), _solver(prec)
    a.set_source((0.4, 0.55, 0.3), 2, 3.0, 2.0, 0.2, 0.3)
    b.set_source((0.4, 0.55, 0.3), 2, 3.0, 2.0, 0.2, 0.3)
    n = 6 * int(np.prod(a.shape))
    ins, outs = [], []
    for i in range(3):
        x = _view(_pinned(n * elem), dt, n)
        x[:] = inputs.random_fields(a.shape, 30 + i).ravel().astype(dt)
        ins.append(x)
        outs.append(_view(_pinned(n * elem), dt, n))
    for i in range(3):  # no synchronisation inside the loop
        a.set_fields_async_ptr(ins[i].ctypes.data, elem, 0.25 * i)
        a.step(2)
        a.fields_async_ptr(outs[i].ctypes.data, elem)
    a.sync()
    for i in range(3):
        b.set_fields(ins[i].astype(np.float64), 0.25 * i)
        b.step(2)
        ref, t = b.fields()
        assert np.array_equal(outs[i], ref.ravel().astype(dt)), i
    assert abs(a.fields()[1] - t) < 1e-12
    a.close()
    b.close()


def test_async_nan_is_refused_and_reported_once():
    from paper_2103_06998_gb300 import adi
    s, r = _solver("fp32"), _solver("fp32")
    n = 6 * int(np.prod(s.shape))
    good = _view(_pinned(n * 4), np.float32, n)
    good[:] = inputs.random_fields(s.shape, 40).ravel()
    bad = _view(_pinned(n * 4), np.float32, n)
    bad[:] = good
    bad[n // 3] = np.inf
    for x in (s, r):
        x.set_fields_f32_ptr(good.ctypes.data, 0.0)
        x.step(1)
    s.set_fields_async_ptr(bad.ctypes.data, 4, 5.0)  # refused on the device
    s.step(1)
    with pytest.raises(adi.AdiError) as e:
        s.sync()
    assert e.value.status == adi.ADI_ENUMERIC
    s.sync()  # reported once
    r.step(1)  # the reference never saw the refused set
    assert np.array_equal(s.fields()[0], r.fields()[0])
    s.close()
    r.close()


def test_async_transfers_need_page_locked_aligned_memory():
    from paper_2103_06998_gb300 import adi
    s = _solver("fp32")
    n = 6 * int(np.prod(s.shape))
    pageable = np.zeros(n, dtype=np.float32)
    pinned = _view(_pinned(n * 4 + 16), np.float32, n)
    for call in (lambda: s.set_fields_async_ptr(pageable.ctypes.data, 4, 0.0),
                 lambda: s.fields_async_ptr(pageable.ctypes.data, 4),
                 lambda: s.set_fields_async_ptr(pinned.ctypes.data, 2, 0.0),
                 lambda: s.fields_async_ptr(pinned.ctypes.data + 2, 4)):
        with pytest.raises(adi.AdiError) as e:
            call()
        assert e.value.status == adi.ADI_EINVAL
    s.sync()
    s.close()


def test_async_calls_mix_with_substeps_and_synchronous_calls():
    # every later call on the handle is ordered after a pending asynchronous transfer
    s, r = _solver("fp32"), _solver("fp32")
    n = 6 * int(np.prod(s.shape))
    x = _view(_pinned(n * 4), np.float32, n)
    x[:] = inputs.random_fields(s.shape, 50).ravel()
    y = _view(_pinned(n * 4), np.float32, n)
    s.set_fields_async_ptr(x.ctypes.data, 4, 0.5)
    for w in range(4):
        s.substep(w)
    s.fields_async_ptr(y.ctypes.data, 4)
    st2 = inputs.random_fields(s.shape, 51)
    s.set_fields(st2, 1.0)  # synchronous set while the read is pending
    s.step(1)
    got, t = s.fields()
    s.sync()
    r.set_fields(x.astype(np.float64), 0.5)
    r.step(1)
    ref1, _ = r.fields()
    assert np.array_equal(y, ref1.ravel().astype(np.float32))
    r.set_fields(st2, 1.0)
    r.step(1)
    ref2, t2 = r.fields()
    assert np.array_equal(got, ref2) and t == t2
    s.close()
    r.close()


def test_async_element_size_change_on_one_handle():
    # floats, then doubles on the same handle (the device staging arrays grow in
    # between), then floats again: each read equals the synchronous sequence
    s, r = _solver("fp32"), _solver("fp32")
    n = 6 * int(np.prod(s.shape))
    seq = []
    for i, elem in enumerate((4, 8, 4)):
        dt = np.float32 if elem == 4 else np.float64
        x = _view(_pinned(n * elem), dt, n)
        x[:] = inputs.random_fields(s.shape, 60 + i).ravel().astype(np.float32)
        y = _view(_pinned(n * elem), dt, n)
        s.set_fields_async_ptr(x.ctypes.data, elem, 0.5 * i)
        s.step(1)
        s.fields_async_ptr(y.ctypes.data, elem)
        seq.append((x, y, dt))
    s.sync()
    for i, (x, y, dt) in enumerate(seq):
        r.set_fields(x.astype(np.float64), 0.5 * i)
        r.step(1)
        ref, _ = r.fields()
        assert np.array_equal(y, ref.ravel().astype(dt)), i
    s.close()
    r.close()
