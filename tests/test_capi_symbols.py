"""The C-ABI library builds, loads and exports every function of the header
(no compute call: runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in sorted(os.listdir(os.path.join(ROOT, "include")))
           if f.endswith(".h")]


def _declared():
    txt = "".join(open(h).read() for h in HEADERS)
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(adi_[a-z0-9_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    from paper_2103_06998_gb300 import adi, build
    if not os.path.exists(adi.LIB_PATH):
        build.build()
    return ctypes.CDLL(adi.LIB_PATH)


def test_header_declares_the_binding_exports():
    from paper_2103_06998_gb300 import adi
    assert set(_declared()) == set(adi.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    missing = [s for s in _declared() if not hasattr(lib, s)]
    assert not missing, missing


def test_status_strings_without_gpu(lib):
    f = lib.adi_status_string
    f.restype = ctypes.c_char_p
    f.argtypes = [ctypes.c_int]
    assert f(0) == b"ADI_OK" and f(4) == b"ADI_ESTATE" and f(99) == b"ADI_UNKNOWN"
    g = lib.adi_last_error
    g.restype = ctypes.c_char_p
    g.argtypes = [ctypes.c_void_p]
    assert g(None)  # never NULL


def test_invalid_arguments_rejected_before_any_cuda_call(lib):
    from paper_2103_06998_gb300 import adi
    L = adi.load_library()
    h = ctypes.c_void_p()
    assert L.adi_create(0, 4, 4, 2, 0.1, None, None, None, None, ctypes.byref(h)) == adi.ADI_EINVAL
    assert L.adi_create(4, 4, 4, 7, 0.1, None, None, None, None, ctypes.byref(h)) == adi.ADI_EINVAL
    assert L.adi_create(4, 4, 4, 2, -1.0, None, None, None, None, ctypes.byref(h)) == adi.ADI_EINVAL
    import numpy as np
    bad = np.full(64, -1.0)
    assert L.adi_create(4, 4, 4, 2, 0.1, adi._dptr(bad), None, None, None, ctypes.byref(h)) == adi.ADI_EINVAL
    assert b"eps and mu" in L.adi_last_error(None)
    assert L.adi_step(None, 1) == adi.ADI_EINVAL
    opt = adi.AdiOptions()
    opt.precision = adi.PREC_FP32
    opt.serial_chains = 2
    assert L.adi_create(4, 4, 4, 2, 0.1, None, None, None, ctypes.byref(opt), ctypes.byref(h)) == adi.ADI_EINVAL
    assert b"serial_chains" in L.adi_last_error(None)
    opt.serial_chains = 0
    opt.reserved[1] = 1
    assert L.adi_create(4, 4, 4, 2, 0.1, None, None, None, ctypes.byref(opt), ctypes.byref(h)) == adi.ADI_EINVAL


def test_net_parameter_vector_layout():
    # 27 CI CO + CO per layer with the padded channel counts of the header
    import numpy as np
    from paper_2103_06998_gb300 import adi, inputs
    assert sum(27 * ci * co + co for ci, co in zip(adi.NET_CI, adi.NET_CO)) == adi.NET_PARAMS
    txt = open(os.path.join(ROOT, "include", "adi_corrector.h")).read()
    assert "#define ADI_NET_PARAMS %d" % adi.NET_PARAMS in txt
    ps = inputs.net_init(5)
    flat = adi.net_flatten(ps)
    back = adi.net_unflatten(flat)
    for (w, b), (w2, b2) in zip(ps, back):
        np.testing.assert_array_equal(np.float32(w), w2)
        np.testing.assert_array_equal(np.float32(b), b2)
    # weight of layer 0, tap (dz, dy, dx) = (1, 2, 0), ci 3, co 7 sits at
    # (9 + 6 + 0) * 16 * 32 + 3 * 32 + 7
    assert flat[15 * 16 * 32 + 3 * 32 + 7] == np.float32(ps[0][0][1, 2, 0, 3, 7])


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    # the binding has no CPU fallback: without the built library every entry point raises
    from paper_2103_06998_gb300 import adi
    monkeypatch.setattr(adi, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        adi.load_library(str(tmp_path / "libadi_maxwell.so"))
    monkeypatch.setattr(adi, "LIB_PATH", str(tmp_path / "libadi_maxwell.so"))
    monkeypatch.setattr(adi.load_library, "__defaults__", (str(tmp_path / "libadi_maxwell.so"),))
    with pytest.raises(RuntimeError, match="not built"):
        adi.axis_bands(4, 2)
    with pytest.raises(RuntimeError, match="not built"):
        adi.Solver((4, 4, 4), 2, 0.01)
