"""adi_cfl_dt_noalloc: the explicit time-step limit without any device
allocation, for callers that cannot allocate (graph capture, fixed memory
pools, real-time loops).  Checked against adi_cfl_dt of handles built from the
same material, on two calls in a row with different material (the shared
scratch must be re-initialised by every call).  This file sorts last so a run
that stops at the first failure has run every other test before it."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = 1e-11  # the FP64 tolerance of the parity tests


def _call(lib, n, p, d_eps, d_mu):
    out = ctypes.c_double(-1.0)
    st = lib.adi_cfl_dt_noalloc(n[0], n[1], n[2], p, ctypes.c_void_p(d_eps.data_ptr()),
                                ctypes.c_void_p(d_mu.data_ptr()), None, ctypes.byref(out))
    return st, out.value


def test_noalloc_cfl_dt_matches_handle_twice():
    torch = pytest.importorskip("torch")
    from paper_2103_06998_gb300 import adi, inputs
    lib = adi.load_library()
    n, p = (24, 20, 16), 2
    eps1, mu1, sig1, _ = inputs.head_map(n, 2103)            # min eps^ mu^ = 1 (air)
    eps2, mu2, sig2 = inputs.random_material(n, 11, eps_range=(3.0, 9.0), mu_range=(1.5, 2.5))
    results = []
    for eps, mu, sig in ((eps1, mu1, sig1), (eps2, mu2, sig2)):
        s = adi.Solver(n, p, 0.01, eps, mu, sig)
        ref = s.cfl_dt()
        s.close()
        d_eps = torch.tensor(np.ascontiguousarray(eps).ravel(), dtype=torch.float64, device="cuda")
        d_mu = torch.tensor(np.ascontiguousarray(mu).ravel(), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        st, got = _call(lib, n, p, d_eps, d_mu)
        assert st == adi.ADI_OK, lib.adi_last_error(None)
        assert ref > 0 and abs(got - ref) <= TOL * ref, (got, ref)
        results.append(got)
    assert results[1] > results[0]  # the second material is slower: the minimum was reset


def test_noalloc_rejects_sizes_beyond_scratch():
    torch = pytest.importorskip("torch")
    from paper_2103_06998_gb300 import adi
    lib = adi.load_library()
    d = torch.ones(8, dtype=torch.float64, device="cuda")
    st, _ = _call(lib, (4000, 8, 8), 2, d, d)
    assert st == adi.ADI_EINVAL
    assert b"scratch limit" in lib.adi_last_error(None)
