"""adi_cfl_dt_noalloc: the explicit time-step limit without any device
allocation, for callers that cannot allocate (services whose device memory all
belongs to their own pool, real-time loops that must not block in the
allocator, plug-ins of an application that owns every allocation).  Checked against adi_cfl_dt of handles built from the
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
    # sizes whose int sum nx + ny + nz wraps around: rejected, nothing is read
    big = 2 ** 31 - 2
    for n in ((big, big, 8), (big, 2, big), (1, big, big)):
        st, _ = _call(lib, n, 2, d, d)
        assert st == adi.ADI_EINVAL, n
        assert b"scratch limit" in lib.adi_last_error(None)


@pytest.mark.parametrize("bad", ["negative_eps", "nan_eps", "zero_mu", "inf_mu"])
def test_noalloc_rejects_bad_material(bad):
    # one bad element among valid ones must give ADI_ENUMERIC, not a limit
    # computed from the remaining rows; a valid call afterwards still works
    torch = pytest.importorskip("torch")
    from paper_2103_06998_gb300 import adi, inputs
    lib = adi.load_library()
    n, p = (12, 10, 9), 2
    eps, mu, _, _ = inputs.head_map(n, 2103)
    eps = np.ascontiguousarray(eps).ravel().copy()
    mu = np.ascontiguousarray(mu).ravel().copy()
    good = (eps.copy(), mu.copy())
    k = 517
    if bad == "negative_eps":
        eps[k] = -3.0
    elif bad == "nan_eps":
        eps[k] = np.nan
    elif bad == "zero_mu":
        mu[k] = 0.0
    else:
        mu[k] = np.inf
    dev = lambda a: torch.tensor(a, dtype=torch.float64, device="cuda")
    st, _ = _call(lib, n, p, dev(eps), dev(mu))
    assert st == adi.ADI_ENUMERIC, (bad, st)
    assert b"finite and > 0" in lib.adi_last_error(None)
    st, got = _call(lib, n, p, dev(good[0]), dev(good[1]))
    assert st == adi.ADI_OK and got > 0
