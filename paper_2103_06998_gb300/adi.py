"""Python binding of the C-ABI in include/adi_maxwell.h and include/adi_corrector.h
(ctypes, marshalling only).

Every step of the method runs in the CUDA kernels of ``libadi_maxwell.so``;
this module only converts arguments.  Loading fails loudly when the library is
missing -- there is no CPU fallback.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libadi_maxwell.so")

ADI_OK, ADI_EINVAL, ADI_ENOMEM, ADI_ECUDA, ADI_ESTATE, ADI_ENUMERIC, ADI_ETIMEOUT = range(7)
PREC_FP64, PREC_FP32, PREC_MIXED = 0, 1, 2
_PREC = {"fp64": PREC_FP64, "fp32": PREC_FP32, "mixed": PREC_MIXED}

# every symbol declared in include/adi_maxwell.h
EXPORTS = ("adi_create", "adi_create_knots", "adi_axis_bands", "adi_axis_tables", "adi_axis_element_matrices",
           "adi_axis_mass_lu", "adi_axis_point_basis",
           "adi_factor", "adi_set_dt", "adi_set_stream", "adi_set_fields",
           "adi_set_fields_f32", "adi_set_source", "adi_step", "adi_substep", "adi_fields", "adi_fields_f32",
           "adi_fields_device", "adi_set_fields_async", "adi_fields_async",
           "adi_cfl_dt", "adi_cfl_dt_noalloc", "adi_sync", "adi_wait_selftest", "adi_norms", "adi_plane", "adi_set_profiling", "adi_kernel_stats", "adi_dims",
           "adi_destroy", "adi_last_error", "adi_status_string", "adi_set_line_tile",
           "adi_batch_create", "adi_batch_set_stream", "adi_batch_handle", "adi_batch_factor", "adi_batch_step", "adi_batch_sync",
           "adi_batch_autotune", "adi_batch_destroy",
           "adi_net_create", "adi_net_set_stream", "adi_net_set_params", "adi_net_get_params", "adi_net_features",
           "adi_net_target", "adi_net_forward", "adi_net_apply", "adi_net_train_step", "adi_net_gradient",
           "adi_net_loss", "adi_fields_distance", "adi_copy_state", "adi_corrector_run", "adi_net_destroy",
           "adi_net_last_error")


class AdiOptions(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("use_graph", ctypes.c_int), ("mixed_no_refine", ctypes.c_int),
                ("mixed_fp64_residual", ctypes.c_int), ("rhs_material", ctypes.c_int), ("serial_chains", ctypes.c_int),
                ("reserved", ctypes.c_int * 2)]


class AdiInstanceDesc(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int), ("p", ctypes.c_int),
                ("dt", ctypes.c_double), ("eps", ctypes.POINTER(ctypes.c_double)),
                ("mu", ctypes.POINTER(ctypes.c_double)), ("sigma", ctypes.POINTER(ctypes.c_double))]


class AdiKernelStat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char_p), ("launches", ctypes.c_longlong),
                ("total_ms", ctypes.c_double), ("bytes_per_launch", ctypes.c_double)]


_lib = None


def load_library(path=LIB_PATH):
    """Load libadi_maxwell.so once; raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("libadi_maxwell.so not built (run paper_2103_06998_gb300.build.build())")
    lib = ctypes.CDLL(path)
    H = ctypes.c_void_p
    D = ctypes.c_double
    I = ctypes.c_int
    P = ctypes.POINTER
    sig = {
        "adi_create": (I, [I, I, I, I, D, P(D), P(D), P(D), P(AdiOptions), P(H)]),
        "adi_create_knots": (I, [I, I, I, I, D, P(D), P(D), P(D), P(D), P(D), P(D), P(AdiOptions), P(H)]),
        "adi_axis_bands": (I, [I, I, P(D), P(D), P(D), P(D), P(D), P(I)]),
        "adi_axis_tables": (I, [I, I, P(D), P(D), P(D)]),
        "adi_axis_element_matrices": (I, [I, I, P(D), P(D)]),
        "adi_axis_mass_lu": (I, [I, I, P(D), I, P(D), P(D), P(D)]),
        "adi_axis_point_basis": (I, [I, I, P(D), D, P(I), P(D)]),
        "adi_factor": (I, [H]),
        "adi_set_dt": (I, [H, D]),
        "adi_set_stream": (I, [H, ctypes.c_void_p]),
        "adi_set_fields": (I, [H, P(D), D]),
        "adi_set_fields_f32": (I, [H, ctypes.c_void_p, D]),
        "adi_set_source": (I, [H, D, D, D, I, D, D, D, D]),
        "adi_step": (I, [H, I]),
        "adi_substep": (I, [H, I]),
        "adi_fields": (I, [H, P(D), P(D)]),
        "adi_fields_f32": (I, [H, ctypes.c_void_p, P(D)]),
        "adi_set_fields_async": (I, [H, ctypes.c_void_p, I, D]),
        "adi_fields_async": (I, [H, ctypes.c_void_p, I]),
        "adi_fields_device": (I, [H, ctypes.c_void_p, ctypes.c_void_p]),
        "adi_cfl_dt": (D, [H]),
        "adi_cfl_dt_noalloc": (I, [I, I, I, I, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, P(D)]),
        "adi_sync": (I, [H]),
        "adi_wait_selftest": (I, [H, I, I]),
        "adi_norms": (I, [H, P(D)]),
        "adi_plane": (I, [H, I, I, D, I, I, P(D)]),
        "adi_set_profiling": (I, [H, I]),
        "adi_kernel_stats": (I, [H, P(AdiKernelStat), I, P(I)]),
        "adi_dims": (I, [H, P(I), P(I), P(I), P(I)]),
        "adi_destroy": (None, [H]),
        "adi_last_error": (ctypes.c_char_p, [H]),
        "adi_status_string": (ctypes.c_char_p, [I]),
        "adi_set_line_tile": (I, [H, I]),
        "adi_batch_create": (I, [I, P(AdiInstanceDesc), P(AdiOptions), P(H)]),
        "adi_batch_handle": (I, [H, I, P(H)]),
        "adi_batch_set_stream": (I, [H, ctypes.c_void_p]),
        "adi_batch_factor": (I, [H]),
        "adi_batch_step": (I, [H, I]),
        "adi_batch_sync": (I, [H]),
        "adi_batch_autotune": (I, [H, ctypes.c_char_p]),
        "adi_batch_destroy": (None, [H]),
        "adi_net_create": (I, [I, I, I, P(H)]),
        "adi_net_set_stream": (I, [H, ctypes.c_void_p]),
        "adi_net_set_params": (I, [H, P(ctypes.c_float), ctypes.c_size_t]),
        "adi_net_get_params": (I, [H, P(ctypes.c_float), ctypes.c_size_t]),
        "adi_net_features": (I, [H, H, ctypes.c_void_p]),
        "adi_net_target": (I, [H, H, H, ctypes.c_void_p]),
        "adi_net_forward": (I, [H, ctypes.c_void_p, ctypes.c_void_p]),
        "adi_net_apply": (I, [H, H, ctypes.c_void_p]),
        "adi_net_train_step": (I, [H, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_float]),
        "adi_net_gradient": (I, [H, ctypes.c_void_p, ctypes.c_void_p, P(ctypes.c_float), P(D)]),
        "adi_net_loss": (I, [H, P(D), P(I)]),
        "adi_fields_distance": (I, [H, H, P(D)]),
        "adi_copy_state": (I, [H, H]),
        "adi_corrector_run": (I, [H, H, H, I, I, I, D, P(I), P(D)]),
        "adi_net_destroy": (None, [H]),
        "adi_net_last_error": (ctypes.c_char_p, [H]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


class AdiError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (status, msg))
        self.status = status


def axis_bands(n, p, breaks=None):
    """adi_axis_bands: the 1D matrices of one axis as the solver builds them (host
    only).  Returns ({"M", "S", "A", "B"}: (N, 2p+1) band arrays, row k column d =
    X[k][k+d-p]; (first, last) interior-stencil row)."""
    L = load_library()
    N, W = n + p, 2 * p + 1
    out = {k: np.zeros((N, W)) for k in "MSAB"}
    inner = (ctypes.c_int * 2)()
    br = None if breaks is None else np.ascontiguousarray(breaks, dtype=np.float64)
    st = L.adi_axis_bands(n, p, None if br is None else _dptr(br), *(_dptr(out[k]) for k in "MSAB"),
                          ctypes.cast(inner, ctypes.POINTER(ctypes.c_int)))
    if st != ADI_OK:
        raise AdiError(st, L.adi_last_error(None).decode())
    return out, (inner[0], inner[1])


def _breaks_arg(breaks):
    return None if breaks is None else np.ascontiguousarray(breaks, dtype=np.float64)


def axis_tables(n, p, breaks=None):
    """adi_axis_tables: (G (N, p+1) element integrals of the basis, largest
    eigenvalue of the Dirichlet-reduced M^{-1} S)."""
    L = load_library()
    G = np.zeros((n + p, p + 1))
    lam = ctypes.c_double()
    br = _breaks_arg(breaks)
    st = L.adi_axis_tables(n, p, None if br is None else _dptr(br), _dptr(G), ctypes.byref(lam))
    if st != ADI_OK:
        raise AdiError(st, L.adi_last_error(None).decode())
    return G, lam.value


def axis_element_matrices(n, p, breaks=None):
    """adi_axis_element_matrices: (n, 4, p+1, p+1) blocks [element][M, S, A, B][test][trial]."""
    L = load_library()
    loc = np.zeros((n, 4, p + 1, p + 1))
    br = _breaks_arg(breaks)
    st = L.adi_axis_element_matrices(n, p, None if br is None else _dptr(br), _dptr(loc))
    if st != ADI_OK:
        raise AdiError(st, L.adi_last_error(None).decode())
    return loc


def axis_mass_lu(n, p, breaks=None, reduced=False):
    """adi_axis_mass_lu: (L (N, p), inv_d (N,), U (N, p)) of the 1D mass matrix."""
    L = load_library()
    N = n + p
    lo, inv_d, up = np.zeros((N, p)), np.zeros(N), np.zeros((N, p))
    br = _breaks_arg(breaks)
    st = L.adi_axis_mass_lu(n, p, None if br is None else _dptr(br), int(bool(reduced)), _dptr(lo), _dptr(inv_d),
                            _dptr(up))
    if st != ADI_OK:
        raise AdiError(st, L.adi_last_error(None).decode())
    return lo, inv_d, up


def axis_point_basis(n, p, x0, breaks=None):
    """adi_axis_point_basis: (first basis index e, values of B_e .. B_{e+p} at x0)."""
    L = load_library()
    first = ctypes.c_int()
    vals = np.zeros(p + 1)
    br = _breaks_arg(breaks)
    st = L.adi_axis_point_basis(n, p, None if br is None else _dptr(br), float(x0), ctypes.byref(first), _dptr(vals))
    if st != ADI_OK:
        raise AdiError(st, L.adi_last_error(None).decode())
    return first.value, vals


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


class Solver:
    """One ADI Maxwell problem on the GPU (owns an adi_handle)."""

    def __init__(self, n, p, dt, eps=None, mu=None, sigma=None, precision="fp32", use_graph=True, _handle=None,
                 refine=True, residual="ff", rhs_material="row", breaks=None, serial_chains=False):
        lib = load_library()
        self._lib = lib
        if _handle is not None:  # an instance owned by a Batch
            self.n = tuple(int(v) for v in n)
            self.p = int(p)
            self.dtype = np.float64 if precision == "fp64" else np.float32
            self.h = _handle
            self.shape = (self.n[2] + p, self.n[1] + p, self.n[0] + p)
            self.dt = float(dt)
            self._owned = False
            return
        self._owned = True
        self.n = tuple(int(v) for v in n)
        self.p = int(p)
        opt = AdiOptions()
        opt.precision = _PREC[precision]
        opt.use_graph = 1 if use_graph else 0
        opt.mixed_no_refine = 0 if refine else 1
        opt.mixed_fp64_residual = 1 if residual == "fp64" else 0
        opt.rhs_material = {"row": 0, "quad": 1}[rhs_material]
        opt.serial_chains = 1 if serial_chains else 0
        self.dtype = np.float64 if precision == "fp64" else np.float32
        keep = []

        def arr(a):
            if a is None:
                return None
            a = np.ascontiguousarray(a, dtype=np.float64)
            keep.append(a)
            return _dptr(a)

        h = ctypes.c_void_p()
        if breaks is None:
            st = lib.adi_create(self.n[0], self.n[1], self.n[2], self.p, float(dt), arr(eps), arr(mu), arr(sigma),
                                ctypes.byref(opt), ctypes.byref(h))
        else:
            bx, by, bz = (None if b is None else arr(b) for b in breaks)
            st = lib.adi_create_knots(self.n[0], self.n[1], self.n[2], self.p, float(dt), bx, by, bz, arr(eps),
                                      arr(mu), arr(sigma), ctypes.byref(opt), ctypes.byref(h))
        if st != ADI_OK:
            raise AdiError(st, lib.adi_last_error(None).decode())
        self.h = h
        self.shape = (self.n[2] + p, self.n[1] + p, self.n[0] + p)
        self.dt = float(dt)

    def _check(self, st):
        if st != ADI_OK:
            raise AdiError(st, self._lib.adi_last_error(self.h).decode())

    def factor(self):
        self._check(self._lib.adi_factor(self.h))

    def set_dt(self, dt):
        self._check(self._lib.adi_set_dt(self.h, float(dt)))
        self.dt = float(dt)

    def set_stream(self, stream_ptr):
        self._check(self._lib.adi_set_stream(self.h, ctypes.c_void_p(int(stream_ptr))))

    def set_fields(self, EH, t=0.0):
        a = np.ascontiguousarray(EH, dtype=np.float64)
        assert a.size == 6 * int(np.prod(self.shape))
        self._check(self._lib.adi_set_fields(self.h, _dptr(a), float(t)))

    def set_fields_ptr(self, host_ptr, t=0.0):
        """Set fields from a raw host pointer to 6 N_c doubles (e.g. pinned memory)."""
        self._check(self._lib.adi_set_fields(self.h, ctypes.cast(ctypes.c_void_p(int(host_ptr)),
                                                                 ctypes.POINTER(ctypes.c_double)), float(t)))

    def set_fields_f32_ptr(self, host_ptr, t=0.0):
        """Set fields from a raw host pointer to 6 N_c floats (e.g. pinned memory)."""
        self._check(self._lib.adi_set_fields_f32(self.h, ctypes.c_void_p(int(host_ptr)), float(t)))

    def set_source(self, x0, comp, amp, f0, t0, s):
        self._check(self._lib.adi_set_source(self.h, float(x0[0]), float(x0[1]), float(x0[2]), int(comp),
                                             float(amp), float(f0), float(t0), float(s)))

    def step(self, n=1):
        self._check(self._lib.adi_step(self.h, int(n)))

    def substep(self, which):
        self._check(self._lib.adi_substep(self.h, int(which)))

    def fields(self):
        out = np.empty((6,) + self.shape, dtype=np.float64)
        t = ctypes.c_double()
        self._check(self._lib.adi_fields(self.h, _dptr(out), ctypes.byref(t)))
        return out, t.value

    def fields_ptr(self, host_ptr):
        t = ctypes.c_double()
        self._check(self._lib.adi_fields(self.h, ctypes.cast(ctypes.c_void_p(int(host_ptr)),
                                                             ctypes.POINTER(ctypes.c_double)), ctypes.byref(t)))
        return t.value

    def fields_f32_ptr(self, host_ptr):
        """Read the fields into a raw host pointer to 6 N_c floats; returns the time."""
        t = ctypes.c_double()
        self._check(self._lib.adi_fields_f32(self.h, ctypes.c_void_p(int(host_ptr)), ctypes.byref(t)))
        return t.value

    def set_fields_async_ptr(self, host_ptr, elem_bytes, t=0.0):
        """Asynchronous set from page-locked host memory (6 N_c floats or doubles)."""
        self._check(self._lib.adi_set_fields_async(self.h, ctypes.c_void_p(int(host_ptr)), int(elem_bytes), float(t)))

    def fields_async_ptr(self, host_ptr, elem_bytes):
        """Asynchronous read into page-locked host memory; valid after sync()."""
        self._check(self._lib.adi_fields_async(self.h, ctypes.c_void_p(int(host_ptr)), int(elem_bytes)))

    def fields_device(self, dev_ptr, stream_ptr=0):
        self._check(self._lib.adi_fields_device(self.h, ctypes.c_void_p(int(dev_ptr)), ctypes.c_void_p(int(stream_ptr))))

    def cfl_dt(self):
        return self._lib.adi_cfl_dt(self.h)

    def sync(self):
        self._check(self._lib.adi_sync(self.h))

    def norms(self):
        """[L2(E), L2(H), H1(E), H1(H), Hcurl(E), Hcurl(H)] of the current state."""
        out = np.zeros(6)
        self._check(self._lib.adi_norms(self.h, _dptr(out)))
        return out

    def plane(self, comp, axis, pos, nu, nv):
        """Component ``comp`` on the plane x_axis = pos, an (nv, nu) array."""
        out = np.zeros((nv, nu))
        self._check(self._lib.adi_plane(self.h, int(comp), int(axis), float(pos), int(nu), int(nv), _dptr(out)))
        return out

    def wait_selftest(self, which, budget):
        self._check(self._lib.adi_wait_selftest(self.h, int(which), int(budget)))

    def set_profiling(self, on):
        self._check(self._lib.adi_set_profiling(self.h, 1 if on else 0))

    def kernel_stats(self):
        buf = (AdiKernelStat * 64)()
        cnt = ctypes.c_int()
        self._check(self._lib.adi_kernel_stats(self.h, buf, 64, ctypes.byref(cnt)))
        return [dict(name=buf[i].name.decode(), launches=buf[i].launches, total_ms=buf[i].total_ms,
                     bytes_per_launch=buf[i].bytes_per_launch) for i in range(min(cnt.value, 64))]

    def set_line_tile(self, lines):
        self._check(self._lib.adi_set_line_tile(self.h, int(lines)))

    def close(self):
        if getattr(self, "h", None) and getattr(self, "_owned", True):
            self._lib.adi_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Many independent problems stepped together (adi_batch_* of the C-ABI).

    ``instances``: list of dicts with keys n (nx, ny, nz), p, dt and optional
    eps, mu, sigma (per-element arrays).  ``solvers[i]`` gives access to the
    single-instance calls (fields, sources) of instance i.
    """

    def __init__(self, instances, precision="fp32"):
        lib = load_library()
        self._lib = lib
        keep = []
        descs = (AdiInstanceDesc * len(instances))()
        for d, inst in zip(descs, instances):
            d.nx, d.ny, d.nz = (int(v) for v in inst["n"])
            d.p = int(inst["p"])
            d.dt = float(inst["dt"])
            for name in ("eps", "mu", "sigma"):
                a = inst.get(name)
                if a is None:
                    setattr(d, name, None)
                else:
                    a = np.ascontiguousarray(a, dtype=np.float64)
                    keep.append(a)
                    setattr(d, name, _dptr(a))
        opt = AdiOptions()
        opt.precision = PREC_FP64 if precision == "fp64" else PREC_FP32
        opt.use_graph = 1
        b = ctypes.c_void_p()
        st = lib.adi_batch_create(len(instances), descs, ctypes.byref(opt), ctypes.byref(b))
        if st != ADI_OK:
            raise AdiError(st, lib.adi_last_error(None).decode())
        self.b = b
        self.solvers = []
        for i, inst in enumerate(instances):
            h = ctypes.c_void_p()
            self._check(lib.adi_batch_handle(b, i, ctypes.byref(h)))
            self.solvers.append(Solver(inst["n"], inst["p"], inst["dt"], precision=precision, _handle=h))

    def _check(self, st):
        if st != ADI_OK:
            raise AdiError(st, self._lib.adi_last_error(None).decode())

    def factor(self):
        self._check(self._lib.adi_batch_factor(self.b))

    def set_stream(self, stream_ptr):
        self._check(self._lib.adi_batch_set_stream(self.b, ctypes.c_void_p(int(stream_ptr))))

    def step(self, n=1):
        self._check(self._lib.adi_batch_step(self.b, int(n)))

    def sync(self):
        self._check(self._lib.adi_batch_sync(self.b))

    def autotune(self, cache_path=None):
        self._check(self._lib.adi_batch_autotune(self.b, cache_path.encode() if cache_path else None))

    def close(self):
        if getattr(self, "b", None):
            for s in self.solvers:
                s.h = None
            self._lib.adi_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------ learned corrector
NET_PARAMS = 83056
NET_CI = (16, 32, 32, 32)     # padded channels of the parameter vector
NET_CO = (32, 32, 32, 16)
NET_REAL = ((9, 32), (32, 32), (32, 32), (32, 6))


def net_flatten(params):
    """List of (w[3,3,3,ci,co], b[co]) with the real channel counts -> the padded
    FP32 parameter vector of include/adi_corrector.h (tap = 9 dz + 3 dy + dx)."""
    out = np.zeros(NET_PARAMS, dtype=np.float32)
    off = 0
    for (w, b), CI, CO in zip(params, NET_CI, NET_CO):
        ci, co = w.shape[3], w.shape[4]
        blk = np.zeros((27, CI, CO), dtype=np.float32)
        blk[:, :ci, :co] = np.asarray(w).reshape(27, ci, co)
        out[off:off + 27 * CI * CO] = blk.ravel()
        off += 27 * CI * CO
        out[off:off + co] = b
        off += CO
    assert off == NET_PARAMS
    return out


def net_unflatten(flat):
    """Inverse of net_flatten (drops the padding)."""
    out = []
    off = 0
    for (ci, co), CI, CO in zip(NET_REAL, NET_CI, NET_CO):
        blk = np.asarray(flat[off:off + 27 * CI * CO], dtype=np.float64).reshape(27, CI, CO)
        off += 27 * CI * CO
        b = np.asarray(flat[off:off + co], dtype=np.float64)
        off += CO
        out.append((blk[:, :ci, :co].reshape(3, 3, 3, ci, co).copy(), b.copy()))
    return out


class Net:
    """The corrector net on a coefficient grid N = (N_x, N_y, N_z) (owns an adi_net).

    Device arrays are passed as integer device pointers (e.g. torch
    ``tensor.data_ptr()``): features X bf16 [V][16], targets / outputs fp32 [V][8]."""

    def __init__(self, N):
        lib = load_library()
        self._lib = lib
        self.N = tuple(int(v) for v in N)
        h = ctypes.c_void_p()
        st = lib.adi_net_create(self.N[0], self.N[1], self.N[2], ctypes.byref(h))
        if st != ADI_OK:
            raise AdiError(st, lib.adi_net_last_error(None).decode())
        self.h = h

    def _check(self, st):
        if st != ADI_OK:
            raise AdiError(st, self._lib.adi_net_last_error(self.h).decode())

    def set_stream(self, stream_ptr):
        self._check(self._lib.adi_net_set_stream(self.h, ctypes.c_void_p(int(stream_ptr))))

    def set_params(self, flat):
        a = np.ascontiguousarray(flat, dtype=np.float32)
        self._check(self._lib.adi_net_set_params(self.h, a.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), a.size))

    def get_params(self):
        a = np.zeros(NET_PARAMS, dtype=np.float32)
        self._check(self._lib.adi_net_get_params(self.h, a.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), a.size))
        return a

    def features(self, solver, X):
        self._check(self._lib.adi_net_features(self.h, solver.h, ctypes.c_void_p(int(X))))

    def target(self, fine, coarse, T):
        self._check(self._lib.adi_net_target(self.h, fine.h, coarse.h, ctypes.c_void_p(int(T))))

    def forward(self, X, Y):
        self._check(self._lib.adi_net_forward(self.h, ctypes.c_void_p(int(X)), ctypes.c_void_p(int(Y))))

    def apply(self, solver, Y):
        self._check(self._lib.adi_net_apply(self.h, solver.h, ctypes.c_void_p(int(Y))))

    def train_step(self, X, T, lr):
        self._check(self._lib.adi_net_train_step(self.h, ctypes.c_void_p(int(X)), ctypes.c_void_p(int(T)),
                                                 float(lr)))

    def gradient(self, X, T):
        g = np.zeros(NET_PARAMS, dtype=np.float32)
        loss = ctypes.c_double()
        self._check(self._lib.adi_net_gradient(self.h, ctypes.c_void_p(int(X)), ctypes.c_void_p(int(T)),
                                               g.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), ctypes.byref(loss)))
        return g, loss.value

    def loss(self):
        s = ctypes.c_double()
        c = ctypes.c_int()
        self._check(self._lib.adi_net_loss(self.h, ctypes.byref(s), ctypes.byref(c)))
        return s.value, c.value

    def close(self):
        if getattr(self, "h", None):
            self._lib.adi_net_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fields_distance(a, b):
    """||fields(a) - fields(b)|| / ||fields(b)|| of two FP32 solvers."""
    lib = load_library()
    r = ctypes.c_double()
    st = lib.adi_fields_distance(a.h, b.h, ctypes.byref(r))
    if st != ADI_OK:
        raise AdiError(st, lib.adi_net_last_error(None).decode())
    return r.value


def copy_state(dst, src):
    lib = load_library()
    st = lib.adi_copy_state(dst.h, src.h)
    if st != ADI_OK:
        raise AdiError(st, lib.adi_net_last_error(None).decode())


def corrector_run(net, coarse, fine, m, k=8, guard_every=8, tol=1e-4):
    """Guarded corrected time loop; returns (fallback windows, largest guard distance)."""
    nf = ctypes.c_int()
    me = ctypes.c_double()
    net._check(net._lib.adi_corrector_run(net.h, coarse.h, fine.h, int(m), int(k), int(guard_every), float(tol),
                                          ctypes.byref(nf), ctypes.byref(me)))
    return nf.value, me.value
