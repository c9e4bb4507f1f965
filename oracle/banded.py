"""1D operators along one axis of a 3D array, and banded line solves (FP64).

Test infrastructure only (see ``oracle/__init__.py``).

Coefficient arrays have shape (Nz, Ny, Nx): x is the fastest index, as in the
paper's reordering of the right-hand side into N_x rows ("blocks of N_x
consecutive rows", section "Incorporating non-regular material data").  Axis
names: x -> array axis 2, y -> axis 1, z -> axis 0.

* ``apply_1d`` is the definition of one Kronecker factor acting on its index
  (a dense matrix product along that axis).
* ``kron3`` applies X (x), Y (y), Z (z): (X (x) Y (x) Z) u of eq. (discrete1).
* ``solve_lines`` solves, for every line along one axis, the banded system
  whose row k is ``base[k, :] + coef[line, k] * stiff[k, :]`` -- the 1D systems
  of the alternating-direction solver with per-test-function material (section
  "Incorporating non-regular material data"; Appendix, eqs. split1/split2).
  The method is plain Gaussian elimination without pivoting restricted to the
  band.  Dirichlet lines are solved on the interior rows only and their two end
  values are zero.

Pins (tests/test_oracle_banded.py): kron3 against numpy.kron on the flattened
array; solve_lines against numpy.linalg.solve on each line's dense matrix and
against scipy.linalg.solve_banded.
"""
import numpy as np

AXIS = {"x": 2, "y": 1, "z": 0}


def apply_1d(mat, u, axis):
    """out[..., l, ...] = sum_i mat[l, i] u[..., i, ...] along ``axis``."""
    ax = AXIS[axis] if isinstance(axis, str) else axis
    out = np.tensordot(mat, u, axes=([1], [ax]))
    return np.moveaxis(out, 0, ax)


def kron3(X, Y, Z, u):
    """(X (x) Y (x) Z) u: X acts on the x index, Y on y, Z on z."""
    return apply_1d(X, apply_1d(Y, apply_1d(Z, u, "z"), "y"), "x")


def band_of(mat, p):
    """Rows of a banded matrix: out[k, d] = mat[k, k + d - p] (0 outside)."""
    N = mat.shape[0]
    out = np.zeros((N, 2 * p + 1))
    for k in range(N):
        for d in range(2 * p + 1):
            j = k + d - p
            if 0 <= j < N:
                out[k, d] = mat[k, j]
    assert np.allclose(mat, band_to_dense(out, p)), "matrix is not banded"
    return out


def band_to_dense(band, p):
    N = band.shape[0]
    out = np.zeros((N, N))
    for k in range(N):
        for d in range(2 * p + 1):
            j = k + d - p
            if 0 <= j < N:
                out[k, j] = band[k, d]
    return out


def _eliminate(ab, r, p):
    """Gaussian elimination without pivoting, vectorised over lines.

    ab: (n, 2p+1, L) rows of each line's banded matrix (ab[k,d,l] = A_l[k,k+d-p]).
    r:  (n, L) right-hand sides.  Both are overwritten.  Returns x (n, L).
    """
    n = ab.shape[0]
    for k in range(n):
        piv = ab[k, p]
        for i in range(k + 1, min(k + p, n - 1) + 1):
            f = ab[i, k - i + p] / piv
            for j in range(k, min(k + p, n - 1) + 1):
                ab[i, j - i + p] -= f * ab[k, j - k + p]
            r[i] -= f * r[k]
    x = np.zeros_like(r)
    for k in range(n - 1, -1, -1):
        s = r[k].copy()
        for j in range(k + 1, min(k + p, n - 1) + 1):
            s -= ab[k, j - k + p] * x[j]
        x[k] = s / ab[k, p]
    return x


def solve_lines(base, rhs, axis, p, dirichlet, stiff=None, coef=None):
    """Solve the banded 1D systems along every line of ``axis``.

    base, stiff: dense N x N matrices (base = M, stiff = S).  ``coef`` has the
    shape of ``rhs`` and scales the stiff part of each row (per-test-function
    material); with ``stiff is None`` every line has the same matrix ``base``.
    """
    ax = AXIS[axis]
    u = np.moveaxis(rhs, ax, 0)
    shape = u.shape
    N = shape[0]
    r = u.reshape(N, -1).copy()
    L = r.shape[1]
    bb = band_of(base, p)
    ab = np.broadcast_to(bb[:, :, None], (N, 2 * p + 1, L)).copy()
    if stiff is not None:
        sb = band_of(stiff, p)
        c = np.moveaxis(coef, ax, 0).reshape(N, -1)
        ab += c[:, None, :] * sb[:, :, None]
    out = np.zeros_like(r)
    if dirichlet:
        out[1:N - 1] = _eliminate(ab[1:N - 1].copy(), r[1:N - 1].copy(), p)
    else:
        out[:] = _eliminate(ab, r, p)
    return np.moveaxis(out.reshape(shape), 0, ax)
