"""Dense brute-force assembly of one ADI sub-step on tiny meshes (test helper).

Independent of the oracle's code: the basis comes from scipy.interpolate.BSpline
(uniform elements, or the element boundaries ``breaks`` per axis), every
integral is a sum over a full 3D Gauss grid (no Kronecker factorisation),
and the rows are written straight from the weak forms (weak1)-(weak4) of the
paper with per-row coefficients a, b, c, d:

  E rows, half step 1:
    (E1,V1) + c (d2 E1, d2 V1) = a (E1o,V1) + b (-d3 H2 + d2 H3, V1) + c (d1 E2o, d2 V1) - b (J1,V1)
    (E2,V2) + c (d3 E2, d3 V2) = a (E2o,V2) + b ( d3 H1 - d1 H3, V2) + c (d2 E3o, d3 V2) - b (J2,V2)
    (E3,V3) + c (d1 E3, d1 V3) = a (E3o,V3) + b (-d2 H1 + d1 H2, V3) + c (d3 E1o, d1 V3) - b (J3,V3)
  E rows, half step 2: stiffness derivative d3, d1, d2 and cross terms
    (d1 E3o, d3 V1), (d2 E1o, d1 V2), (d3 E2o, d2 V3).
  H rows: (H_new, V) = (H_old, V) - d (C1 E_alpha, V) + d (C2 E_beta, V),
    C1 E = (d2 E3, d3 E1, d1 E2), C2 E = (d3 E2, d1 E3, d2 E1).

The full system is solved with numpy.linalg.solve on the unconstrained DOFs.
"""
import numpy as np
from scipy.interpolate import BSpline


def _edges(n, breaks):
    return np.linspace(0, 1, n + 1) if breaks is None else np.asarray(breaks, dtype=np.float64)


def _basis_1d(n, p, x, breaks=None):
    t = np.concatenate([np.zeros(p), _edges(n, breaks), np.ones(p)])
    N = n + p
    v = np.zeros((len(x), N))
    d = np.zeros((len(x), N))
    for i in range(N):
        c = np.zeros(N)
        c[i] = 1.0
        s = BSpline(t, c, p, extrapolate=False)
        v[:, i] = np.nan_to_num(s(x))
        d[:, i] = np.nan_to_num(s.derivative()(x))
    return v, d


def _gauss(n, q, breaks=None):
    g, w = np.polynomial.legendre.leggauss(q)
    b = _edges(n, breaks)
    x = np.concatenate([0.5 * (b[e] + b[e + 1]) + 0.5 * (b[e + 1] - b[e]) * g for e in range(n)])
    ww = np.concatenate([0.5 * (b[e + 1] - b[e]) * w for e in range(n)])
    return x, ww


class Dense3D:
    """Dense 3D operators on the tensor B-spline space of (nx, ny, nz), p."""

    def __init__(self, n, p, breaks=None):
        self.n, self.p = n, p
        self.breaks = tuple(breaks) if breaks is not None else (None, None, None)
        bx, by, bz = self.breaks
        nx, ny, nz = n
        self.N = (nx + p, ny + p, nz + p)
        q = p + 2
        (x, wx), (y, wy), (z, wz) = _gauss(nx, q, bx), _gauss(ny, q, by), _gauss(nz, q, bz)
        vx, dx = _basis_1d(nx, p, x, bx)
        vy, dy = _basis_1d(ny, p, y, by)
        vz, dz = _basis_1d(nz, p, z, bz)
        # index order (k, j, i) with i (x) fastest, points (qz, qy, qx)
        self.W = np.kron(np.kron(wz, wy), wx)
        self.phi = np.kron(np.kron(vz, vy), vx)
        self.grad = (np.kron(np.kron(vz, vy), dx),   # d/dx1
                     np.kron(np.kron(vz, dy), vx),   # d/dx2
                     np.kron(np.kron(dz, vy), vx))   # d/dx3
        self.pts = (x, y, z)
        self.vals1d = (vx, vy, vz)

    def inner(self, test_deriv, trial_deriv):
        """G[row, col] = int D_test B_row D_trial B_col (None = no derivative)."""
        T = self.phi if test_deriv is None else self.grad[test_deriv]
        U = self.phi if trial_deriv is None else self.grad[trial_deriv]
        return T.T @ (self.W[:, None] * U)

    def inner_w(self, test_deriv, trial_deriv, elem_field):
        """G[row, col] = sum_e f_e int_e D_test B_row D_trial B_col for a
        per-element field f (nz, ny, nx): the weight of every Gauss point is
        multiplied by f of the element that holds it."""
        T = self.phi if test_deriv is None else self.grad[test_deriv]
        U = self.phi if trial_deriv is None else self.grad[trial_deriv]
        return T.T @ ((self.W * self._at_points(elem_field))[:, None] * U)

    def _at_points(self, elem_field):
        nx, ny, nz = self.n
        q = self.p + 2
        ex = np.repeat(np.arange(nx), q)
        ey = np.repeat(np.arange(ny), q)
        ez = np.repeat(np.arange(nz), q)
        return elem_field[ez[:, None, None], ey[None, :, None], ex[None, None, :]].ravel()

    def free(self, dirs):
        """Mask of unconstrained DOFs for Dirichlet directions ``dirs`` (0,1,2)."""
        Nx, Ny, Nz = self.N
        k, j, i = np.meshgrid(np.arange(Nz), np.arange(Ny), np.arange(Nx), indexing="ij")
        m = np.ones((Nz, Ny, Nx), dtype=bool)
        for d, idx, Nd in ((0, i, Nx), (1, j, Ny), (2, k, Nz)):
            if d in dirs:
                m &= (idx > 0) & (idx < Nd - 1)
        return m.ravel()

    def point_row(self, x0):
        """B_rst(x0) for all rst (flattened)."""
        out = []
        for d in range(3):
            v, _ = _basis_1d(self.n[d], self.p, np.array([x0[d]]), self.breaks[d])
            out.append(v[0])
        return np.kron(np.kron(out[2], out[1]), out[0])

    def hat(self, elem_field):
        """int f B_rst / int B_rst for a per-element field (nz, ny, nx)."""
        nx, ny, nz = self.n
        q = self.p + 2
        ex = np.repeat(np.arange(nx), q)
        ey = np.repeat(np.arange(ny), q)
        ez = np.repeat(np.arange(nz), q)
        fq = elem_field[ez[:, None, None], ey[None, :, None], ex[None, None, :]].ravel()
        num = self.phi.T @ (self.W * fq)
        den = self.phi.T @ self.W
        return (num / den).reshape(self.N[2], self.N[1], self.N[0])


E_DIR = ((1, 2), (0, 2), (0, 1))
H_DIR = ((0,), (1,), (2,))


def e_substep(D, half, E, H, a, b, c, J=None, elem=None):
    """Dense solve of the E rows of half step ``half``; returns (E1, E2, E3).
    elem = (a_e, b_e, c_e, b_src): per-element coefficients inside the
    right-hand side integrals (and b of the source row) instead of the row
    scaling by a, b, c; the left-hand side stays row-scaled by c."""
    f = lambda u: np.asarray(u).ravel()
    a, b, c = f(a), f(b), f(c)
    mass = D.inner(None, None)
    E = [f(u) for u in E]
    H = [f(u) for u in H]
    if half == 1:
        stiff = (1, 2, 0)
        cross = ((1, 0, E[1]), (2, 1, E[2]), (0, 2, E[0]))   # (test deriv, trial deriv, field)
    else:
        stiff = (2, 0, 1)
        cross = ((2, 0, E[2]), (0, 1, E[0]), (1, 2, E[1]))
    if elem is None:
        G = lambda td, ud, k: k * D.inner(td, ud)          # row-scaled
        ka, kb, kc, bsrc = a[:, None], b[:, None], c[:, None], b
    else:
        G = lambda td, ud, k: D.inner_w(td, ud, k)         # coefficient in the integrand
        ka, kb, kc, bsrc = elem
    curl = (-G(None, 2, kb) @ H[1] + G(None, 1, kb) @ H[2],
            G(None, 2, kb) @ H[0] - G(None, 0, kb) @ H[2],
            -G(None, 1, kb) @ H[0] + G(None, 0, kb) @ H[1])
    out = []
    for i in range(3):
        s = stiff[i]
        lhs = mass + c[:, None] * D.inner(s, s)
        td, ud, fld = cross[i]
        rhs = G(None, None, ka) @ E[i] + curl[i] + G(td, ud, kc) @ fld
        if J is not None:
            rhs = rhs - bsrc * J[i]
        m = D.free(E_DIR[i])
        x = np.zeros_like(rhs)
        x[m] = np.linalg.solve(lhs[np.ix_(m, m)], rhs[m])
        out.append(x.reshape(D.N[2], D.N[1], D.N[0]))
    return out


def h_substep(D, H, E_alpha, E_beta, d, d_elem=None):
    """Dense solve of the H rows; d_elem: per-element d inside the integrals
    instead of the row scaling by d."""
    f = lambda u: np.asarray(u).ravel()
    d = f(d)
    mass = D.inner(None, None)
    Ea = [f(u) for u in E_alpha]
    Eb = [f(u) for u in E_beta]
    if d_elem is None:
        G = lambda ud: d[:, None] * D.inner(None, ud)
    else:
        G = lambda ud: D.inner_w(None, ud, d_elem)
    C1 = (G(1) @ Ea[2], G(2) @ Ea[0], G(0) @ Ea[1])
    C2 = (G(2) @ Eb[1], G(0) @ Eb[2], G(1) @ Eb[0])
    out = []
    for i in range(3):
        rhs = mass @ f(H[i]) - C1[i] + C2[i]
        m = D.free(H_DIR[i])
        x = np.zeros_like(rhs)
        x[m] = np.linalg.solve(mass[np.ix_(m, m)], rhs[m])
        out.append(x.reshape(D.N[2], D.N[1], D.N[0]))
    return out
