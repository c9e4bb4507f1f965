"""One ADI time step of the IGA-FEM Maxwell scheme (FP64 reference).

Test infrastructure only (see ``oracle/__init__.py``).

The time scheme is eqs. (scheme1a)-(scheme1d): two half steps, each implicit in
one part of the split curl C1 - C2.  After discretisation with B-splines each
E half step is eq. (discrete1) / (discrete3) and each H half step eq.
(discrete2) / (discrete4), with the block matrices M, K1, K2, R1, R2, C1, C2
written out after eq. (discrete4).  Row-wise material follows section
"Incorporating non-regular material data": every row rst uses the row's
coefficients a, b, c, d (``oracle.material``).  Readings of the paper taken here:

* C2's third row is M(x)A(x)M (the d/dx2 of the curl split), not M(x)M(x)A.
* In eq. (discrete4) the C1 term carries a minus sign, as in eq. (scheme1d)
  and eq. (strong4).
* The left-hand side of each E component is row-scaled M + c S in one direction
  (its "stiffness" direction) and M in the other two.  As in the Appendix
  (eqs. split1, split2) the direction that carries the material is solved first,
  then the two mass directions.
* Boundary conditions E x n = 0, H . n = 0: E_i has zero first and last
  B-spline coefficients in the two directions other than i, H_i in direction i.
* The current source -J enters the E rows as -b (J, B_rst) at the midpoint
  time of each half step, t_n + tau/4 and t_n + 3 tau/4.
* Material in the right-hand side, two readings.  "row" (the paper's, default):
  every row rst is scaled by its coefficients a, b, c, d formed from the row's
  hat values.  "quad": the right-hand side integrals carry the per-element
  coefficients inside the integrand, sum_e kappa_e int_e (...) B_rst with
  kappa_e in {a_e, b_e, c_e, d_e} formed from the element's eps, mu, sigma by the
  same formulas (the source row then uses b of the element holding the dipole);
  the left-hand sides stay row-scaled, which keeps their Kronecker structure.
  Both agree for uniform material.

Components are ordered (E1, E2, E3, H1, H2, H3), each an array (Nz, Ny, Nx).

Pins: tests/test_oracle_bruteforce.py (one sub-step equals a dense solve of the
full system assembled by 3D quadrature from the weak form, uniform and
heterogeneous material), tests/test_oracle_manufactured.py (the paper's L2 and
H(curl) error bounds for u_A and second order in tau), tests/test_oracle_
stability.py (bounded energy at tau far above the explicit limit).
"""
from dataclasses import dataclass, field

import numpy as np

from . import bspline
from .banded import apply_1d, kron3, solve_lines
from . import material

# direction of the stiffness (material) solve of E_i in half step 1 and 2
STIFF_DIR = {1: ("y", "z", "x"), 2: ("z", "x", "y")}
# Dirichlet directions: E_i is tangential-constrained in the two directions != i
E_DIRICHLET = ({"y", "z"}, {"x", "z"}, {"x", "y"})
H_DIRICHLET = ({"x"}, {"y"}, {"z"})


@dataclass
class Problem:
    n: tuple                # (nx, ny, nz) elements
    p: int                  # B-spline degree
    tau: float              # time step
    a: np.ndarray           # row coefficients, shape (Nz, Ny, Nx)
    b: np.ndarray
    c: np.ndarray
    d: np.ndarray
    mats: dict = field(default_factory=dict)   # axis -> (M, S, A, B)
    source: dict = None     # point source (see set_source)
    rhs_material: str = "row"   # "row" or "quad" (see the module docstring)
    elem: dict = None       # "quad": per-element coefficients a, b, c, d, shape (nz, ny, nx)
    breaks: tuple = None    # per-axis element boundaries (x, y, z), None: uniform elements

    @property
    def shape(self):
        nx, ny, nz = self.n
        p = self.p
        return (nz + p, ny + p, nx + p)


def make_problem(n, p, tau, eps=None, mu=None, sigma=None, rhs_material="row", breaks=None):
    """Build the 1D matrices and the per-row coefficients.

    eps, mu, sigma: per-element arrays (nz, ny, nx) or None for 1, 1, 0.
    rhs_material: "row" (the paper's row scaling) or "quad" (per-element
    coefficients inside the right-hand side integrals).
    breaks: per-axis element boundaries (x, y, z), each n_d + 1 increasing values
    from 0 to 1, or None for uniform elements.
    """
    nx, ny, nz = n
    shp_e = (nz, ny, nx)
    eps = np.ones(shp_e) if eps is None else np.asarray(eps, dtype=np.float64)
    mu = np.ones(shp_e) if mu is None else np.asarray(mu, dtype=np.float64)
    sigma = np.zeros(shp_e) if sigma is None else np.asarray(sigma, dtype=np.float64)
    br = tuple(breaks) if breaks is not None else (None, None, None)
    eh = material.row_hats(eps, n, p, br)
    mh = material.row_hats(mu, n, p, br)
    sh = material.row_hats(sigma, n, p, br)
    a, b, c, d = material.coefficients(eh, mh, sh, tau)
    mats = {"x": bspline.matrices_1d(nx, p, breaks=br[0]), "y": bspline.matrices_1d(ny, p, breaks=br[1]),
            "z": bspline.matrices_1d(nz, p, breaks=br[2])}
    prob = Problem(n=tuple(n), p=p, tau=tau, a=a, b=b, c=c, d=d, mats=mats, rhs_material=rhs_material,
                   breaks=br)
    if rhs_material == "quad":
        ae, be, ce, de = material.coefficients(eps, mu, sigma, tau)
        prob.elem = dict(a=ae, b=be, c=ce, d=de)
    elif rhs_material != "row":
        raise ValueError("rhs_material must be 'row' or 'quad'")
    return prob


def set_source(prob, x0, comp, amp, f0, t0, s):
    """Point dipole J = amp g(t) delta(x - x0) e_comp, comp in {0, 1, 2}.

    (J_comp, B_rst) = amp g(t) B_r(x0) B_s(y0) B_t(z0),
    g(t) = sin(2 pi f0 (t - t0)) exp(-((t - t0) / s)^2).
    """
    nx, ny, nz = prob.n
    br = prob.breaks if prob.breaks is not None else (None, None, None)
    wx = bspline.point_values(nx, prob.p, x0[0], br[0])
    wy = bspline.point_values(ny, prob.p, x0[1], br[1])
    wz = bspline.point_values(nz, prob.p, x0[2], br[2])
    prob.source = dict(w=np.einsum("k,j,i->kji", wz, wy, wx), comp=comp, amp=amp, x0=tuple(x0),
                       f0=f0, t0=t0, s=s)


def source_profile(src, t):
    return np.sin(2 * np.pi * src["f0"] * (t - src["t0"])) * np.exp(-((t - src["t0"]) / src["s"]) ** 2)


def _K(prob, ops, u):
    """Kronecker term: ops = (X, Y, Z) names among 'M', 'S', 'A', 'B'."""
    idx = {"M": 0, "S": 1, "A": 2, "B": 3}
    X = prob.mats["x"][idx[ops[0]]]
    Y = prob.mats["y"][idx[ops[1]]]
    Z = prob.mats["z"][idx[ops[2]]]
    return kron3(X, Y, Z, u)


def _quad_axes(prob):
    """Per axis: Gauss points (p + 1 per element, exact for the degree-2p
    integrands), weights, element of each point, basis values and derivatives."""
    if getattr(prob, "_qa", None) is None:
        out = []
        br = prob.breaks if prob.breaks is not None else (None, None, None)
        for ne, b in zip(prob.n, br):
            x, w, e = bspline.gauss_points(ne, prob.p + 1, b)
            v, d = bspline.eval_basis(ne, prob.p, x, e, b)
            out.append((w, e, v, d))
        prob._qa = out
    return prob._qa


def _Kq(prob, ops, u, kappa):
    """sum_e kappa_e int_e (D_test B_rst) (D_trial u) over the elements e: the
    Kronecker term named by ``ops`` with the per-element coefficient ``kappa``
    (nz, ny, nx) inside the integral.  Per axis, A puts the derivative on the
    trial function, B on the test function, S on both, M on neither."""
    qa = _quad_axes(prob)
    trial = [qa[a][3] if ops[a] in "AS" else qa[a][2] for a in range(3)]
    test = [qa[a][3] if ops[a] in "BS" else qa[a][2] for a in range(3)]
    val = apply_1d(trial[0], apply_1d(trial[1], apply_1d(trial[2], u, "z"), "y"), "x")
    (wx, ex, _, _), (wy, ey, _, _), (wz, ez, _, _) = qa
    wk = np.einsum("k,j,i->kji", wz, wy, wx) * kappa[ez[:, None, None], ey[None, :, None], ex[None, None, :]]
    return apply_1d(test[0].T, apply_1d(test[1].T, apply_1d(test[2].T, val * wk, "z"), "y"), "x")


def _term(prob, ops, u, coef):
    """coef in 'a', 'b', 'c', 'd' or '1': the row-scaled term, or under "quad"
    the term with the per-element coefficient inside the integral."""
    if prob.rhs_material == "quad":
        kappa = np.ones(prob.elem["a"].shape) if coef == "1" else prob.elem[coef]
        return _Kq(prob, ops, u, kappa)
    k = 1.0 if coef == "1" else getattr(prob, coef)
    return k * _K(prob, ops, u)


def _source_b(prob):
    """b of the source row: the row's b ("row"), or b of the element that holds
    the dipole ("quad", the element convention of the point evaluation)."""
    if prob.rhs_material != "quad":
        return prob.b
    x0 = prob.source["x0"]
    br = prob.breaks if prob.breaks is not None else (None, None, None)
    e = [bspline.element_of(prob.n[a], x0[a], br[a]) for a in range(3)]
    return prob.elem["b"][e[2], e[1], e[0]]


def rhs_E(prob, half, E, H, t_mid):
    """Right-hand sides of the E rows, eq. (dupa1ab) for half step 1 (R1) and
    the analogous rows of eq. (discrete3) for half step 2 (R2), row-scaled."""
    E1, E2, E3 = E
    H1, H2, H3 = H
    T = lambda ops, u, k: _term(prob, ops, u, k)
    curl = (
        -T("MMA", H2, "b") + T("MAM", H3, "b"),
        T("MMA", H1, "b") - T("AMM", H3, "b"),
        -T("MAM", H1, "b") + T("AMM", H2, "b"),
    )
    if half == 1:   # R1 = [[0, A(x)B(x)M, 0], [0, 0, M(x)A(x)B], [B(x)M(x)A, 0, 0]]
        cross = (T("ABM", E2, "c"), T("MAB", E3, "c"), T("BMA", E1, "c"))
    else:           # R2 = [[0, 0, A(x)M(x)B], [B(x)A(x)M, 0, 0], [0, M(x)B(x)A, 0]]
        cross = (T("AMB", E3, "c"), T("BAM", E1, "c"), T("MBA", E2, "c"))
    out = []
    for i, Ei in enumerate(E):
        r = T("MMM", Ei, "a") + curl[i] + cross[i]
        if prob.source is not None and prob.source["comp"] == i:
            src = prob.source
            r = r - _source_b(prob) * src["amp"] * source_profile(src, t_mid) * src["w"]
        out.append(r)
    return out


def solve_E(prob, half, rhs):
    """Stiffness direction first (row-scaled M + c S), then the two mass
    directions (Appendix, eqs. split1 and split2)."""
    out = []
    for i in range(3):
        sd = STIFF_DIR[half][i]
        dirs = [sd] + [ax for ax in ("x", "y", "z") if ax != sd]
        u = rhs[i]
        for k, ax in enumerate(dirs):
            M, S, _, _ = prob.mats[ax]
            dch = ax in E_DIRICHLET[i]
            if k == 0:
                u = solve_lines(M, u, ax, prob.p, dch, stiff=S, coef=prob.c)
            else:
                u = solve_lines(M, u, ax, prob.p, dch)
        out.append(u)
    return out


def rhs_H(prob, H, E_alpha, E_beta):
    """RHS of M H_new = M H_old - d C1 E_alpha + d C2 E_beta.

    Half step 1 (eq. discrete2): alpha = E^n, beta = E^{n+1/2}.
    Half step 2 (eq. discrete4, minus sign on C1): alpha = E^{n+1}, beta = E^{n+1/2}.
    C1 = [[0,0,MAM],[MMA,0,0],[0,AMM,0]], C2 = [[0,MMA,0],[0,0,AMM],[MAM,0,0]].
    """
    H1, H2, H3 = H
    Ea1, Ea2, Ea3 = E_alpha
    Eb1, Eb2, Eb3 = E_beta
    T = lambda ops, u: _term(prob, ops, u, "d")
    C1 = (T("MAM", Ea3), T("MMA", Ea1), T("AMM", Ea2))
    C2 = (T("MMA", Eb2), T("AMM", Eb3), T("MAM", Eb1))
    return [_K(prob, "MMM", H[i]) - C1[i] + C2[i] for i in range(3)]


def solve_H(prob, rhs):
    out = []
    for i in range(3):
        u = rhs[i]
        for ax in ("x", "y", "z"):
            M = prob.mats[ax][0]
            u = solve_lines(M, u, ax, prob.p, ax in H_DIRICHLET[i])
        out.append(u)
    return out


def step(prob, state, t):
    """One full step: (E^n, H^n) at time t -> (E^{n+1}, H^{n+1})."""
    E = state[:3]
    H = state[3:]
    tau = prob.tau
    E_half = solve_E(prob, 1, rhs_E(prob, 1, E, H, t + 0.25 * tau))
    H_half = solve_H(prob, rhs_H(prob, H, E, E_half))
    E_new = solve_E(prob, 2, rhs_E(prob, 2, E_half, H_half, t + 0.75 * tau))
    H_new = solve_H(prob, rhs_H(prob, H_half, E_new, E_half))
    return E_new + H_new


def run(prob, state, t0, nsteps):
    state = [np.array(u, dtype=np.float64) for u in state]
    t = t0
    for _ in range(nsteps):
        state = step(prob, state, t)
        t += prob.tau
    return state, t


def zero_state(prob):
    return [np.zeros(prob.shape) for _ in range(6)]


def apply_dirichlet(state):
    """Zero the constrained boundary coefficients (E_i tangential, H_i normal)."""
    out = []
    for i, u in enumerate(state):
        u = np.array(u, dtype=np.float64)
        dirs = E_DIRICHLET[i] if i < 3 else H_DIRICHLET[i - 3]
        if "x" in dirs:
            u[:, :, 0] = 0.0
            u[:, :, -1] = 0.0
        if "y" in dirs:
            u[:, 0, :] = 0.0
            u[:, -1, :] = 0.0
        if "z" in dirs:
            u[0, :, :] = 0.0
            u[-1, :, :] = 0.0
        out.append(u)
    return out
