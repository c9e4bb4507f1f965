"""Seeded synthetic inputs: material maps, dipole positions, random fields.

This module holds input generators only -- none of the method's arithmetic.
Both the GPU library's callers and the CPU oracle's tests take their inputs
from here; neither side imports the other.

Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014; the public-domain 64-bit mixer
with constants 0x9E3779B97F4A7C15, 0xBF58476D1CE4E5B9, 0x94D049BB133111EB),
hashed on (seed, stream, index), so every value is independent of the order of
evaluation.

Head-like 3-phase map (stand-in for the MRI head of the paper, whose classes
are air, tissue and skull; the scan itself is not available): each element is
classified by its centroid against two nested ellipsoids,

* centre 0.5 + U(-0.03, 0.03) per axis, outer semi-axes (0.36, 0.30, 0.40)
  (x, y, z) times 1 + U(-0.05, 0.05), skull thickness 0.04;
* inside the inner ellipsoid: tissue, eps_r = 50 (1 + U(-0.1, 0.1)),
  sigma = 0.7 (1 + U(-0.1, 0.1)), independent per element;
* between the two: skull, eps_r = 12, sigma = 0.05;
* outside: air, eps_r = 1, sigma = 0;  mu_r = 1 everywhere.
Units are non-dimensional with eps0 = mu0 = c0 = 1.
"""
import numpy as np

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)
_G = np.uint64(0x9E3779B97F4A7C15)
_C1 = np.uint64(0xBF58476D1CE4E5B9)
_C2 = np.uint64(0x94D049BB133111EB)

# streams of the generator
S_CENTRE, S_AXES, S_EPS, S_SIGMA, S_DIPOLE, S_FIELD, S_SIZE = 0, 1, 2, 3, 4, 5, 6


def splitmix64(x):
    """SplitMix64 output function applied to state ``x`` (uint64 array)."""
    with np.errstate(over="ignore"):
        z = (np.asarray(x, dtype=np.uint64) + _G) & _M64
        z = ((z ^ (z >> np.uint64(30))) * _C1) & _M64
        z = ((z ^ (z >> np.uint64(27))) * _C2) & _M64
        return z ^ (z >> np.uint64(31))


def uniform(seed, stream, index):
    """U[0, 1) doubles for integer ``index`` (array) in (seed, stream)."""
    with np.errstate(over="ignore"):
        key = splitmix64(np.uint64(seed) * np.uint64(0x100000001B3) + np.uint64(stream))
        z = splitmix64(key + np.asarray(index, dtype=np.uint64))
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def head_map(n, seed):
    """Per-element (eps, mu, sigma), each of shape (nz, ny, nx), and the
    element class (0 air, 1 skull, 2 tissue)."""
    nx, ny, nz = n
    c = 0.5 + (uniform(seed, S_CENTRE, np.arange(3)) * 0.06 - 0.03)
    ao = np.array([0.36, 0.30, 0.40]) * (1.0 + (uniform(seed, S_AXES, np.arange(3)) * 0.1 - 0.05))
    ai = ao - 0.04
    zc = (np.arange(nz) + 0.5) / nz
    yc = (np.arange(ny) + 0.5) / ny
    xc = (np.arange(nx) + 0.5) / nx
    Z, Y, X = np.meshgrid(zc, yc, xc, indexing="ij")
    ri = ((X - c[0]) / ai[0]) ** 2 + ((Y - c[1]) / ai[1]) ** 2 + ((Z - c[2]) / ai[2]) ** 2
    ro = ((X - c[0]) / ao[0]) ** 2 + ((Y - c[1]) / ao[1]) ** 2 + ((Z - c[2]) / ao[2]) ** 2
    cls = np.zeros((nz, ny, nx), dtype=np.int8)
    cls[ro < 1.0] = 1
    cls[ri < 1.0] = 2
    idx = np.arange(nx * ny * nz, dtype=np.uint64).reshape(nz, ny, nx)
    ueps = uniform(seed, S_EPS, idx)
    usig = uniform(seed, S_SIGMA, idx)
    eps = np.ones((nz, ny, nx))
    sigma = np.zeros((nz, ny, nx))
    eps[cls == 1] = 12.0
    sigma[cls == 1] = 0.05
    t = cls == 2
    eps[t] = 50.0 * (1.0 + (ueps[t] * 0.2 - 0.1))
    sigma[t] = 0.7 * (1.0 + (usig[t] * 0.2 - 0.1))
    mu = np.ones((nz, ny, nx))
    return eps, mu, sigma, cls


def dipole(seed):
    """Point dipole: position U[0.2, 0.8]^3, z-directed (component E3),
    Gaussian-modulated sine with f0 = 2, s = 1/f0, t0 = 3 s, amplitude 1."""
    x0 = 0.2 + 0.6 * uniform(seed, S_DIPOLE, np.arange(3))
    f0 = 2.0
    s = 1.0 / f0
    return dict(x0=tuple(float(v) for v in x0), comp=2, amp=1.0, f0=f0, t0=3.0 * s, s=s)


def random_fields(shape, seed, scale=1.0):
    """Six components of U(-scale, scale) coefficients, shape (6,) + shape."""
    size = 6 * int(np.prod(shape))
    u = uniform(seed, S_FIELD, np.arange(size, dtype=np.uint64))
    return ((u * 2.0 - 1.0) * scale).reshape((6,) + tuple(shape))


def random_material(n, seed, eps_range=(1.0, 50.0), sigma_range=(0.0, 0.7),
                    mu_range=(1.0, 1.0)):
    """Unstructured per-element material with independent uniform values."""
    nx, ny, nz = n
    idx = np.arange(nx * ny * nz, dtype=np.uint64).reshape(nz, ny, nx)
    ue = uniform(seed, S_EPS, idx)
    us = uniform(seed, S_SIGMA, idx)
    um = uniform(seed, S_CENTRE + 100, idx)
    eps = eps_range[0] + (eps_range[1] - eps_range[0]) * ue
    sigma = sigma_range[0] + (sigma_range[1] - sigma_range[0]) * us
    mu = mu_range[0] + (mu_range[1] - mu_range[0]) * um
    return eps, mu, sigma


def batch_instances(count=48, seed=2103, n_lo=32, n_hi=128):
    """Heterogeneous batch: instance i has elements per axis drawn from
    U{n_lo..n_hi} and p from {2, 3} (seed + i), its own head map and dipole
    (seed + i).  Returns dicts with n, p, eps, mu, sigma, source."""
    out = []
    for i in range(count):
        s = seed + i
        u = uniform(s, S_SIZE, np.arange(4))
        n = tuple(int(n_lo + np.floor(u[k] * (n_hi - n_lo + 1))) for k in range(3))
        p = 2 if u[3] < 0.5 else 3
        eps, mu, sigma, _ = head_map(n, s)
        out.append(dict(n=n, p=p, eps=eps, mu=mu, sigma=sigma, source=dipole(s)))
    return out


S_NET = 7


def net_init(seed, layers=((9, 32), (32, 32), (32, 32), (32, 6)), last_scale=0.1):
    """Initial corrector weights: w[dz, dy, dx, ci, co] ~ U(-r, r), r = sqrt(6 / (27 ci))
    (He-uniform for ReLU), the last layer scaled by ``last_scale``; biases 0.
    Returns a list of (w, b) FP64 arrays."""
    out = []
    for l, (ci, co) in enumerate(layers):
        size = 27 * ci * co
        u = uniform(seed, S_NET, np.arange(size, dtype=np.uint64) + np.uint64(l << 24))
        r = np.sqrt(6.0 / (27 * ci)) * (last_scale if l == len(layers) - 1 else 1.0)
        out.append((((u * 2.0 - 1.0) * r).reshape(3, 3, 3, ci, co), np.zeros(co)))
    return out
