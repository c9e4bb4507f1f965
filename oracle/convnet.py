"""Learned coarse-step corrector: 3D convolution net, loss, gradients, Adam (FP64).

Test infrastructure only (see ``oracle/__init__.py``).

The paper has no learned component.  The corrector is an addition on top of the
ADI method: one ADI step of length 8 tau is followed by a small convolution net
that predicts the difference between eight steps of length tau and that one
step, both started from the same state.  Definitions written out here:

* ``conv3d``: channels-last arrays ``u[z, y, x, c]``, weights ``w[dz, dy, dx,
  ci, co]`` (3 x 3 x 3 taps), bias ``b[co]``, zero padding of one voxel:

      out[z, y, x, co] = b[co] + sum_{dz, dy, dx, ci}
                         u[z + dz - 1, y + dy - 1, x + dx - 1, ci] w[dz, dy, dx, ci, co]

  (a cross-correlation, as in convolutional nets).  Voxels are the coefficient
  points of the B-spline space (the net runs on the coefficient grid).
* ``forward``: layers 9 -> 32 -> 32 -> 32 -> 6, ReLU after the first three.
* ``mse``: mean of the squared error over all voxels and output channels.
* ``backward``: reverse-mode derivative of mse(forward(x)) by the chain rule,
  layer by layer; the derivative of ReLU at 0 is taken as 0.
* ``adam``: Kingma and Ba, "Adam: a method for stochastic optimization"
  (ICLR 2015), Algorithm 1, with bias-corrected moments.
* ``features`` / ``apply_correction``: what the net sees and how its output is
  used.  Input channels: the six field components divided by
  s = sqrt(mean of the squared coefficients of all six components) of the
  coarse state, then the row coefficients a, 2b/tau, 4c/tau^2 of the coarse
  step (dimensionless, in (-1, 1]; they determine eps^, mu^, sigma^ for a given
  tau).  Target: (fine - coarse) / s.  Correction: coarse + s * net(x), then
  the Dirichlet coefficients are set to zero again.

Pins (tests/test_oracle_convnet.py): conv3d against a per-voxel brute-force sum
and against a single-tap impulse response (fixes the orientation); gradients
against central finite differences; the transpose used in backward against the
adjoint identity <conv(u), v> = <u, conv^T(v)>; Adam against its closed form
under a constant gradient; features against their scale invariance and the
uniform-material values (1, 1, 1).
"""
import numpy as np

# channels of the four layers
LAYERS = ((9, 32), (32, 32), (32, 32), (32, 6))
N_IN, N_OUT = 9, 6


def _shifted(u, dz, dy, dx):
    """u[z + dz - 1, y + dy - 1, x + dx - 1, :] with zeros outside the grid."""
    Z, Y, X, _ = u.shape
    pad = np.zeros((Z + 2, Y + 2, X + 2, u.shape[3]))
    pad[1:-1, 1:-1, 1:-1] = u
    return pad[dz:dz + Z, dy:dy + Y, dx:dx + X]


def conv3d(u, w, b=None):
    """3 x 3 x 3 cross-correlation with zero padding; u (Z,Y,X,ci), w (3,3,3,ci,co)."""
    Z, Y, X, _ = u.shape
    out = np.zeros((Z, Y, X, w.shape[4]))
    for dz in range(3):
        for dy in range(3):
            for dx in range(3):
                out += np.tensordot(_shifted(u, dz, dy, dx), w[dz, dy, dx], axes=([3], [0]))
    if b is not None:
        out += b
    return out


def conv3d_transpose(v, w):
    """Adjoint of conv3d without bias: returns g with <conv3d(u, w), v> = <u, g>.

    g[q, ci] = sum_{taps, co} v[q - tap + 1, co] w[tap, ci, co]."""
    Z, Y, X, _ = v.shape
    pad = np.zeros((Z + 2, Y + 2, X + 2, w.shape[3]))
    for dz in range(3):
        for dy in range(3):
            for dx in range(3):
                pad[dz:dz + Z, dy:dy + Y, dx:dx + X] += np.tensordot(v, w[dz, dy, dx], axes=([3], [1]))
    return pad[1:-1, 1:-1, 1:-1]


def conv3d_weight_grad(u, v):
    """dL/dw[tap, ci, co] = sum_q u[q + tap - 1, ci] v[q, co] for out = conv3d(u, w)."""
    gw = np.zeros((3, 3, 3, u.shape[3], v.shape[3]))
    for dz in range(3):
        for dy in range(3):
            for dx in range(3):
                gw[dz, dy, dx] = np.tensordot(_shifted(u, dz, dy, dx), v, axes=([0, 1, 2], [0, 1, 2]))
    return gw


def relu(x):
    return np.maximum(x, 0.0)


def forward(params, x):
    """params: list of (w, b) per layer.  Returns [x, a1, a2, a3, y] (inputs of
    every layer and the output)."""
    acts = [np.asarray(x, dtype=np.float64)]
    h = acts[0]
    for l, (w, b) in enumerate(params):
        h = conv3d(h, w, b)
        if l < len(params) - 1:
            h = relu(h)
        acts.append(h)
    return acts


def mse(y, t):
    return float(np.mean((y - t) ** 2))


def backward(params, acts, t):
    """Gradients of mse(acts[-1], t) for every (w, b), and of the input."""
    y = acts[-1]
    g = 2.0 * (y - t) / y.size          # dL/dy
    grads = [None] * len(params)
    for l in range(len(params) - 1, -1, -1):
        w, _ = params[l]
        u = acts[l]                     # input of layer l
        grads[l] = (conv3d_weight_grad(u, g), g.sum(axis=(0, 1, 2)))
        g = conv3d_transpose(g, w)      # dL/du
        if l > 0:
            g = g * (u > 0.0)           # through the ReLU that produced u
    return grads, g


def adam(w, grad, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update at step t >= 1; returns (w, m, v)."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mhat = m / (1.0 - beta1 ** t)
    vhat = v / (1.0 - beta2 ** t)
    return w - lr * mhat / (np.sqrt(vhat) + eps), m, v


def field_scale(state):
    """s = sqrt(mean of the squared coefficients over all six components)."""
    return float(np.sqrt(sum(np.sum(np.asarray(u, np.float64) ** 2) for u in state) /
                         sum(np.asarray(u).size for u in state)))


def features(state, a, b, c, tau):
    """Net input (Z, Y, X, 9) and the scale s of a coarse state."""
    s = field_scale(state)
    inv = 1.0 / s if s > 0.0 else 0.0
    ch = [np.asarray(u, np.float64) * inv for u in state]
    ch += [np.asarray(a, np.float64), 2.0 * np.asarray(b) / tau, 4.0 * np.asarray(c) / tau ** 2]
    return np.stack(ch, axis=-1), s


def target(fine, coarse, s):
    """(fine - coarse) / s, channels last (Z, Y, X, 6)."""
    inv = 1.0 / s if s > 0.0 else 0.0
    return np.stack([(np.asarray(f, np.float64) - g) * inv for f, g in zip(fine, coarse)], axis=-1)


def apply_correction(state, y, s):
    """coarse + s * y, then the Dirichlet coefficients zeroed."""
    from .maxwell_adi import apply_dirichlet
    return apply_dirichlet([np.asarray(u, np.float64) + s * y[..., i] for i, u in enumerate(state)])
