"""Pins of the corrector net oracle (oracle/convnet.py) against definitions that
do not reuse its code: brute-force sums, impulse responses, finite differences,
the adjoint identity and Adam's closed form."""
import itertools

import numpy as np

from oracle import convnet as cn
from paper_2103_06998_gb300 import inputs


def _rand(shape, seed):
    return np.random.default_rng(seed).standard_normal(shape)


def test_conv3d_equals_brute_force_sum():
    u = _rand((3, 4, 5, 2), 1)
    w = _rand((3, 3, 3, 2, 3), 2)
    b = _rand(3, 3)
    got = cn.conv3d(u, w, b)
    Z, Y, X, _ = u.shape
    for z, y, x in itertools.product(range(Z), range(Y), range(X)):
        for co in range(3):
            acc = b[co]
            for dz, dy, dx, ci in itertools.product(range(3), range(3), range(3), range(2)):
                zz, yy, xx = z + dz - 1, y + dy - 1, x + dx - 1
                if 0 <= zz < Z and 0 <= yy < Y and 0 <= xx < X:
                    acc += u[zz, yy, xx, ci] * w[dz, dy, dx, ci, co]
            assert abs(got[z, y, x, co] - acc) < 1e-12


def test_conv3d_impulse_response_fixes_orientation():
    # a unit impulse at q gives out[q - tap + 1] = w[tap]: the tap (0, 0, 0)
    # weight appears one voxel further along every axis
    u = np.zeros((5, 5, 5, 1))
    u[2, 2, 2, 0] = 1.0
    w = np.zeros((3, 3, 3, 1, 1))
    w[0, 1, 2, 0, 0] = 7.0
    out = cn.conv3d(u, w)
    assert out[3, 2, 1, 0] == 7.0 and np.count_nonzero(out) == 1


def test_transpose_is_the_adjoint():
    u = _rand((4, 3, 5, 3), 4)
    v = _rand((4, 3, 5, 2), 5)
    w = _rand((3, 3, 3, 3, 2), 6)
    lhs = np.sum(cn.conv3d(u, w) * v)
    rhs = np.sum(u * cn.conv3d_transpose(v, w))
    assert abs(lhs - rhs) < 1e-10 * abs(lhs)


def test_gradients_match_central_differences():
    layers = ((9, 4), (4, 4), (4, 4), (4, 6))
    params = inputs.net_init(11, layers, last_scale=1.0)
    params = [(w, _rand(b.shape, 20 + i) * 0.1) for i, (w, b) in enumerate(params)]
    x = _rand((3, 4, 5, 9), 7)
    t = _rand((3, 4, 5, 6), 8)
    acts = cn.forward(params, x)
    grads, gx = cn.backward(params, acts, t)
    rng = np.random.default_rng(9)

    def loss(ps, xx):
        return cn.mse(cn.forward(ps, xx)[-1], t)

    h = 1e-6
    for l in range(4):
        for which in (0, 1):
            arr = params[l][which]
            for _ in range(6):
                idx = tuple(rng.integers(0, s) for s in arr.shape)
                keep = arr[idx]
                arr[idx] = keep + h
                fp = loss(params, x)
                arr[idx] = keep - h
                fm = loss(params, x)
                arr[idx] = keep
                fd = (fp - fm) / (2 * h)
                an = grads[l][which][idx]
                assert abs(fd - an) <= 1e-6 * max(abs(fd), 1e-3), (l, which, idx, fd, an)
    for _ in range(6):
        idx = tuple(rng.integers(0, s) for s in x.shape)
        keep = x[idx]
        x[idx] = keep + h
        fp = loss(params, x)
        x[idx] = keep - h
        fm = loss(params, x)
        x[idx] = keep
        fd = (fp - fm) / (2 * h)
        assert abs(fd - gx[idx]) <= 1e-6 * max(abs(fd), 1e-3)


def test_relu_derivative_at_zero_is_zero():
    # a layer input exactly 0 passes no gradient back
    w = np.zeros((3, 3, 3, 1, 1))
    w[1, 1, 1, 0, 0] = 1.0
    params = [(w, np.array([-1.0])), (w.copy(), np.zeros(1))]
    x = np.ones((1, 1, 1, 1))     # layer 1: relu(1 - 1) = 0
    acts = cn.forward(params, x)
    grads, gx = cn.backward(params, acts, np.ones((1, 1, 1, 1)))
    assert acts[1][0, 0, 0, 0] == 0.0 and gx[0, 0, 0, 0] == 0.0


def test_adam_closed_form_under_constant_gradient():
    # with a constant gradient the bias-corrected moments are g and g^2
    # exactly, so every step moves w by -lr g / (|g| + eps)
    g = np.array([0.3, -2.0, 1e-3])
    w = np.zeros(3)
    m = np.zeros(3)
    v = np.zeros(3)
    for t in range(1, 6):
        w, m, v = cn.adam(w, g, m, v, t, lr=0.01)
    np.testing.assert_allclose(w, -5 * 0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12)


def test_adam_minimises_a_quadratic():
    target = np.array([1.0, -3.0, 0.5])
    w = np.zeros(3)
    m = np.zeros(3)
    v = np.zeros(3)
    for t in range(1, 3001):
        w, m, v = cn.adam(w, w - target, m, v, t, lr=0.01)
    assert np.max(np.abs(w - target)) < 1e-3


def test_features_scale_invariance_and_uniform_material():
    st = [_rand((3, 4, 5), 30 + i) for i in range(6)]
    shp = (3, 4, 5)
    tau = 0.05
    a = np.ones(shp)
    b = np.full(shp, tau / 2)
    c = np.full(shp, tau ** 2 / 4)
    f1, s1 = cn.features(st, a, b, c, tau)
    f2, s2 = cn.features([3.0 * u for u in st], a, b, c, tau)
    np.testing.assert_allclose(f1, f2, rtol=1e-14, atol=1e-14)
    assert abs(s2 - 3.0 * s1) < 1e-14 * s2
    np.testing.assert_allclose(f1[..., 6:], 1.0, rtol=1e-14)
    assert abs(np.sqrt(np.mean(f1[..., :6] ** 2)) - 1.0) < 1e-14
    # the correction with the exact target reproduces the fine state
    fine = [u + 0.01 * _rand(shp, 40 + i) for i, u in enumerate(st)]
    from oracle import maxwell_adi as ma
    st_d = ma.apply_dirichlet(st)
    fine_d = ma.apply_dirichlet(fine)
    y = cn.target(fine_d, st_d, s1)
    got = cn.apply_correction(st_d, y, s1)
    for g_, f_ in zip(got, fine_d):
        np.testing.assert_allclose(g_, f_, rtol=1e-13, atol=1e-15)
