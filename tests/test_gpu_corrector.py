"""GPU parity of the learned corrector (tcgen05 convolutions, weight gradients,
features / target / apply, Adam, guarded loop) against the FP64 oracle.

Both sides use the same BF16 weights and the same BF16 input X (read back from
the GPU).  The GPU also rounds every hidden activation to BF16; the
``rounded`` oracle forward does the same between layers, so the two differ only
by the FP32 summation order (and the rare BF16 tie that it flips): relative l2
<= 2e-3.  Against the plain FP64 forward the bound is 2e-2, the same bound the
gradients must meet (BF16 activations and output gradients, FP32 sums).
"""
import numpy as np
import pytest

from oracle import convnet as cn
from oracle import maxwell_adi as ma
from paper_2103_06998_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _adi():
    from paper_2103_06998_gb300 import adi
    return adi


def bf16(a):
    """Round to the nearest BF16 (ties to even), returned as float64."""
    a = np.ascontiguousarray(a, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b)))


def _params(seed, bias=0.05):
    ps = inputs.net_init(seed, last_scale=1.0)
    rng = np.random.default_rng(seed)
    return [(bf16(w), bf16(rng.standard_normal(b.shape) * bias)) for w, b in ps]


def _solver(n, p, seed, tau=0.02, k=1):
    adi = _adi()
    eps, mu, sigma, _ = inputs.head_map(n, 2103)
    s = adi.Solver(n, p, tau * k, eps, mu, sigma, precision="fp32")
    s.factor()
    st = ma.apply_dirichlet(list(inputs.random_fields(s.shape, seed)))
    s.set_fields(np.array(st), 0.5)
    return s, st, (eps, mu, sigma)


# The library works on its own non-blocking streams: device-wide synchronisation
# separates torch's allocations and reads from the library's kernels.
def _X(N):
    V = N[0] * N[1] * N[2]
    x = torch.zeros((V, 16), dtype=torch.bfloat16, device="cuda")
    torch.cuda.synchronize()
    return x


def _F(N):
    V = N[0] * N[1] * N[2]
    x = torch.zeros((V, 8), dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    return x


def _grid(x, N):
    """[V][C] device tensor -> (Nz, Ny, Nx, C) float64."""
    torch.cuda.synchronize()
    return x.float().cpu().numpy().astype(np.float64).reshape(N[2], N[1], N[0], -1)


def rounded_forward(params, x):
    h = x
    for l, (w, b) in enumerate(params):
        h = cn.conv3d(h, w, b)
        if l < 3:
            h = bf16(cn.relu(h))
    return h


def _forward_case(n, p, seed):
    adi = _adi()
    s, st, _ = _solver(n, p, seed)
    N = (n[0] + p, n[1] + p, n[2] + p)
    net = adi.Net(N)
    params = _params(seed)
    net.set_params(adi.net_flatten(params))
    X = _X(N)
    Y = _F(N)
    net.features(s, X.data_ptr())
    net.forward(X.data_ptr(), Y.data_ptr())
    torch.cuda.synchronize()
    x = _grid(X, N)[..., :9]
    y = _grid(Y, N)
    # features against the oracle (one BF16 rounding apart)
    prob = ma.make_problem(n, p, 0.02, *inputs.head_map(n, 2103)[:3])
    fx, sc = cn.features(st, prob.a, prob.b, prob.c, 0.02)
    assert np.all(np.abs(x - bf16(fx)) <= 2.0 ** -7 * np.abs(fx) + 1e-30)
    ref_r = rounded_forward(params, x)
    ref = cn.forward(params, x)[-1]
    assert np.all(y[..., 6:] == 0.0)
    e_r = rel(y[..., :6], ref_r)
    e = rel(y[..., :6], ref)
    net.close()
    s.close()
    return e_r, e


def test_small_forward_matches_oracle():
    # grids with N_x <= 16: one 128-row MMA tile per block, several blocks
    e_r, e = _forward_case((11, 7, 5), 2, 1)
    assert e_r < 2e-3 and e < 2e-2, (e_r, e)
    e_r, e = _forward_case((3, 2, 1), 2, 2)  # a single ragged block, fewer voxels than one tile
    assert e_r < 2e-3 and e < 2e-2, (e_r, e)


@pytest.mark.parametrize("n,p", [((38, 9, 4), 2), ((137, 5, 3), 3), ((62, 21, 6), 1), ((14, 62, 38), 2)])
def test_forward_multi_tile_and_segments(n, p):
    # N_x = 40, 140 (two x segments, two 128-row MMA tiles per plane), 63 (ragged y
    # units), 16 x 64 x 40 (work units of several z planes: the plane ring is reused)
    e_r, e = _forward_case(n, p, 3)
    assert e_r < 2e-3 and e < 2e-2, (e_r, e)


def test_gradients_match_oracle():
    adi = _adi()
    n, p = (14, 6, 5), 2
    s, st, _ = _solver(n, p, 4)
    N = (n[0] + p, n[1] + p, n[2] + p)
    net = adi.Net(N)
    params = _params(5)
    net.set_params(adi.net_flatten(params))
    X = _X(N)
    net.features(s, X.data_ptr())
    rng = np.random.default_rng(6)
    t = np.zeros((N[2], N[1], N[0], 8), dtype=np.float32)
    t[..., :6] = rng.standard_normal(t[..., :6].shape) * 0.3
    T = torch.from_numpy(t.reshape(-1, 8)).cuda()
    torch.cuda.synchronize()
    g, loss = net.gradient(X.data_ptr(), T.data_ptr())
    x = _grid(X, N)[..., :9]
    acts = cn.forward(params, x)
    ref_loss = cn.mse(acts[-1], t[..., :6].astype(np.float64))
    grads, _ = cn.backward(params, acts, t[..., :6].astype(np.float64))
    got = adi.net_unflatten(g)
    assert abs(loss - ref_loss) < 1e-2 * ref_loss
    for l in range(4):
        assert rel(got[l][0], grads[l][0]) < 2e-2, (l, rel(got[l][0], grads[l][0]))
        assert rel(got[l][1], grads[l][1]) < 2e-2, (l, rel(got[l][1], grads[l][1]))
    # the padding of the parameter vector gets no gradient
    real = adi.net_flatten([(np.ones_like(w), np.ones_like(b)) for w, b in params]) != 0.0
    assert np.all(g[~real] == 0.0)
    net.close()
    s.close()


def test_target_and_apply_match_oracle():
    adi = _adi()
    n, p = (9, 8, 7), 2
    coarse, st_c, _ = _solver(n, p, 7)
    fine, st_f, _ = _solver(n, p, 8)
    N = (n[0] + p, n[1] + p, n[2] + p)
    net = adi.Net(N)
    X = _X(N)
    T = _F(N)
    net.features(coarse, X.data_ptr())
    net.target(fine, coarse, T.data_ptr())
    torch.cuda.synchronize()
    sc = cn.field_scale(st_c)
    ref_t = cn.target(st_f, st_c, sc)
    assert rel(_grid(T, N)[..., :6], ref_t) < 1e-6
    # apply the exact target: the coarse solver then holds the fine state
    net.apply(coarse, T.data_ptr())
    got, _ = coarse.fields()
    want = cn.apply_correction(st_c, ref_t, sc)
    assert rel(np.array(got), np.array(want)) < 1e-6
    net.close()
    coarse.close()
    fine.close()


def test_adam_step_matches_oracle():
    adi = _adi()
    n, p = (6, 6, 6), 2
    s, st, _ = _solver(n, p, 9)
    N = (n[0] + p,) * 3
    net = adi.Net(N)
    params = _params(10)
    flat = adi.net_flatten(params)
    net.set_params(flat)
    X = _X(N)
    net.features(s, X.data_ptr())
    T = _F(N)
    g, _ = net.gradient(X.data_ptr(), T.data_ptr())
    net.train_step(X.data_ptr(), T.data_ptr(), 1e-3)
    got = net.get_params()
    w, m, v = cn.adam(flat.astype(np.float64), g.astype(np.float64), 0.0, 0.0, 1, 1e-3)
    assert np.max(np.abs(got - w)) < 1e-6
    net.close()
    s.close()


def _pairs(net, n, p, tau, k, seeds, per_map, warm):
    adi = _adi()
    N = tuple(v + p for v in n)
    out = []
    for sd in seeds:
        eps, mu, sigma, _ = inputs.head_map(n, sd)
        src = inputs.dipole(sd)
        fine = adi.Solver(n, p, tau, eps, mu, sigma)
        coarse = adi.Solver(n, p, k * tau, eps, mu, sigma)
        for s in (fine, coarse):
            s.factor()
            s.set_source(src["x0"], src["comp"], src["amp"], src["f0"], src["t0"], src["s"])
        fine.step(warm)
        for _ in range(per_map):
            adi.copy_state(coarse, fine)
            coarse.step(1)
            fine.step(k)
            X = _X(N)
            T = _F(N)
            net.features(coarse, X.data_ptr())
            net.target(fine, coarse, T.data_ptr())
            out.append((X, T))
        fine.close()
        coarse.close()
    torch.cuda.synchronize()
    return out


def test_training_reduces_the_coarse_step_error():
    # what the trained net gains over the plain coarse step: on held-out maps
    # the corrected coarse step is closer to k fine steps than the coarse step
    adi = _adi()
    n, p, k = (14, 14, 14), 2, 8
    N = tuple(v + p for v in n)
    tau = 4.0 * 0.3651 / 14
    net = adi.Net(N)
    net.set_params(adi.net_flatten(inputs.net_init(2103)))
    train = _pairs(net, n, p, tau, k, range(10000, 10006), 6, 20)
    test = _pairs(net, n, p, tau, k, range(20000, 20002), 4, 24)
    for ep in range(40):
        for X, T in train:
            net.train_step(X.data_ptr(), T.data_ptr(), 1e-3 if ep < 30 else 3e-4)
    Y = _F(N)
    base = fix = 0.0
    for X, T in test:
        net.forward(X.data_ptr(), Y.data_ptr())
        torch.cuda.synchronize()
        t = T[:, :6].double()
        base += float((t ** 2).sum())
        fix += float(((t - Y[:, :6].double()) ** 2).sum())
    gain = np.sqrt(base / fix)
    net.close()
    assert gain > 1.5, gain


def test_guarded_loop_follows_its_rule():
    adi = _adi()
    n, p, k, m, every = (10, 9, 8), 2, 4, 6, 3
    N = tuple(v + p for v in n)
    eps, mu, sigma, _ = inputs.head_map(n, 2103)
    src = inputs.dipole(2103)
    tau = 0.02

    def mk(dt):
        s = adi.Solver(n, p, dt, eps, mu, sigma)
        s.factor()
        s.set_source(src["x0"], src["comp"], src["amp"], src["f0"], src["t0"], src["s"])
        s.set_fields(np.array(ma.apply_dirichlet(list(inputs.random_fields(s.shape, 12)))), 0.7)
        return s

    net = adi.Net(N)
    net.set_params(adi.net_flatten(_params(13, bias=0.0)))
    # never falls back: equals corrected coarse steps taken by hand, bit for bit
    coarse, fine = mk(k * tau), mk(tau)
    nf, err = adi.corrector_run(net, coarse, fine, m, k, every, 1e30)
    assert nf == 0 and err > 0.0
    got, t1 = coarse.fields()
    ref = mk(k * tau)
    X, Y = _X(N), _F(N)
    for _ in range(m):
        ref.step(1)
        net.features(ref, X.data_ptr())
        net.forward(X.data_ptr(), Y.data_ptr())
        net.apply(ref, Y.data_ptr())
    want, t2 = ref.fields()
    assert abs(t1 - t2) < 1e-12 and np.array_equal(got, want)
    # always falls back: the plain fine trajectory
    coarse2, fine2 = mk(k * tau), mk(tau)
    nf, _ = adi.corrector_run(net, coarse2, fine2, m, k, every, 1e-30)
    assert nf == (m + every - 1) // every
    got2, t3 = coarse2.fields()
    plain = mk(tau)
    plain.step(k * m)
    want2, t4 = plain.fields()
    assert abs(t3 - t4) < 1e-9
    assert rel(np.array(got2), np.array(want2)) < 1e-6
    for s in (coarse, fine, ref, coarse2, fine2, plain):
        s.close()
    net.close()


def test_net_rejects_bad_arguments():
    adi = _adi()
    N = (7, 6, 5)
    net = adi.Net(N)
    X = _X(N)
    Y = _F(N)
    with pytest.raises(adi.AdiError) as e:
        net.forward(X.data_ptr() + 4, Y.data_ptr())  # not 16-byte aligned
    assert e.value.status == adi.ADI_EINVAL
    with pytest.raises(adi.AdiError) as e:
        net.set_params(np.zeros(adi.NET_PARAMS - 1, dtype=np.float32))
    assert e.value.status == adi.ADI_EINVAL
    bad = np.zeros(adi.NET_PARAMS, dtype=np.float32)
    bad[3] = np.nan
    with pytest.raises(adi.AdiError) as e:
        net.set_params(bad)
    assert e.value.status == adi.ADI_ENUMERIC
    s, _, _ = _solver((3, 3, 3), 2, 1)  # another grid
    with pytest.raises(adi.AdiError) as e:
        net.features(s, X.data_ptr())
    assert e.value.status == adi.ADI_EINVAL
    s.close()
    net.close()
