"""Training data, training and evaluation of the learned coarse-step corrector.

Every step runs in the library's kernels (``adi_net_*``, ``adi_step``); this
module only sequences the calls and keeps the device arrays (torch tensors).

* ``pairs``: for each seeded head-like map, a fine solver (time step tau =
  4 dt_CFL) runs from zero fields with the map's dipole; after ``warm`` steps,
  every k fine steps the state is copied into a coarse solver (k tau), which
  takes one step.  X = features of the coarse result, T = (fine - coarse) / s.
* ``train``: Adam on the mean squared error, one pair per step, pairs shuffled
  every epoch with a seeded permutation.
* ``evaluate``: relative l2 of (T - net(X)) against that of T over held-out
  pairs: the gain of the corrected coarse step over the plain one.

Command line: ``python -m paper_2103_06998_gb300.corrector --out weights.f32``
trains on 2,000 pairs at 64^3 elements (p = 2, maps 10000 + i, dipole carrier
frequencies 2 and 1 alternating) and writes the FP32 parameter vector of
include/adi_corrector.h.  At the same Courant number a field driven at f0 = 1
on 64^3 has the wavelength in grid units of f0 = 2 on 128^3, the resolution the
corrector runs at; without those maps the net over-corrects there.
"""
import argparse
import os
import sys
import time

import numpy as np

from . import adi, inputs

HERE = os.path.dirname(os.path.abspath(__file__))
WEIGHTS = os.path.join(HERE, "weights", "corrector_64_p2_k8.f32")


def _torch():
    import torch
    return torch


def cfl_tau(n, p, eps, mu, sigma, factor=4.0):
    """factor x the explicit CFL limit of the map (the library's adi_cfl_dt)."""
    s = adi.Solver(n, p, 1.0, eps, mu, sigma)
    dt = factor * s.cfl_dt()
    s.close()
    return dt


def solver_pair(n, p, k, seed, tau=None, f0=None, tau_factor=4.0):
    """Fine (tau) and coarse (k tau) FP32 solvers on map `seed` with its dipole
    (carrier frequency f0 if given, else the dipole's own, with s = 1/f0, t0 = 3 s);
    tau defaults to tau_factor x the map's explicit limit."""
    eps, mu, sigma, _ = inputs.head_map(n, seed)
    if tau is None:
        tau = cfl_tau(n, p, eps, mu, sigma, tau_factor)
    src = inputs.dipole(seed)
    if f0 is not None:
        src = dict(src, f0=f0, s=1.0 / f0, t0=3.0 / f0)
    out = []
    for dt in (tau, k * tau):
        s = adi.Solver(n, p, dt, eps, mu, sigma)
        s.factor()
        s.set_source(src["x0"], src["comp"], src["amp"], src["f0"], src["t0"], src["s"])
        out.append(s)
    return out[0], out[1], tau


def pairs(net, n, p, k, seeds, per_map, warm_time=0.5, f0s=(None,), tau_factor=4.0):
    """List of (X, T) device tensors, `per_map` consecutive pairs per map; map i
    is driven at carrier frequency f0s[i % len(f0s)] (None: the dipole's own);
    fine step tau_factor x the explicit limit, coarse step k times that."""
    torch = _torch()
    N = tuple(v + p for v in n)
    V = N[0] * N[1] * N[2]
    out = []
    for m, sd in enumerate(seeds):
        fine, coarse, tau = solver_pair(n, p, k, sd, f0=f0s[m % len(f0s)], tau_factor=tau_factor)
        fine.step(max(1, int(round(warm_time / tau))))
        for _ in range(per_map):
            X = torch.zeros((V, 16), dtype=torch.bfloat16, device="cuda")
            T = torch.zeros((V, 8), dtype=torch.float32, device="cuda")
            torch.cuda.synchronize()
            adi.copy_state(coarse, fine)
            coarse.step(1)
            fine.step(k)
            net.features(coarse, X.data_ptr())
            net.target(fine, coarse, T.data_ptr())
            out.append((X, T))
        fine.sync()
        coarse.sync()
        fine.close()
        coarse.close()
    torch.cuda.synchronize()
    return out


def train(net, data, epochs, lr=1e-3, lr_final=1e-4, seed=2103, log=None):
    """Adam over `epochs` passes; lr decays geometrically to lr_final.  Returns
    the mean loss per epoch."""
    hist = []
    rng = np.random.default_rng(seed)
    total = epochs * len(data)
    step = 0
    for ep in range(epochs):
        for i in rng.permutation(len(data)):
            X, T = data[i]
            r = lr * (lr_final / lr) ** (step / max(1, total - 1))
            net.train_step(X.data_ptr(), T.data_ptr(), r)
            step += 1
        s, c = net.loss()
        hist.append(s / max(c, 1))
        if log:
            log("epoch %d loss %.4e" % (ep, hist[-1]))
    return hist


def evaluate(net, data):
    """Relative l2 errors (plain coarse step, corrected coarse step) against the
    k fine steps, summed over `data`: ||T|| and ||T - net(X)|| over ||X_fields + T||
    (all scaled by the same s; X holds coarse / s rounded to BF16)."""
    torch = _torch()
    base = fix = ref = 0.0
    Y = None
    for X, T in data:
        if Y is None or Y.shape != T.shape:
            Y = torch.zeros_like(T)
            torch.cuda.synchronize()
        net.forward(X.data_ptr(), Y.data_ptr())
        torch.cuda.synchronize()
        t = T[:, :6].double()
        base += float((t ** 2).sum())
        fix += float(((t - Y[:, :6].double()) ** 2).sum())
        ref += float(((X[:, :6].double() + t) ** 2).sum())
    return float(np.sqrt(base / ref)), float(np.sqrt(fix / ref))


def save(flat, path):
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    np.asarray(flat, dtype="<f4").tofile(path)


def load(path=WEIGHTS):
    a = np.fromfile(path, dtype="<f4")
    if a.size != adi.NET_PARAMS:
        raise ValueError("%s: expected %d floats, found %d" % (path, adi.NET_PARAMS, a.size))
    return a


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--out", default=WEIGHTS)
    ap.add_argument("--n", type=int, default=64)
    ap.add_argument("--p", type=int, default=2)
    ap.add_argument("--k", type=int, default=8)
    ap.add_argument("--tau-factor", type=float, default=4.0, help="fine time step in units of the explicit limit")
    ap.add_argument("--maps", type=int, default=80)
    ap.add_argument("--per-map", type=int, default=25)
    ap.add_argument("--epochs", type=int, default=6)
    ap.add_argument("--test-maps", type=int, default=4)
    ap.add_argument("--f0", default="2,1",
                    help="carrier frequencies of the training maps, cycled (2 = the workloads' dipole; 1 at 64^3 "
                         "has the grid-unit wavelength of 2 at 128^3, the inference resolution)")
    a = ap.parse_args(argv)
    log = lambda m: print(m, flush=True)
    n = (a.n,) * 3
    N = tuple(v + a.p for v in n)
    net = adi.Net(N)
    net.set_params(adi.net_flatten(inputs.net_init(2103)))
    t0 = time.time()
    f0s = tuple(float(v) for v in a.f0.split(","))
    data = pairs(net, n, a.p, a.k, range(10000, 10000 + a.maps), a.per_map, f0s=f0s, tau_factor=a.tau_factor)
    held = pairs(net, n, a.p, a.k, range(20000, 20000 + a.test_maps), a.per_map, tau_factor=a.tau_factor)
    log("pairs: %d train, %d held out, %.1f s" % (len(data), len(held), time.time() - t0))
    b0, f0 = evaluate(net, held)
    t0 = time.time()
    train(net, data, a.epochs, log=log)
    log("training: %.1f s" % (time.time() - t0))
    b1, f1 = evaluate(net, held)
    log("held-out relative error against %d fine steps: plain coarse step %.4e, corrected %.4e "
        "(gain %.2f; untrained net %.2f)" % (a.k, b1, f1, b1 / f1, b0 / f0))
    save(net.get_params(), a.out)
    log("wrote %s" % a.out)
    net.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
