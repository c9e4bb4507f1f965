"""Benchmark: field DOF-steps/s of the ADI isogeometric Maxwell step on GB300.

Workload: 256^3 elements, p = 2 (258^3 coefficients x 6 components), seeded
head-like 3-phase material map (seed 2103), z-directed point dipole, tau = 4x
the explicit CFL limit, FP32 arithmetic.  One bench "step" is one full ADI time
step (four sub-solves).  The working set (fields + row coefficients, ~0.7 GB)
is far larger than the 129 MB L2, so no explicit flush is needed between
steps.

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU
oracle instead (the only reference that exists for this method).  With
``--gpus N`` under torchrun every rank steps its own independent replica
(the single-instance path does not shard without an exchange step).
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "field DOF-steps/s at 256^3 p=2 (mixed/learned vs FP32 GPU), % HBM roofline"
UNIT = "DOF-steps/s"
N_ELEM = 256
P = 2
SEED = 2103
FP64_PEAK_TFLOPS = 1.25  # nominal dense FP64 of GB300


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--n", type=int, default=N_ELEM, help="elements per axis (default 256)")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64", "mixed"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--mode", default="single", choices=["single", "batched", "learned"],
                    help="batched: 48 heterogeneous instances (32-128 elements per axis, p in {2,3}); "
                         "learned: guarded corrector at 128^3 against plain steps")
    ap.add_argument("--weights", default=None, help="learned: corrector parameter file (FP32)")
    ap.add_argument("--coarse-steps", type=int, default=400, help="learned: coarse steps of the guarded run")
    ap.add_argument("--tol", type=float, default=1e-4, help="learned: guard tolerance (relative l2 per coarse step)")
    ap.add_argument("--p", type=int, default=P, help="B-spline degree of the single-instance workload (default 2)")
    ap.add_argument("--serial-chains", action="store_true",
                    help="run the three per-component chains of a half step one after another (default: concurrent)")
    ap.add_argument("--no-extras", action="store_true",
                    help="single mode: skip the mixed, batched and learned measurements added to the line")
    return ap.parse_args()


def workload(n):
    from paper_2103_06998_gb300 import inputs
    eps, mu, sigma, _ = inputs.head_map((n, n, n), SEED)
    src = inputs.dipole(SEED)
    return eps, mu, sigma, src


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def kernel_source_hash():
    """Hash of the step kernels' source with comments and whitespace removed, so
    that only code changes invalidate recorded counters."""
    import re
    h = hashlib.sha256()
    for f in ("adi_kernels.cu", "adi_internal.h"):
        txt = open(os.path.join(ROOT, "paper_2103_06998_gb300", "csrc", f)).read()
        txt = re.sub(r"/\*.*?\*/", " ", txt, flags=re.S)
        txt = re.sub(r"//[^\n]*", " ", txt)
        h.update(" ".join(txt.split()).encode())
    return h.hexdigest()[:12]


def ncu_traffic(kernel, n):
    """Per-launch DRAM bytes of ``kernel`` from the committed ncu summary, or
    None when the summary was taken on a different kernel source."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.txt")
    if not os.path.exists(path):
        return None
    src = kernel_source_hash()
    for line in open(path):
        parts = line.split()
        if len(parts) >= 4 and not line.startswith("#") and parts[0] == kernel and parts[1] == str(n) and parts[3] == src:
            return float(parts[2])
    return None


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        self.f.flush()
        rows = []
        for line in open(self.f.name):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i in range(4) if r[i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def cpu_baseline(n, eps, mu, sigma, src, tau):
    """The FP64 oracle on the host cores, on a bounded sample: the E and H
    sub-solves of half step 1 of one time step at the full size (half of a
    time step), scaled to DOF-steps/s."""
    from oracle import maxwell_adi as ma
    from paper_2103_06998_gb300 import inputs
    prob = ma.make_problem((n, n, n), P, tau, eps, mu, sigma)
    ma.set_source(prob, src["x0"], src["comp"], src["amp"], src["f0"], src["t0"], src["s"])
    st = ma.apply_dirichlet(list(inputs.random_fields(prob.shape, 3)))
    t0 = time.perf_counter()
    E_half = ma.solve_E(prob, 1, ma.rhs_E(prob, 1, st[:3], st[3:], 1.5 + 0.25 * tau))
    ma.solve_H(prob, ma.rhs_H(prob, st[3:], st[:3], E_half))
    dt = time.perf_counter() - t0
    Nc = (n + P) ** 3
    return {"value": 6 * Nc * 0.5 / dt, "unit": UNIT, "cores": len(os.sched_getaffinity(0)), "kind": "oracle",
            "sample": "E and H sub-solves of half step 1 (half a time step) at %d^3, p=2, FP64 numpy "
                      "(BLAS threads = all cores); %.1f s" % (n, dt)}


def job_rate(local_s, units, world, device=None):
    """Whole-job rate when this rank processed `units` in `local_s` seconds: the
    units of all ranks over the slowest rank's time (max over ranks).  Returns
    (rate, slowest time)."""
    import torch
    t = torch.tensor([float(local_s)], dtype=torch.float64, device=device)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(u, op=dist.ReduceOp.SUM)
    s = float(t.item())
    return float(u.item()) / s, s


def l2_note(n, esize=4):
    """How the L2 is handled: the working set of the step (six field and four
    row-coefficient arrays) against the 129 MB L2."""
    ws = 10 * (n + P) ** 3 * esize
    if ws > 129e6:
        return "working set %.2f GB > 129 MB L2 (no flush needed)" % (ws / 1e9)
    return "working set %.0f MB fits in the 129 MB L2 (not flushed: small-case timing only)" % (ws / 1e6)


def config_of(n, tau, world):
    """The workload description shared by both arms (tau printed to 12 digits:
    each arm computes the explicit limit in its own code)."""
    return {"workload": "ADI IGA Maxwell step, %d^3 elements, p=%d, head-like 3-phase map seed %d, "
                        "dipole, tau=4 dt_CFL" % (n, P, SEED), "n": n, "p": P, "tau": float("%.12g" % tau),
            "l2": l2_note(n), "parallelism": "replicas" if world > 1 else "single GPU"}


def run_reference(args, rank, world):
    """The FP64 oracle on the host cores.  Each bench step is a bounded sample of
    the workload: half a time step (the E and H sub-solves of half step 1, each
    right-hand side and its nine line solves) at the full size, counted as 0.5
    time step."""
    if rank != 0:
        return
    n = args.n
    eps, mu, sigma, src = workload(n)
    from oracle import material
    from oracle import maxwell_adi as ma
    from paper_2103_06998_gb300 import inputs
    eh = material.row_hats(eps, (n, n, n), P)
    tau = 4.0 * material.cfl_dt((n, n, n), P, eh, material.row_hats(mu, (n, n, n), P))
    prob = ma.make_problem((n, n, n), P, tau, eps, mu, sigma)
    ma.set_source(prob, src["x0"], src["comp"], src["amp"], src["f0"], src["t0"], src["s"])
    st = ma.apply_dirichlet(list(inputs.random_fields(prob.shape, 3)))
    Nc = (n + P) ** 3

    def one():  # half a time step: E half 1 (RHS + 9 line solves) and H half 1 (RHS + 9 line solves)
        E_half = ma.solve_E(prob, 1, ma.rhs_E(prob, 1, st[:3], st[3:], 1.5 + 0.25 * tau))
        ma.solve_H(prob, ma.rhs_H(prob, st[3:], st[:3], E_half))

    for _ in range(args.warmup):
        one()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        one()
    dt = time.perf_counter() - t0
    value = 6 * Nc * 0.5 * args.steps / dt
    cores = len(os.sched_getaffinity(0))
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * dt / (0.5 * args.steps), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference", "config": config_of(n, tau, world),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "each step: the E and H sub-solves of half step 1 (two right-hand sides and "
                                       "18 line solves, counted as half a time step) at full size, FP64 numpy"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def batched_result(precision, steps, warmup, rank=0, local=0):
    """48 independent instances of uneven size (seeded), each with its own head
    map and dipole, tau = 4 dt_CFL per instance, stepped together by one CUDA
    graph per step; line tiles chosen by the library's autotuner.  Returns the
    measurement, and for instance 0 its one-step error against the FP64 GPU step
    from the same state."""
    import torch
    from paper_2103_06998_gb300 import adi, inputs
    torch.cuda.set_device(local)
    insts = inputs.batch_instances(48, SEED + 1000 * rank)
    for d in insts:
        d["dt"] = 1.0
    b = adi.Batch(insts, precision=precision)
    for s, d in zip(b.solvers, insts):
        s.set_dt(4.0 * s.cfl_dt())
    b.factor()
    for s, d in zip(b.solvers, insts):
        src = d["source"]
        s.set_source(src["x0"], src["comp"], src["amp"], src["f0"], src["t0"], src["s"])
        n, p = d["n"], d["p"]
        s.set_fields(np.zeros((6, n[2] + p, n[1] + p, n[0] + p)), 1.0)
    b.autotune(os.path.join(tempfile.gettempdir(), "adi_line_tiles.txt"))
    stream = torch.cuda.Stream()  # a real stream: the legacy default stream cannot be captured
    torch.cuda.set_stream(stream)
    b.set_stream(stream.cuda_stream)
    for _ in range(warmup):
        b.step(1)
    b.sync()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        ev0.record(stream)
        b.step(steps)
        ev1.record(stream)
        b.sync()
        torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    dof = sum(6 * (d["n"][0] + d["p"]) * (d["n"][1] + d["p"]) * (d["n"][2] + d["p"]) for d in insts)
    # instance 0 (untimed): one step from a random state against the FP64 GPU step
    d0, s0 = insts[0], b.solvers[0]
    n0, p0 = d0["n"], d0["p"]
    st = inputs.random_fields((n0[2] + p0, n0[1] + p0, n0[0] + p0), 7) * 1e-3
    r64 = adi.Solver(n0, p0, s0.dt, d0["eps"], d0["mu"], d0["sigma"], precision="fp64")
    r64.factor()
    src = d0["source"]
    for sv in (s0, r64):
        sv.set_source(src["x0"], src["comp"], src["amp"], src["f0"], src["t0"], src["s"])
        sv.set_fields(st, 1.5)
        sv.step(1)
    b.sync()
    e_a, _ = s0.fields()
    e_b, _ = r64.fields()
    r64.close()
    b.close()
    torch.cuda.set_stream(torch.cuda.default_stream())
    return {"value": dof * steps / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms / steps, "steps": steps,
            "warmup": warmup, "total_dof": dof, "instances": [[d["n"][0], d["n"][1], d["n"][2], d["p"]] for d in insts],
            "error_vs_fp64_per_step": float(np.sqrt(np.sum((e_a - e_b) ** 2) / np.sum(e_b ** 2))),
            "error_instance": [n0[0], n0[1], n0[2], p0],
            "workload": "48 instances, elements per axis U{32..128}, p in {2,3}, head-like maps seeds 2103+i, "
                        "dipoles, tau = 4 dt_CFL each, one CUDA graph of all instances per step",
            "clocks": clk.summary()}


def run_batched(args, rank, world, local):
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    r = batched_result(args.precision, args.steps, args.warmup, rank, local)
    # each rank steps its own 48 instances: all ranks' DOF-steps over the slowest rank's time
    value, _ = job_rate(r["ms_per_step"] * args.steps * 1e-3, r["total_dof"] * args.steps, world, "cuda")
    if world > 1:
        dist.destroy_process_group()
    if rank == 0:
        line = {"metric": "field DOF-steps/s, 48 heterogeneous instances", "value": value,
                "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": r["ms_per_step"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32" if args.precision == "fp32" else "f64", "data": "synthetic",
                "error_vs_fp64_per_step": r["error_vs_fp64_per_step"],
                "config": {"workload": r["workload"], "total_dof": r["total_dof"], "instances": r["instances"]},
                "clocks": r["clocks"]}
        print(json.dumps(line), flush=True)


def learned_result(n, m, warmup, steps, tol, weights=None, verify=None, local=0):
    """Learned coarse-step corrector (weights trained by paper_2103_06998_gb300.corrector
    at 64^3) on an n^3-element head map: the guarded loop (k = 8, guard on the
    first step of every window of 8 coarse steps, tolerance ``tol`` relative l2)
    against plain steps of tau, in simulated time per second; an untimed
    verification compares the first ``verify`` corrected and plain coarse steps
    with 8 plain steps from the same state."""
    import torch
    from paper_2103_06998_gb300 import adi, corrector
    torch.cuda.set_device(local)
    k, every = 8, 8
    verify = m if verify is None else min(verify, m)
    N = (n + P,) * 3
    Nc = N[0] * N[1] * N[2]
    fine, coarse, tau = corrector.solver_pair((n, n, n), P, k, SEED)
    start, extra1, _ = corrector.solver_pair((n, n, n), P, k, SEED, tau=tau)
    probe, extra2, _ = corrector.solver_pair((n, n, n), P, k, SEED, tau=k * tau)
    extra1.close()
    extra2.close()
    stream = torch.cuda.Stream()  # one stream for all: graphs replay, no cross-stream waits
    torch.cuda.set_stream(stream)
    for sv in (fine, coarse, start, probe):
        sv.set_stream(stream.cuda_stream)
    net = adi.Net(N)
    net.set_stream(stream.cuda_stream)
    net.set_params(corrector.load(weights or corrector.WEIGHTS))
    warm = int(round(1.0 / tau))
    start.set_fields(np.zeros((6,) + N), 0.0)
    start.step(warm)                               # t ~ 1: the pulse has left the dipole
    # ---- plain steps of tau
    adi.copy_state(fine, start)
    fine.step(max(3, warmup))
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    nplain = 8 * max(8, steps)
    with ClockSampler(local) as clk:
        ev0.record(stream)
        fine.step(nplain)
        ev1.record(stream)
        torch.cuda.synchronize()
        ms_plain = ev0.elapsed_time(ev1) / nplain
        # ---- the net alone (features + forward + apply of one coarse step)
        X = torch.zeros((Nc, 16), dtype=torch.bfloat16, device="cuda")
        Y = torch.zeros((Nc, 8), dtype=torch.float32, device="cuda")
        torch.cuda.synchronize()
        adi.copy_state(coarse, start)
        coarse.step(1)
        net.features(coarse, X.data_ptr())
        for _ in range(3):
            net.forward(X.data_ptr(), Y.data_ptr())
        torch.cuda.synchronize()
        R = 20
        ev0.record(stream)
        for _ in range(R):
            net.forward(X.data_ptr(), Y.data_ptr())
        ev1.record(stream)
        torch.cuda.synchronize()
        ms_net = ev0.elapsed_time(ev1) / R
        ev0.record(stream)
        coarse.step(R)
        ev1.record(stream)
        torch.cuda.synchronize()
        ms_coarse = ev0.elapsed_time(ev1) / R
        # ---- the guarded loop (host decisions at every guard: wall clock)
        adi.copy_state(coarse, start)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        nfall, gmax = adi.corrector_run(net, coarse, fine, m, k, every, tol)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
    # ---- verification (untimed): along the plain trajectory from the same start,
    # every coarse step (plain and corrected) against k plain steps from its state
    state, extra3, _ = corrector.solver_pair((n, n, n), P, k, SEED, tau=tau)
    extra3.close()
    state.set_stream(stream.cuda_stream)
    adi.copy_state(state, start)
    e_fix, e_plain = [], []
    for _ in range(verify):
        adi.copy_state(fine, state)
        fine.step(k)
        adi.copy_state(probe, state)
        probe.step(1)
        e_plain.append(adi.fields_distance(probe, fine))
        adi.copy_state(coarse, state)
        coarse.step(1)
        net.features(coarse, X.data_ptr())
        net.forward(X.data_ptr(), Y.data_ptr())
        net.apply(coarse, Y.data_ptr())
        e_fix.append(adi.fields_distance(coarse, fine))
        adi.copy_state(state, fine)
    state.close()
    for sv in (fine, coarse, start, probe):
        sv.close()
    net.close()
    torch.cuda.set_stream(torch.cuda.default_stream())
    flops_alg = 27 * 2 * sum(ci * co for ci, co in adi.NET_REAL) * Nc
    d = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    peak = float(d["bf16_tflops"])
    sim_plain = tau / (ms_plain * 1e-3)
    sim_learned = m * k * tau / wall
    return {"n": n, "tau": tau, "k": k, "guard_every": every, "tol": tol, "coarse_steps": m, "start_t": warm * tau,
            "plain": {"sim_per_s": sim_plain, "ms_per_step": ms_plain, "dof_steps_per_s": 6 * Nc / (ms_plain * 1e-3)},
            "learned": {"sim_per_s": sim_learned, "speedup_vs_plain": sim_learned / sim_plain,
                        "ms_per_coarse_step_guarded": wall * 1e3 / m,
                        "fallback_windows": nfall, "windows": (m + every - 1) // every, "guard_max_err": gmax,
                        "ms_coarse_step": ms_coarse, "ms_net_forward": ms_net},
            "verification": {"steps": verify, "corrected_err_median": float(np.median(e_fix)),
                             "corrected_err_max": float(np.max(e_fix)),
                             "plain_coarse_err_median": float(np.median(e_plain)),
                             "plain_coarse_err_max": float(np.max(e_plain)),
                             "gain_median": float(np.median(np.array(e_plain) / np.array(e_fix)))},
            "roofline": {"bound": "tensor", "kernel": "conv_kernel (4 launches of one forward)",
                         "achieved": flops_alg / (ms_net * 1e-3) / 1e12, "peak": peak, "unit": "TFLOP/s",
                         "frac": flops_alg / (ms_net * 1e-3) / 1e12 / peak, "traffic": None,
                         "peak_source": "measured (MEASURED_PEAKS.json bf16_tflops)"},
            "clocks": clk.summary()}


def run_learned(args, rank, world, local):
    n = args.n if args.n != N_ELEM else 128
    r = learned_result(n, args.coarse_steps, args.warmup, args.steps, args.tol, args.weights, local=local)
    if rank == 0:
        line = {"metric": "simulated time per second, learned corrector vs plain FP32 ADI, %d^3 p=2" % n,
                "value": r["learned"]["sim_per_s"], "unit": "simulated s / s", "n_gpus": world,
                "steps": args.coarse_steps, "warmup": args.warmup,
                "ms_per_step": r["learned"]["ms_per_coarse_step_guarded"], "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "bf16 net / f32 solver", "data": "synthetic",
                "config": {"workload": "%d^3 elements, p=2, head-like map seed %d, dipole, tau = 4 dt_CFL, k = %d, "
                                       "guard every %d coarse steps, tol %g, start t = %.3f"
                                       % (n, SEED, r["k"], r["guard_every"], r["tol"], r["start_t"]),
                           "tau": r["tau"], "coarse_steps": r["coarse_steps"]},
                "plain": r["plain"], "learned": r["learned"], "verification": r["verification"],
                "roofline": r["roofline"], "clocks": r["clocks"]}
        print(json.dumps(line), flush=True)


def quad_result(n, tau, eps, mu, sigma, src, st, steps, warmup, local=0):
    """The quad reading of the material (per-element coefficients inside the
    right-hand side integrals) on the same workload in FP32: time per step, and
    its one-step error against the FP64 GPU step of the same reading."""
    import torch
    from paper_2103_06998_gb300 import adi
    out = {}
    for prec in ("fp64", "fp32"):
        s = adi.Solver((n, n, n), P, tau, eps, mu, sigma, precision=prec, rhs_material="quad")
        s.factor()
        s.set_source(src["x0"], src["comp"], src["amp"], src["f0"], src["t0"], src["s"])
        stream = torch.cuda.Stream()
        torch.cuda.set_stream(stream)
        s.set_stream(stream.cuda_stream)
        s.set_fields(st, 1.5)
        s.step(1)
        out[prec] = s.fields()[0]
        if prec == "fp32":
            for _ in range(warmup):
                s.step(1)
            torch.cuda.synchronize()
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            with ClockSampler(local) as clk:
                ev0.record(stream)
                s.step(steps)
                ev1.record(stream)
                torch.cuda.synchronize()
            ms = ev0.elapsed_time(ev1) / steps
            s.set_profiling(True)
            s.step(1)
            stats = s.kernel_stats()
            s.set_profiling(False)
        s.close()
        torch.cuda.set_stream(torch.cuda.default_stream())
    a, b = out["fp32"], out["fp64"]
    Nc = (n + P) ** 3
    return {"value": 6 * Nc / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms, "steps": steps, "warmup": warmup,
            "error_vs_fp64_per_step": float(np.sqrt(np.sum((a - b) ** 2) / np.sum(b ** 2))), "dtype": "f32",
            "reading": "per-element eps, mu, sigma inside the right-hand side integrals (ADI_RHS_QUAD)",
            "kernels_ms_per_step": {k["name"]: k["total_ms"] for k in stats}, "clocks": clk.summary()}


def mixed_result(n, tau, eps, mu, sigma, src, st, ref64, steps, warmup, local=0):
    """The mixed-precision step on the same workload: time per step over ``steps``
    graph replays, and its one-step error against the FP64 GPU step ``ref64``
    taken from the state ``st``."""
    import torch
    from paper_2103_06998_gb300 import adi
    s = adi.Solver((n, n, n), P, tau, eps, mu, sigma, precision="mixed")
    s.factor()
    s.set_source(src["x0"], src["comp"], src["amp"], src["f0"], src["t0"], src["s"])
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    s.set_stream(stream.cuda_stream)
    s.set_fields(st, 1.5)
    s.step(1)
    got, _ = s.fields()
    err = float(np.sqrt(np.sum((got - ref64) ** 2) / np.sum(ref64 ** 2)))
    for _ in range(warmup):
        s.step(1)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        ev0.record(stream)
        s.step(steps)
        ev1.record(stream)
        torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / steps
    # per-kernel device times of one step (events around every launch, graph off)
    s.set_profiling(True)
    s.step(1)
    stats = s.kernel_stats()
    s.set_profiling(False)
    s.close()
    torch.cuda.set_stream(torch.cuda.default_stream())
    Nc = (n + P) ** 3
    return {"value": 6 * Nc / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms, "steps": steps, "warmup": warmup,
            "error_vs_fp64_per_step": err, "dtype": "bf16 tiles / f32 solves / f64 residual",
            "sim_per_s": tau / (ms * 1e-3),
            "kernels_ms_per_step": {k["name"]: k["total_ms"] for k in stats}, "clocks": clk.summary()}


def main():
    global P
    args = parse()
    P = args.p
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.mode == "batched":
        return run_batched(args, rank, world, local)
    if args.mode == "learned":
        return run_learned(args, rank, world, local)

    import torch
    import torch.distributed as dist
    from paper_2103_06998_gb300 import adi, inputs

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    n = args.n
    eps, mu, sigma, src = workload(n)
    # tau = 4 x explicit limit (the library computes the limit for these data)
    s = adi.Solver((n, n, n), P, 1.0, eps, mu, sigma, precision=args.precision, serial_chains=args.serial_chains)
    tau = 4.0 * s.cfl_dt()
    s.set_dt(tau)
    s.factor()
    s.set_source(src["x0"], src["comp"], src["amp"], src["f0"], src["t0"], src["s"])
    stream = torch.cuda.Stream()  # a real stream: the step is replayed as a CUDA graph on it
    torch.cuda.set_stream(stream)
    s.set_stream(stream.cuda_stream)
    Nc = (n + P) ** 3
    state = inputs.random_fields((n + P,) * 3, 3) * 1e-3   # seeded random state (plus the dipole)
    s.set_fields(state, 1.0)
    dof_steps = 6 * Nc

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    # ---- warm-up, then the timed region (device events on the launch stream)
    for _ in range(args.warmup):
        s.step(1)
    barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            s.step(1)
        ev1.record(stream)
        barrier()
    value, s_max = job_rate(ev0.elapsed_time(ev1) * 1e-3, dof_steps * args.steps, world, "cuda")
    ms_max = s_max * 1e3

    # ---- per-kernel device times over the same number of steps (events around
    # every launch on the same stream, graph off), for the roofline
    s.set_profiling(True)
    for _ in range(args.steps):
        s.step(1)
    stats = s.kernel_stats()
    s.set_profiling(False)
    tot = sum(k["total_ms"] for k in stats)
    dom = max(stats, key=lambda k: k["total_ms"])
    launches_per_step = sum(k["launches"] for k in stats) / args.steps
    avg_ms = dom["total_ms"] / dom["launches"]
    hbm, peak_kind = peaks()
    achieved = dom["bytes_per_launch"] / (avg_ms * 1e-3) / 1e9
    traffic = ncu_traffic(dom["name"], n)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                "traffic": traffic, "kernel": dom["name"], "peak_source": peak_kind + " (MEASURED_PEAKS.json hbm_gbs)"
                if peak_kind == "measured" else "fallback 6.8 TB/s"}
    fp64_terms = 18 if dom["name"] == "resid_E64" else (12 if args.precision == "fp64" and dom["name"] == "rhs_E"
                                                         else 0)
    if fp64_terms:
        # FP64-ALU bound (GB300's FP64 rate is 1/64 of FP32): Kronecker terms x 3 passes x (2p+1) FMAs per
        # point (18 terms in the mixed-mode residual, the 12 of the E right-hand side in the FP64 step)
        flops = fp64_terms * 3 * (2 * P + 1) * 2 * Nc
        roofline.update({"bound": "alu", "achieved": flops / (avg_ms * 1e-3) / 1e12, "peak": FP64_PEAK_TFLOPS,
                         "unit": "TFLOP/s", "frac": flops / (avg_ms * 1e-3) / 1e12 / FP64_PEAK_TFLOPS,
                         "peak_source": "nominal FP64 of GB300 (no measured FP64 peak)"})
    roofline.update({
                "step_frac": (50 * Nc * (8 if args.precision == "fp64" else 4)) / (ms_max * 1e-3 / args.steps) / 1e9 / hbm,
                "kernels": {k["name"]: {"launches_per_step": k["launches"] / args.steps,
                                        "ms_per_launch": k["total_ms"] / k["launches"],
                                        "share": k["total_ms"] / tot,
                                        "GBps": k["bytes_per_launch"] / (k["total_ms"] / k["launches"] * 1e-3) / 1e9}
                            for k in stats}})

    # ---- end to end through the C-ABI with pinned host buffers: each step sets the
    # fields from host memory, steps, and reads the fields back.  The state's own
    # precision on the host side (floats for the FP32 and mixed handles, whose state
    # is FP32: the same values as through doubles), and the double form as a second
    # figure.
    def e2e_run(host_t, set_fn, get_fn):
        host_in = torch.empty(6 * Nc, dtype=host_t, pin_memory=True)
        host_out = torch.empty(6 * Nc, dtype=host_t, pin_memory=True)
        host_in.numpy()[:] = inputs.random_fields((n + P,) * 3, 5).ravel() * 1e-3
        for _ in range(max(1, min(args.warmup, 2))):  # untimed warm-up of the same sequence
            set_fn(host_in.data_ptr(), 1.0)
            s.step(1)
            get_fn(host_out.data_ptr())
        s.sync()
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            set_fn(host_in.data_ptr(), 1.0)
            s.step(1)
            get_fn(host_out.data_ptr())
        s.sync()  # the asynchronous form's transfers complete here
        barrier()
        rate, _ = job_rate((time.perf_counter() - t0) / args.e2e_steps, dof_steps, world, "cuda")
        nb = 6 * Nc * host_in.element_size()
        return {"value": rate, "unit": UNIT, "h2d_bytes_per_step": nb, "d2h_bytes_per_step": nb}

    # the asynchronous calls copy each set during the step before it and each read during the step after it
    eb = 8 if args.precision == "fp64" else 4
    ht = torch.float64 if eb == 8 else torch.float32
    e2e = e2e_run(ht, lambda ptr, t: s.set_fields_async_ptr(ptr, eb, t), lambda ptr: s.fields_async_ptr(ptr, eb))
    e2e["calls"] = "adi_set_fields_async / adi_step / adi_fields_async, host %s" % ("f64" if eb == 8 else "f32")
    e2e["sync_f64_host"] = e2e_run(torch.float64, s.set_fields_ptr, s.fields_ptr)
    if eb == 4:
        e2e["sync_f32_host"] = e2e_run(torch.float32, s.set_fields_f32_ptr, s.fields_f32_ptr)

    # ---- per-step error against the FP64 GPU step from the same state (untimed)
    err64 = None
    st = ref64 = None
    if args.precision != "fp64" and rank == 0:
        st = inputs.random_fields((n + P,) * 3, 7) * 1e-3
        s64 = adi.Solver((n, n, n), P, tau, eps, mu, sigma, precision="fp64")
        s64.factor()
        for sv in (s, s64):
            sv.set_source(src["x0"], src["comp"], src["amp"], src["f0"], src["t0"], src["s"])
            sv.set_fields(st, 1.5)
            sv.step(1)
        a, _ = s.fields()
        ref64, _ = s64.fields()
        s64.close()
        err64 = float(np.sqrt(np.sum((a - ref64) ** 2) / np.sum(ref64 ** 2)))

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(n, eps, mu, sigma, src, tau)
    s.close()
    torch.cuda.set_stream(torch.cuda.default_stream())
    clocks = clk.summary()
    extras = {}
    if rank == 0 and world == 1 and not args.no_extras and args.precision == "fp32":
        # the other forms of the method, each measured here on its own workload (untimed by the driver's
        # clock of the FP32 step above): mixed precision and the quad reading of the material on the same
        # 256^3 map, the 48-instance batch, and the guarded learned corrector at 128^3
        try:
            extras["mixed"] = mixed_result(n, tau, eps, mu, sigma, src, st, ref64, 5, 2, local)
            extras["mixed"]["vs_fp32_sim_time"] = extras["mixed"]["sim_per_s"] / (tau / (ms_max * 1e-3 / args.steps))
        except Exception as ex:  # reported, never silently dropped
            extras["mixed"] = {"error": repr(ex)}
        try:
            extras["quad"] = quad_result(n, tau, eps, mu, sigma, src, st, 5, 2, local)
        except Exception as ex:
            extras["quad"] = {"error": repr(ex)}
        try:
            extras["batched"] = batched_result("fp32", 10, 3, rank, local)
        except Exception as ex:
            extras["batched"] = {"error": repr(ex)}
        try:
            extras["learned"] = learned_result(128, 64, 3, 8, 1e-4, verify=16, local=local)
        except Exception as ex:
            extras["learned"] = {"error": repr(ex)}
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": {"fp32": "f32", "fp64": "f64", "mixed": "bf16 tiles / f32 / f64 residual"}[args.precision],
                "data": "synthetic", "error_vs_fp64_per_step": err64,
                "config": config_of(n, tau, world),
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": int(round(launches_per_step * args.steps)),
                "clocks": clocks}
        line.update(extras)
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
