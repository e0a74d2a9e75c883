#!/usr/bin/env python
"""Forward + adjoint MLUPS of the discrete adjoint LBM on one GB300 per rank.

One step = for each Re of the workload: forward solve to the residual
tolerance, adjoint solve to the residual tolerance and dJ/dgamma, from rest,
with inputs already resident in HBM.  value = cell updates (forward + adjoint
steps x nodes, summed over ranks) / max-over-ranks time.  L2 is flushed
between timed steps by writing a buffer larger than L2.

--impl reference times the FP64 CPU oracle on bounded samples of the same
workload on the host cores (there is no reference code to run).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fwd+adjoint MLUPS (% HBM roofline); served sens/s & p50/p99 vs plain FP32"
RES = (50.0, 100.0, 500.0)
TOL = 1e-6
CAP = 200000
CHECK = 1000
FWD_BYTES = {"fp32": 19 * 4 * 2 + 4 + 1, "fp64": 19 * 8 * 2 + 8 + 1,
             "fp16": 19 * 2 * 2 + 4 + 1, "bf16": 19 * 2 * 2 + 4 + 1}
ADJ_BYTES = {"fp32": 19 * 4 * 2 + 12 + 4 + 1, "fp64": 19 * 8 * 2 + 24 + 8 + 1,
             "fp16": 19 * 4 * 2 + 12 + 4 + 1, "bf16": 19 * 4 * 2 + 12 + 4 + 1}
THERM_BYTES = 7 * 4 * 2 + 12 + 4 + 1   # D3Q7 FP32 populations + frozen u + gamma + flag
# DRAM bytes per node per launch (dram__bytes_read.sum + dram__bytes_write.sum
# / nodes) from one ncu capture of the current kernels on a 160^3 pipe bend
# (FP32 forward and adjoint, FP16 paired forward); traffic grows with the node
# count, so a launch on N nodes moves N times this.
TRAFFIC_B_PER_NODE = {("adjoint", "fp32"): 156.9, ("forward", "fp32"): 145.5, ("forward", "fp16"): 70.9}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--n", type=int, default=64, help="pipe-bend lattice edge")
    p.add_argument("--storage", default="fp32", choices=["fp32", "fp64", "fp16", "bf16"])
    p.add_argument("--roof-n", type=int, default=320, help="edge of the >L2 roofline lattice")
    p.add_argument("--roof-launches", type=int, default=20)
    p.add_argument("--lattice", default="pipe", choices=["pipe", "heatsink"],
                   help="kernels mode: pipe bend (flow kernels) or heat sink (all four)")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--cap", type=int, default=CAP,
                   help="step cap per solve phase (lower it only for profiler launch lists)")
    p.add_argument("--mode", default="full", choices=["full", "kernels", "precision", "autograd", "serve", "batchcmp",
                                                 "levelset", "stability"],
                   help="kernels: time the fused step kernels on a --roof-n lattice; "
                        "precision: heat sink in FP32/FP16/BF16 storage, error per field against FP64 "
                        "at the same per-phase step counts; "
                        "autograd: the filtered / projected gradient loop; serve: the served "
                        "streams; batchcmp: batched vs single-context throughput; levelset: the "
                        "level-set optimiser on the 2D pipe bend; stability: largest stable inlet "
                        "speed per relaxation time for the forward, discrete and continuous adjoint")
    p.add_argument("--iters", type=int, default=50, help="autograd / levelset modes: optimisation iterations")
    p.add_argument("--nreq", type=int, default=256, help="served requests of the as-specified stream")
    p.add_argument("--cases", default="", help="batchcmp: run only the cases whose name contains this")
    p.add_argument("--fp16-tol-factor", type=float, default=0.25,
                   help="serving: the 16-bit path's extra run uses this times the tolerance")
    p.add_argument("--nreq-stable", type=int, default=64,
                   help="served requests of the stable-Re stream (0: skip it)")
    p.add_argument("--no-serve", action="store_true")
    p.add_argument("--no-extra", action="store_true", help="skip the level-set and paper heat-sink legs")
    p.add_argument("--stab-steps", type=int, default=1000000, help="stability mode: iterations per run")
    p.add_argument("--stab-iters", type=int, default=6, help="stability mode: bisection steps")
    p.add_argument("--stab-umin", type=float, default=0.005)
    p.add_argument("--stab-umax", type=float, default=0.5)
    p.add_argument("--stab-taus", type=float, nargs="+", default=[0.52, 0.55, 0.6, 0.8])
    return p.parse_args()


def run_precision(args):
    """128x64x32 heat sink (D3Q19 + D3Q7, Re 50): each storage solves every
    phase (flow, temperature, temperature adjoint, flow adjoint) to 1e-6; an
    FP64 run then takes exactly the same number of steps of each phase, and
    the rel-L2 error of every field is taken against it (equal step counts
    separate rounding from the distance to the fixed point; the FP64 path
    matches the FP64 oracle to 1e-11 per step and at convergence in the tests)."""
    import numpy as np
    import torch

    from paper_2501_02161_gb300 import build as B
    from paper_2501_02161_gb300 import inputs as I
    from paper_2501_02161_gb300.solver import Solver

    B.build()
    torch.cuda.set_device(0)
    lat = I.heat_sink(re=50.0, seed=4)
    phases = ((0, "flow"), (1, "temperature"), (3, "temperature_adjoint"), (2, "flow_adjoint"))

    def solve(storage, steps=None):
        s = Solver.from_lattice(lat, storage=storage, device="cuda:0")
        got = {}
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for ph, name in phases:
            if steps is None:
                r = s.solve_phase(ph, tol=TOL, max_steps=400000, check_every=CHECK, strict=False)
            else:
                r = s.solve_phase(ph, tol=0, max_steps=steps[name], check_every=CHECK, strict=False)
            got[name] = r.steps
            if r.status < 0:
                s.close()
                return None, got, None
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        rho, u, T = s.fields(torch.float64)
        fs, gs = s.adjoint_fields(torch.float64)
        f = {"rho": rho, "u": u, "T": T, "f*": fs, "g*": gs,
             "dJ/dgamma": s.sensitivity(dtype=torch.float64), "J": torch.tensor([s.objective()])}
        s.close()
        return {k: v.cpu().numpy() for k, v in f.items()}, got, dt

    out = {"mode": "precision", "workload": "heat sink 128x64x32, Re 50, Pr 7, k_r 100; every phase "
                                            "to 1e-6, FP64 reference at the same per-phase step counts",
           "fields": {}}
    for storage in ("fp32", "fp16", "bf16"):
        f, steps, dt = solve(storage)
        rec = {"steps": steps}
        if f is None:
            rec["status"] = "diverged"
        else:
            ref, _, _ = solve("fp64", steps)
            rec["MLUPS"] = round(sum(steps.values()) * lat.n / dt / 1e6, 1)
            rec["rel_l2_vs_fp64_same_steps"] = {
                k: float(np.linalg.norm(f[k] - ref[k]) / np.linalg.norm(ref[k])) for k in f}
        out["fields"][storage] = rec
    print(json.dumps(out))


def run_autograd(args):
    """The autograd workload: 96x48x24 heat sink, density filter (radius 2) +
    Heaviside projection (beta 8), --iters projected-gradient steps, each a
    forward + adjoint through the C-ABI with warm starts."""
    import torch

    from paper_2501_02161_gb300 import build as B
    from paper_2501_02161_gb300 import inputs as I
    from paper_2501_02161_gb300.autograd import SolveOpts, projected_gradient_loop
    from paper_2501_02161_gb300.solver import Solver

    B.build()
    torch.cuda.set_device(0)
    lat = I.heat_sink(nx=96, ny=48, nz=24, re=50.0, seed=4)
    opts = SolveOpts(tol=1e-5, max_steps=200000, check_every=500, warm=True)
    # untimed: one iteration on a throw-away solver loads the libraries the
    # filter (conv3d) and the solver use and captures the step graphs' code
    w = Solver.from_lattice(lat, storage=args.storage, device="cuda:0")
    projected_gradient_loop(w, lat, iters=1, step=0.05, volume=0.6, opts=opts)
    w.close()
    s = Solver.from_lattice(lat, storage=args.storage, device="cuda:0")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rho, hist = projected_gradient_loop(s, lat, iters=args.iters, step=0.05, volume=0.6, opts=opts)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    print(json.dumps({"mode": "autograd", "workload": "heat sink 96x48x24 Re 50, filter r=2, "
                      "projection beta=8, volume fraction 0.6 penalty, tol 1e-5 warm-started",
                      "iters": args.iters, "seconds": round(dt, 2),
                      "s_per_iter": round(dt / args.iters, 3),
                      "J": [round(h["J"], 6) for h in hist],
                      "loss": [round(h["loss"], 6) for h in hist]}))


def run_levelset(args):
    """The paper's optimiser on the 64 x 64 D2Q9 pipe bend (FP64, tau 0.6):
    --iters level-set iterations (Eq. 14-15, lambda of Eq. 67, sigma 5e-3,
    fluid fraction bound 0.08 pi as in the paper's 2D case), each a forward +
    adjoint solve through the C-ABI, warm-started."""
    import math

    import torch

    from paper_2501_02161_gb300 import build as B
    from paper_2501_02161_gb300 import inputs as I
    from paper_2501_02161_gb300.levelset import level_set_loop
    from paper_2501_02161_gb300.solver import Solver

    B.build()
    torch.cuda.set_device(0)
    lat = I.workload("pipe_bend_2d_64x64")
    s = Solver.from_lattice(lat, storage="fp64", device="cuda:0")
    t0 = time.perf_counter()
    phi, hist = level_set_loop(s, lat, iters=args.iters, K=0.1, sigma=5e-3, vmax=0.08 * math.pi,
                               tol=1e-6, max_steps=200000, check_every=1000)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    s.close()
    print(json.dumps({"mode": "levelset", "workload": "2D D2Q9 pipe bend 64x64, FP64, level set "
                      "(K 0.1, sigma 5e-3, V_max 0.08 pi), forward + adjoint to 1e-6 warm-started",
                      "iters": args.iters, "seconds": round(dt, 2),
                      "s_per_iter": round(dt / max(args.iters, 1), 3),
                      "J": [round(h["J"], 6) for h in hist],
                      "fluid_fraction": [round(h["fluid_fraction"], 4) for h in hist],
                      "lambda": [round(h["lambda"], 6) for h in hist]}))


def run_serve(args, nreq=None, device="cuda:0"):
    """Config-5 serving: seeded sensitivity / optimisation-step requests over
    32^3 ... 192x96x48 lattices, half thermal, 20 % optimisation steps,
    forward + adjoint to 1e-4 (20000-step cap per phase).
    "as_specified": Re ~ U[10, 500], --nreq requests (256 by default), offline
    (all at t=0) and online (Poisson arrivals at 0.8 x the batched FP32 offline
    rate), each through (a) the sequential plain-FP32 path, (b) the batched
    FP32 server, (c) the batched server with FP16 flow storage; with BGK at
    these inlet widths most requests above Re ~ 80 diverge and count as
    failed (by_shape / by_re break the failures down).
    "stable_re": Re ~ U[10, 80] (the paper's 3D range), --nreq-stable
    requests, offline, the same three paths.
    "accuracy": for up to 8 completed sensitivity requests of the stable
    stream, dJ/dgamma of the sequential FP32 and batched FP16 results against
    a reference solve of the same request (FP64 storage, tolerance 1e-8).
    Latency = completion - arrival; sens/s = completed requests / wall time."""
    import numpy as np
    import torch

    from paper_2501_02161_gb300 import build as B
    from paper_2501_02161_gb300.serve import (Server, lattice_for, make_requests, serve_sequential,
                                              summarize)
    from paper_2501_02161_gb300.solver import Solver

    B.build()
    n = nreq or args.nreq
    tol, cap, K = 1e-4, 20000, 500

    def rel(a, b):
        return float(torch.linalg.norm(a.double() - b.double()) /
                     torch.linalg.norm(b.double()).clamp_min(1e-30))

    def agree(res, ref):
        errs = [rel(a.sens, b.sens) for a, b in zip(res, ref)
                if a.status >= 0 and b.status >= 0 and a.sens is not None and b.sens is not None]
        return {"median": float(np.median(errs)) if errs else None,
                "max": float(np.max(errs)) if errs else None, "n": len(errs)}

    def warm():
        # one-time costs (module loading, first allocations, graph captures of
        # the batch) are paid here, outside every timed run
        w = make_requests(4, seed=11, rate=None, re_range=(10.0, 40.0),
                          shapes=[(32, 32, 32), (64, 64, 64)])
        serve_sequential(w, "fp32", tol=tol, max_steps=cap, check_every=K, realtime=False,
                         device=device)
        for storage in ("fp32", "fp16"):
            srv = Server(storage, check_every=K, max_slots=32, tol=tol, max_steps=cap, device=device)
            srv.run(w, realtime=False)
            srv.close()

    def run_all(reqs, realtime):
        res = {}
        res["sequential_fp32"] = serve_sequential(reqs, "fp32", tol=tol, max_steps=cap,
                                                  check_every=K, realtime=realtime, device=device)
        for storage in ("fp32", "fp16"):
            srv = Server(storage, check_every=K, max_slots=32, tol=tol, max_steps=cap, device=device)
            res[f"batched_{storage}"] = srv.run(reqs, realtime=realtime)
            srv.close()
        summ = {k: summarize(v, requests=reqs) for k, v in res.items()}
        for k in ("batched_fp32", "batched_fp16"):
            summ[k]["dJdgamma_rel_l2_vs_sequential_fp32"] = agree(res[k], res["sequential_fp32"])
        return summ, res

    def accuracy(reqs, res, count=8):
        """dJ/dgamma of each result set against a reference solve of the same
        request (FP64 storage, tolerance 1e-8), over the first `count`
        sensitivity requests every set completed"""
        keys = list(res)
        refs = []
        for k, q in enumerate(reqs):
            if len(refs) >= count:
                break
            if q.kind != "sens" or any(res[key][k].status != 0 for key in keys):
                continue
            s = Solver.from_lattice(lattice_for(q), storage="fp64", device=device)
            rf = s.forward(tol=1e-8, max_steps=400000, check_every=K, strict=False)
            ra = s.adjoint(tol=1e-8, max_steps=400000, check_every=K, strict=False) if rf.status >= 0 else rf
            if ra.status >= 0:
                refs.append((k, q, s.sensitivity(dtype=torch.float64)))
            s.close()
        out = {"reference": "same request, FP64 storage, forward + adjoint to 1e-8", "n": len(refs),
               "requests": [{"shape": list(q.shape), "re": round(q.re, 1), "thermal": q.thermal}
                            for _, q, _ in refs]}
        for key in keys:
            errs = [rel(res[key][k].sens.to(ref.device), ref) for k, _, ref in refs]
            out[key] = {"median": float(np.median(errs)) if errs else None,
                        "max": float(np.max(errs)) if errs else None,
                        "per_request": [round(e, 7) for e in errs]}
        return out

    out = {"requests_per_stream": n, "tol": tol, "max_steps_per_phase": cap, "check_every": K,
           "shapes": "32^3, 64^3, 96x48x24, 128x64x32, 192x96x48", "thermal_fraction": 0.5,
           "opt_step_fraction": 0.2}
    warm()
    spec = {}
    spec["offline"], _ = run_all(make_requests(n, seed=5, rate=None), False)
    off = spec["offline"]["batched_fp32"]
    rate = 0.8 * n / max(off["wall_s"], 1e-9)
    spec["online_rate_per_s"] = round(rate, 3)
    spec["online"], _ = run_all(make_requests(n, seed=5, rate=rate), True)
    out["as_specified_re_10_500"] = spec
    ns = args.nreq_stable
    if ns > 0:
        reqs = make_requests(ns, seed=5, rate=None, re_range=(10.0, 80.0))
        summ, res = run_all(reqs, False)
        # the 16-bit path at a tighter stopping rule, for a comparison at
        # matched dJ/dgamma accuracy
        tight = tol * args.fp16_tol_factor
        srv = Server("fp16", check_every=K, max_slots=32, tol=tight, max_steps=cap, device=device)
        res["batched_fp16_tight"] = srv.run(reqs, realtime=False)
        srv.close()
        summ["batched_fp16_tight"] = summarize(res["batched_fp16_tight"], requests=reqs)
        summ["batched_fp16_tight"]["tol"] = tight
        out["stable_re_10_80"] = {"requests": ns, "offline": summ, "accuracy": accuracy(reqs, res)}
    return out


def run_stability(args):
    """The stability test of Sec. 3.1 (Fig. 6) on the CUDA path: the 2D pipe
    bend's initial geometry (empty chamber, gamma = 1 on the design nodes),
    for each relaxation time the largest inlet speed u_max at which the run
    does not diverge within --stab-steps iterations (the paper: 1e6), for the
    forward LBM, the forward + discrete adjoint and the forward + continuous
    adjoint.  Bisection on log(u_max) in [--stab-umin, --stab-umax]."""
    import math

    import torch

    from paper_2501_02161_gb300 import build as B
    from paper_2501_02161_gb300 import inputs as I
    from paper_2501_02161_gb300.solver import Solver

    B.build()
    torch.cuda.set_device(0)
    N = args.stab_steps
    K = 1000

    def stable(tau, umax, scheme):
        lat = I.pipe_bend_2d(tau=tau, umax=umax, gamma_value=1.0)
        s = Solver.from_lattice(lat, storage="fp64", device="cuda:0")
        try:
            r = s.forward(tol=0, max_steps=N, check_every=K, strict=False)
            if r.status < 0:
                return False
            if scheme is None:
                return True
            s.set_adjoint_scheme(scheme)
            r = s.adjoint(tol=0, max_steps=N, check_every=K, strict=False)
            return r.status >= 0
        finally:
            s.close()

    def limit(tau, scheme, hi_bound=None):
        lo, hi = math.log(args.stab_umin), math.log(hi_bound or args.stab_umax)
        if not stable(tau, math.exp(lo), scheme):
            return 0.0
        if stable(tau, math.exp(hi), scheme):
            return math.exp(hi)
        for _ in range(args.stab_iters):
            mid = 0.5 * (lo + hi)
            if stable(tau, math.exp(mid), scheme):
                lo = mid
            else:
                hi = mid
        return math.exp(lo)

    out = {"mode": "stability", "workload": "2D D2Q9 pipe bend 64x64, gamma = 1 on design nodes, FP64",
           "iterations": N, "bisection_steps": args.stab_iters, "u_max_range": [args.stab_umin, args.stab_umax],
           "rows": []}
    t0 = time.perf_counter()
    for tau in args.stab_taus:
        fwd = limit(tau, None)
        row = {"tau": tau, "forward": round(fwd, 5),
               "discrete_adjoint": round(limit(tau, "discrete", fwd), 5) if fwd > 0 else 0.0,
               "continuous_adjoint": round(limit(tau, "continuous", fwd), 5) if fwd > 0 else 0.0}
        out["rows"].append(row)
        print(json.dumps(row), flush=True)
    out["seconds"] = round(time.perf_counter() - t0, 1)
    print(json.dumps(out))


def run_batchcmp(args):
    """Throughput of the batched kernels against the single-context path on
    the same lattices and step counts (forward + adjoint, fixed steps)."""
    import torch

    from paper_2501_02161_gb300 import build as B
    from paper_2501_02161_gb300 import inputs as I
    from paper_2501_02161_gb300.serve import Batch
    from paper_2501_02161_gb300.solver import Solver

    B.build()
    torch.cuda.set_device(0)

    def single(lats, steps):
        ss = [Solver.from_lattice(l, device="cuda:0") for l in lats]
        for s in ss:
            s.forward(tol=0, max_steps=1000, check_every=500)
            s.adjoint(tol=0, max_steps=1000, check_every=500)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for s in ss:
            s.forward(tol=0, max_steps=steps, check_every=500)
            s.adjoint(tol=0, max_steps=steps, check_every=500)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        for s in ss:
            s.close()
        return dt

    def batched(lats, steps, solo_tiles=None):
        b = Batch("fp32", 500, 32, solo_tiles)
        ss = [Solver.from_lattice(l, device="cuda:0") for l in lats]
        for s in ss:
            b.admit(s, 0.0, 1000, True)
        while b.step():
            pass
        b.poll()
        for s in ss:
            b.admit(s, 0.0, steps, True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        while b.step():
            pass
        dt = time.perf_counter() - t0
        b.poll()
        b.close()
        for s in ss:
            s.close()
        return dt

    cases = [("1 x 192x96x48", [I.pipe_bend_3d(n=192, ny=96, nz=48, width=12, re=20.0)], 4000),
             ("1 x 64^3", [I.pipe_bend_3d(n=64, re=20.0)], 10000),
             ("4 x 64^3", [I.pipe_bend_3d(n=64, re=20.0, seed=k) for k in range(4)], 4000),
             ("16 x 32^3", [I.pipe_bend_3d(n=32, re=20.0, seed=k) for k in range(16)], 4000),
             ("32 x 32^3", [I.pipe_bend_3d(n=32, re=20.0, seed=k) for k in range(32)], 2000),
             ("32 x 16^3", [I.pipe_bend_3d(n=16, width=4, re=10.0, seed=k) for k in range(32)], 4000),
             ("mix 32^3+64^3+96x48x24+128x64x32+192x96x48",
              [I.pipe_bend_3d(n=32, re=20.0), I.pipe_bend_3d(n=64, re=20.0),
               I.pipe_bend_3d(n=96, ny=48, nz=24, width=12, re=20.0),
               I.pipe_bend_3d(n=128, ny=64, nz=32, width=16, re=20.0),
               I.pipe_bend_3d(n=192, ny=96, nz=48, width=12, re=20.0)], 4000)]
    out = {"mode": "batchcmp", "storage": "fp32", "steps": "forward N + adjoint N per lattice"}
    for name, lats, steps in cases:
        if args.cases and args.cases not in name:
            continue
        nodes = sum(l.n for l in lats)
        ts, tb, tp = single(lats, steps), batched(lats, steps), batched(lats, steps, 0)
        t1 = batched(lats, steps, 1)   # every lattice on its own graph and stream
        out[name] = {"single_MLUPS": round(2 * nodes * steps / ts / 1e6, 1),
                     "batched_MLUPS": round(2 * nodes * steps / tb / 1e6, 1),
                     "packed_only_MLUPS": round(2 * nodes * steps / tp / 1e6, 1),
                     "solo_only_MLUPS": round(2 * nodes * steps / t1 / 1e6, 1)}
    print(json.dumps(out))


def run_kernels(args):
    """Per-launch time and achieved GB/s of the fused forward and adjoint
    kernels on a pipe bend of edge --roof-n (CUDA events on their stream)."""
    import torch

    from paper_2501_02161_gb300 import build as B
    from paper_2501_02161_gb300 import inputs as I
    from paper_2501_02161_gb300.solver import Solver

    B.build()
    torch.cuda.set_device(0)
    hbm, kind = peaks()
    if args.lattice == "heatsink":
        n = args.roof_n
        big = I.heat_sink(nx=n, ny=n // 2, nz=n // 4, re=50.0, seed=4)
    else:
        big = I.pipe_bend_3d(n=args.roof_n, re=100.0, seed=1)
    sb = Solver.from_lattice(big, storage=args.storage, device="cuda:0")
    sb.forward(tol=0, max_steps=2, check_every=2, reset=True)
    sb.time_steps(0, 3)
    fwd_ms = sb.time_steps(0, args.roof_launches)
    rows = [("forward", fwd_ms, FWD_BYTES[args.storage])]
    if big.thermal:
        sb.time_steps(1, 3)
        rows.append(("thermal_forward", sb.time_steps(1, args.roof_launches), THERM_BYTES))
        sb.time_steps(3, 3)
        rows.append(("thermal_adjoint", sb.time_steps(3, args.roof_launches), THERM_BYTES))
    sb.time_steps(2, 3)
    adj_ms = sb.time_steps(2, args.roof_launches)
    rows.append(("adjoint", adj_ms, ADJ_BYTES[args.storage] + (12 if big.thermal else 0)))
    nb = big.n
    out = {"mode": "kernels", "lattice": [big.nx, big.ny, big.nz], "workload": big.name,
           "storage": args.storage, "nodes": nb, "peak_GB/s": hbm, "peak_kind": kind}
    for name, ms, bpn in rows:
        gbs = bpn * nb / (ms * 1e-3) / 1e9
        out[name] = {"ms_per_launch": ms, "bytes_per_node": bpn, "GB/s": round(gbs, 1),
                     "frac": round(gbs / hbm, 4), "MLUPS": round(nb / (ms * 1e-3) / 1e6, 1)}
    print(json.dumps(out))


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi samples every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [t.strip() for t in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def aggregate_ranks(total_ms: float, total_ups: float, device):
    """Whole-job figures over replicas: the slowest rank's time and the sum of
    the cell updates of all ranks (weak scaling, no data-path collective)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    u = torch.tensor([float(total_ups)], dtype=torch.float64, device=device)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2501_02161_gb300 import build as B
    from paper_2501_02161_gb300 import inputs as I
    from paper_2501_02161_gb300 import _capi as C
    from paper_2501_02161_gb300.solver import Solver

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if rank == 0:
        B.build()
    if world > 1:
        dist.barrier()
    C.lib()

    lats = {re: I.pipe_bend_3d(n=args.n, re=re, seed=1) for re in RES}
    N = lats[RES[0]].n
    solvers = {re: Solver.from_lattice(lat, storage=args.storage, device=dev)
               for re, lat in lats.items()}
    sens = torch.empty(N, dtype=torch.float32, device=dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def one_step():
        """(updates of solves that produced dJ/dgamma, updates spent on solves
        that diverged, kernel launches, per-Re record)"""
        ups, lost, launches, per = 0, 0, 0, {}
        for re, s in solvers.items():
            rf = s.forward(tol=TOL, max_steps=args.cap, check_every=CHECK, reset=True, strict=False)
            ra = (s.adjoint(tol=TOL, max_steps=args.cap, check_every=CHECK, reset=True, strict=False)
                  if rf.status >= 0 else rf.__class__(0, float("nan"), 0.0, 0.0, 0.0, rf.status))
            if ra.status >= 0:
                s.sensitivity(out=sens)
                ups += (rf.steps + ra.steps) * N
            else:
                lost += (rf.steps + ra.steps) * N
            launches += (rf.steps + math.ceil(rf.steps / CHECK) + 1 +
                         ra.steps + math.ceil(ra.steps / CHECK) + 1 + 1)
            per[re] = {"fwd_steps": rf.steps, "adj_steps": ra.steps, "J": rf.J,
                       "fwd_residual": rf.residual, "adj_residual": ra.residual,
                       "status": [C.STATUS_NAMES[rf.status], C.STATUS_NAMES[ra.status]]}
        return ups, lost, launches, per

    for _ in range(args.warmup):
        one_step()
        flush.fill_(1.0)
    torch.cuda.synchronize()
    clocks = Clocks(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    total_ms, total_ups, total_lost, total_launch, per = 0.0, 0, 0, 0, None
    for _ in range(args.steps):
        flush.fill_(float(_))
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        ups, lost, nl, per = one_step()
        e1.record()
        torch.cuda.synchronize()
        total_ms += e0.elapsed_time(e1)
        total_ups += ups
        total_lost += lost
        total_launch += nl
    clk = clocks.stop()
    if world > 1:
        dist.barrier()
        total_ms, total_ups = aggregate_ranks(total_ms, total_ups, dev)
    value = total_ups / (total_ms * 1e-3) / 1e6

    hbm, peak_kind = peaks()
    # kernel time shares inside the workload: per-launch duration at 64^3
    s0 = solvers[RES[1]]
    s0.forward(tol=0, max_steps=2, check_every=2, reset=True)
    fwd_ms_w = s0.time_steps(0, 200)
    adj_ms_w = s0.time_steps(2, 200)
    fsteps = sum(v["fwd_steps"] for v in per.values())
    asteps = sum(v["adj_steps"] for v in per.values())
    fwd_share = fsteps * fwd_ms_w / (fsteps * fwd_ms_w + asteps * adj_ms_w)
    at_workload = {
        "fwd": {"ms": fwd_ms_w, "GB/s": FWD_BYTES[args.storage] * N / (fwd_ms_w * 1e-3) / 1e9},
        "adj": {"ms": adj_ms_w, "GB/s": ADJ_BYTES[args.storage] * N / (adj_ms_w * 1e-3) / 1e9},
        "fwd_time_share": fwd_share,
        "note": f"{args.n}^3 populations fit in L2 (129 MB); rates above HBM are L2 rates"}

    roof = None
    if args.roof_n > 0:
        del solvers
        torch.cuda.empty_cache()
        big = I.pipe_bend_3d(n=args.roof_n, re=100.0, seed=1)
        sb = Solver.from_lattice(big, storage=args.storage, device=dev)
        sb.forward(tol=0, max_steps=2, check_every=2, reset=True)
        sb.time_steps(0, 3)
        fwd_ms = sb.time_steps(0, args.roof_launches)
        sb.time_steps(2, 3)
        adj_ms = sb.time_steps(2, args.roof_launches)
        nb = big.n
        kern = "adjoint" if fwd_share < 0.5 else "forward"
        ms = adj_ms if kern == "adjoint" else fwd_ms
        byts = (ADJ_BYTES if kern == "adjoint" else FWD_BYTES)[args.storage] * nb
        ach = byts / (ms * 1e-3) / 1e9
        tpn = TRAFFIC_B_PER_NODE.get((kern, args.storage))
        roof = {"bound": "hbm", "achieved": round(ach, 1), "peak": hbm, "unit": "GB/s",
                "frac": round(ach / hbm, 4),
                "traffic": round(tpn * nb) if tpn else None,
                "traffic_note": ("bytes per launch, ncu DRAM bytes per node at 160^3 x nodes"
                                 if tpn else None),
                "peak_kind": peak_kind,
                "kernel": f"k_flow_{'adjoint' if kern == 'adjoint' else 'step'} D3Q19 {args.storage}",
                "workload": f"pipe bend {args.roof_n}^3 ({nb} nodes, {byts/1e9:.2f} GB algorithmic per launch)",
                "bytes_per_node": (ADJ_BYTES if kern == "adjoint" else FWD_BYTES)[args.storage],
                "ms_per_launch": ms,
                "other": {"forward_GB/s": round(FWD_BYTES[args.storage] * nb / (fwd_ms * 1e-3) / 1e9, 1),
                          "adjoint_GB/s": round(ADJ_BYTES[args.storage] * nb / (adj_ms * 1e-3) / 1e9, 1),
                          "forward_MLUPS": round(nb / (fwd_ms * 1e-3) / 1e6, 1),
                          "adjoint_MLUPS": round(nb / (adj_ms * 1e-3) / 1e6, 1)}}
        sb.close()
        del sb
        torch.cuda.empty_cache()

    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(args, lats, dev)

    levelset = paper_hs = None
    if rank == 0 and not args.no_extra:
        levelset = levelset_leg(dev)
        paper_hs = paper_heat_sink_leg(dev)

    served = None
    if not args.no_serve:
        served = run_serve(args, device=dev)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(lats[RES[1]], fwd_steps=20, adj_steps=6)

    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 1), "unit": "MLUPS", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(total_ms / args.steps, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": {"fp32": "f32", "fp64": "f64",
                                                               "fp16": "f16-offset/f32",
                                                               "bf16": "bf16-offset/f32"}[args.storage],
            "data": "synthetic",
            "config": {"workload": f"3D D3Q19 pipe bend {args.n}^3, gamma = filtered noise (seed 1), "
                                   f"Re in {list(RES)}, forward + adjoint to residual {TOL} + dJ/dgamma",
                       "lattice": [args.n] * 3, "storage": args.storage, "check_every": CHECK,
                       "l2": "flushed (512 MB write) between timed steps",
                       "parallelism": f"replicas x{world}"},
            "per_re": {str(k): v for k, v in per.items()},
            "diverged": {"note": "updates of solves that diverged (no dJ/dgamma) are not counted "
                                 "in value; their time is",
                         "updates_per_step": int(total_lost // max(args.steps, 1)),
                         "MLUPS_if_counted": round((total_ups + total_lost) / (total_ms * 1e-3) / 1e6, 1)},
            "roofline": roof, "roofline_at_workload": at_workload,
            "cpu_baseline": cpu, "e2e": e2e, "clocks": clk, "served": served,
            "levelset": levelset, "paper_heat_sink": paper_hs,
            "gpu_launches": int(total_launch),
        }
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


def levelset_leg(dev, iters=40):
    """The paper's optimiser (Eq. 13-15, 66-67) on the 64 x 64 D2Q9 pipe bend
    (FP64, tau 0.6, V_max 0.08 pi): per-iteration time of forward + adjoint
    (warm-started, tolerance 1e-6) + dJ/dgamma + the level-set update.  From
    the empty chamber (phi = 1) the volume term lowers phi by about K lambda
    per iteration, so solid first appears after about 16 iterations; 40 show
    the fluid fraction falling towards V_max while J rises (Sec. 3.1, Fig. 4)."""
    import torch

    from paper_2501_02161_gb300 import inputs as I
    from paper_2501_02161_gb300.levelset import level_set_loop
    from paper_2501_02161_gb300.solver import Solver

    lat = I.workload("pipe_bend_2d_64x64")
    s = Solver.from_lattice(lat, storage="fp64", device=dev)
    level_set_loop(s, lat, iters=1, K=0.25, sigma=5e-3, vmax=0.08 * math.pi, tol=1e-6,
                   max_steps=200000, check_every=1000)   # untimed: captures the step graphs
    s.close()
    s = Solver.from_lattice(lat, storage="fp64", device=dev)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _, hist = level_set_loop(s, lat, iters=iters, K=0.25, sigma=5e-3, vmax=0.08 * math.pi,
                             tol=1e-6, max_steps=200000, check_every=1000)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    s.close()
    return {"workload": "2D D2Q9 pipe bend 64x64 FP64 from the empty chamber, level set K 0.25, "
                        "sigma 5e-3, V_max 0.08 pi, solves to 1e-6 warm-started",
            "iters": iters, "s_per_iter": round(dt / iters, 4),
            "every": 4,
            "J": [round(h["J"], 6) for h in hist[::4]] + [round(hist[-1]["J"], 6)],
            "fluid_fraction": [round(h["fluid_fraction"], 4) for h in hist[::4]]
            + [round(hist[-1]["fluid_fraction"], 4)]}


def paper_heat_sink_leg(dev, re_values=(60.0,)):
    """The paper's heat-sink problem (Sec. 3.3): a quarter domain with
    symmetry planes, pressure-driven inlet holding T = 0 (Eq. 70), heat
    generated in the solid (Eq. 69, 71) and J = -sum Q (Eq. 72), Pr 7.1,
    conductivity ratio 100; forward (flow + temperature) and adjoint to 1e-6
    in FP32, node updates per second over all phases."""
    import torch

    from paper_2501_02161_gb300 import inputs as I
    from paper_2501_02161_gb300.solver import Solver

    out = {"workload": "quarter heat sink 192x48x24 (full channel 192x96x48), FP32, tol 1e-6"}
    for re in re_values:
        lat = I.heat_sink_quarter(nx=192, ny=48, nz=24, re=re)
        s = Solver.from_lattice(lat, storage="fp32", device=dev)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        steps = {}
        status = "ok"
        for ph, name in ((0, "flow"), (1, "temperature"), (3, "temperature_adjoint"), (2, "flow_adjoint")):
            r = s.solve_phase(ph, tol=1e-6, max_steps=1000000, check_every=1000, strict=False)
            steps[name] = r.steps
            if r.status < 0:
                status = "diverged"
                break
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        rec = {"steps": steps, "seconds": round(dt, 3), "status": status,
               "MLUPS": round(sum(steps.values()) * lat.n / dt / 1e6, 1)}
        if status == "ok":
            rec["J_Q"] = s.objective()
            sens = s.sensitivity(dtype=torch.float64)
            rec["dJdgamma_abs_max"] = float(sens.abs().max())
        s.close()
        out[f"re_{re:g}"] = rec
    return out


def run_e2e(args, lats, dev):
    """Same metric through the C-ABI with host buffers: each step uploads the
    inputs (flags, gamma, boundary values) from pinned host memory and reads
    dJ/dgamma back; the copies are inside the timed region."""
    import numpy as np
    import torch

    from paper_2501_02161_gb300.solver import Solver

    host = {}
    for re, lat in lats.items():
        host[re] = (torch.from_numpy(lat.flags.copy()).pin_memory(),
                    torch.from_numpy(lat.gamma.astype(np.float32)).pin_memory(),
                    torch.from_numpy(lat.bcval.astype(np.float32)).pin_memory())
    N = lats[RES[0]].n
    out = torch.empty(N, dtype=torch.float32).pin_memory()
    solvers = {re: Solver.from_lattice(lat, storage=args.storage, device=dev)
               for re, lat in lats.items()}

    def step():
        ups = 0
        for re, s in solvers.items():
            fl, ga, bc = host[re]
            s.set_flags(fl)
            s.set_gamma(ga)
            s.set_bc_values(bc)
            rf = s.forward(tol=TOL, max_steps=CAP, check_every=CHECK, reset=True, strict=False)
            if rf.status < 0:
                continue  # diverged: no dJ/dgamma, its updates are not counted
            ra = s.adjoint(tol=TOL, max_steps=CAP, check_every=CHECK, reset=True, strict=False)
            if ra.status >= 0:
                s.sensitivity(out=out)
                ups += (rf.steps + ra.steps) * N
        return ups

    step()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ups = 0
    for _ in range(max(1, args.steps)):
        ups += step()
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    for s in solvers.values():
        s.close()
    return {"value": round(ups / dt / 1e6, 1), "unit": "MLUPS",
            "h2d_bytes_per_step": int(len(RES) * N * (1 + 4 + 16)),
            "d2h_bytes_per_step": int(len(RES) * N * 4)}


def cpu_baseline(lat, fwd_steps, adj_steps):
    """The FP64 oracle on a bounded sample of the same workload (host cores)."""
    from oracle import oracle as O
    O.build()
    orc = O.Oracle(lat)
    t0 = time.perf_counter()
    orc.flow_run(fwd_steps)
    t1 = time.perf_counter()
    orc.adjoint_run(adj_steps)
    t2 = time.perf_counter()
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    ups = (fwd_steps + adj_steps) * lat.n
    return {"value": round(ups / (t2 - t0) / 1e6, 3), "unit": "MLUPS", "cores": cores,
            "kind": "oracle",
            "sample": f"{lat.name} Re={lat.re}: {fwd_steps} forward + {adj_steps} "
                      f"adjoint steps from rest, FP64, OpenMP over nodes "
                      f"(forward {fwd_steps * lat.n / (t1 - t0) / 1e6:.2f} MLUPS, "
                      f"adjoint {adj_steps * lat.n / (t2 - t1) / 1e6:.2f} MLUPS)"}


# ---------------------------------------------------------------------------
# reference arm: the oracle, as it stands, on the host cores
# ---------------------------------------------------------------------------

def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_2501_02161_gb300 import inputs as I
    lats = {re: I.pipe_bend_3d(n=args.n, re=re, seed=1) for re in RES}
    fwd, adj = 8, 2

    def step():
        t0 = time.perf_counter()
        ups = 0
        from oracle import oracle as O
        for lat in lats.values():
            orc = O.Oracle(lat)
            orc.flow_run(fwd)
            orc.adjoint_run(adj)
            ups += (fwd + adj) * lat.n
        return ups, time.perf_counter() - t0

    from oracle import oracle as O
    O.build()
    for _ in range(args.warmup):
        step()
    tot_u, tot_t = 0, 0.0
    for _ in range(args.steps):
        u, t = step()
        tot_u += u
        tot_t += t
    v = tot_u / tot_t / 1e6
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    line = {"impl": "reference", "metric": METRIC, "value": round(v, 3), "unit": "MLUPS",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(tot_t / args.steps * 1e3, 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"3D D3Q19 pipe bend {args.n}^3, Re in {list(RES)}; "
                                   f"bounded sample per step: {fwd} forward + {adj} adjoint steps per Re",
                       "lattice": [args.n] * 3},
            "cpu_baseline": {"value": round(v, 3), "unit": "MLUPS", "cores": cores,
                             "kind": "oracle",
                             "sample": f"{fwd} forward + {adj} adjoint oracle steps per Re from rest"},
            "e2e": {"value": round(v, 3), "unit": "MLUPS", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


if __name__ == "__main__":
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    elif a.mode == "kernels":
        run_kernels(a)
    elif a.mode == "precision":
        run_precision(a)
    elif a.mode == "autograd":
        run_autograd(a)
    elif a.mode == "levelset":
        run_levelset(a)
    elif a.mode == "batchcmp":
        run_batchcmp(a)
    elif a.mode == "stability":
        run_stability(a)
    elif a.mode == "serve":
        import torch
        torch.cuda.set_device(0)
        print(json.dumps({"mode": "serve", **run_serve(a, nreq=a.nreq)}))
    else:
        run_ours(a)
