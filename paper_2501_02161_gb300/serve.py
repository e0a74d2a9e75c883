"""Serving: continuous batching of sensitivity and optimisation-step requests.

Requests of mixed lattice shapes and Re arrive over time.  The server admits
them, in arrival order, as batch slots and HBM budget free up (admission by
the device footprint each context needs), keeps finished designs resident so
that an optimisation-step request on the same design warm-starts from its
populations, and advances every resident lattice together: one
`lbm_batch_step` runs K steps of every resident lattice, each on its own
CUDA graph and stream by default (all concurrently), or, below a chosen tile
threshold, packed into one graph of persistent kernels that walk the tiles
of all packed lattices.  Lattices that arrive while others run join at the
next step.  The baseline serves the same requests one at a time through
the plain single-context FP32 path.  All solver work runs in the CUDA library;
this module only schedules.
"""
from __future__ import annotations

import ctypes
import itertools
import time
from collections import OrderedDict, deque
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass, field

import numpy as np
import torch

from . import _capi as C
from . import inputs as I
from .solver import STORAGES, Report, Solver

SHAPES = [(32, 32, 32), (64, 64, 64), (96, 48, 24), (128, 64, 32), (192, 96, 48)]


@dataclass
class Request:
    rid: int
    arrival: float          # seconds after the start of the run
    shape: tuple
    re: float
    thermal: bool
    kind: str               # "sens" or "opt" (optimisation step on an earlier design)
    design: int             # design id (opt requests refer to an earlier sens request's design)
    seed: int


@dataclass
class Result:
    rid: int
    kind: str
    arrival: float
    admitted: float = float("nan")
    done: float = float("nan")
    status: int = 0
    steps: int = 0
    J: float = float("nan")
    warm: bool = False
    sens: torch.Tensor | None = None

    @property
    def latency(self) -> float:
        return self.done - self.arrival


def make_requests(n: int = 256, seed: int = 5, rate: float | None = None,
                  shapes=SHAPES, opt_frac: float = 0.2, thermal_frac: float = 0.5,
                  re_range=(10.0, 500.0)) -> list:
    """Seeded request stream: shapes uniform over `shapes`, Re ~ U[re_range],
    thermal with probability thermal_frac, a fraction opt_frac of
    optimisation-step requests on earlier designs, Poisson arrivals at `rate`
    requests per second (all at t=0 when rate is None)."""
    rng = np.random.default_rng(seed)
    arr = np.random.default_rng([seed, 1])   # arrivals: own stream, contents do not depend on rate
    t = 0.0
    reqs = []
    sens_ids = []
    for k in range(n):
        if rate:
            t += arr.exponential(1.0 / rate)
        if sens_ids and rng.random() < opt_frac:
            base = reqs[sens_ids[rng.integers(len(sens_ids))]]
            reqs.append(Request(k, t, base.shape, base.re, base.thermal, "opt", base.design, base.seed))
        else:
            shape = shapes[rng.integers(len(shapes))]
            reqs.append(Request(k, t, tuple(shape), float(rng.uniform(*re_range)),
                                bool(rng.random() < thermal_frac), "sens", k, int(rng.integers(1 << 30))))
            sens_ids.append(k)
    return reqs


def lattice_for(req: Request):
    nx, ny, nz = req.shape
    if req.thermal:
        return I.heat_sink(nx=nx, ny=ny, nz=nz, re=req.re, seed=req.seed % 100000)
    return I.pipe_bend_3d(n=nx, ny=ny, nz=nz, width=max(2, min(ny, nz) // 4), re=req.re,
                          seed=req.seed % 100000)


class LatticePrep:
    """Builds the lattices of the next few requests on worker threads while the
    GPU works (host numpy only; a lattice is a pure function of its request, so
    results do not change).  Both the server and the sequential baseline use it."""

    def __init__(self, workers: int = 2, ahead: int = 8):
        self.pool = ThreadPoolExecutor(max_workers=workers)
        self.futs = {}
        self.ahead = ahead

    def want(self, reqs, skip=lambda r: False):
        """Start building the first `ahead` requests of `reqs` (in order)."""
        for r in itertools.islice((r for r in reqs if not skip(r)), self.ahead):
            if r.rid not in self.futs:
                self.futs[r.rid] = self.pool.submit(lattice_for, r)

    def get(self, req):
        f = self.futs.pop(req.rid, None)
        return f.result() if f is not None else lattice_for(req)

    def drop(self, req):
        f = self.futs.pop(req.rid, None)
        if f is not None:
            f.cancel()

    def close(self):
        self.pool.shutdown(wait=True, cancel_futures=True)
        self.futs.clear()


def footprint(lat, storage: str) -> int:
    return int(C.lib().lbm_footprint_bytes(lat.stencil, lat.nx, lat.ny, lat.nz,
                                           STORAGES[storage], int(lat.thermal)))


def footprint_of(req: Request, storage: str) -> int:
    """Device bytes of the context a request needs (without building its lattice)."""
    nx, ny, nz = req.shape
    return int(C.lib().lbm_footprint_bytes(C.LBM_D3Q19, nx, ny, nz, STORAGES[storage],
                                           int(req.thermal)))


def opt_step_gamma(lat, gamma: torch.Tensor, sens: torch.Tensor, step: float = 0.05) -> torch.Tensor:
    """One projected-gradient update of the design nodes (fluid nodes)."""
    design = torch.as_tensor((lat.flags & 7) == I.FLUID, device=gamma.device)
    g = sens.to(gamma.dtype)
    scale = g[design].abs().max().clamp_min(1e-30)
    return torch.where(design, (gamma - step * g / scale).clamp(0.0, 1.0), gamma)


class Batch:
    """Thin owner of an lbm_batch (same names as the C-ABI)."""

    def __init__(self, storage: str = "fp32", check_every: int = 500, max_slots: int = 32,
                 solo_tiles: int | None = None, budget_bytes: int = 0):
        """solo_tiles: lattices with at least this many 256-node tiles run their
        own single-lattice graph beside the packed launch (0: pack every
        lattice; None: the library's default, 1: every lattice on its own
        graph and stream).
        budget_bytes: device memory the batch's contexts may hold together,
        admitted or kept for a warm start (0: no limit); the library counts it."""
        self.lib = C.lib()
        self._b = ctypes.c_void_p()
        C.check(self.lib.lbm_batch_create(ctypes.byref(self._b), STORAGES[storage],
                                          int(check_every), int(max_slots), int(budget_bytes)),
                "lbm_batch_create")
        if solo_tiles is not None:
            C.check(self.lib.lbm_batch_set_solo_tiles(self._b, int(solo_tiles)),
                    "lbm_batch_set_solo_tiles")
        self.max_slots = max_slots
        self._slots = (ctypes.c_int * max_slots)()
        self._ctxs = (ctypes.c_void_p * max_slots)()
        self._reps = (C.lbm_report * max_slots)()

    def admit(self, solver: Solver, tol: float, max_steps: int, reset: bool) -> int:
        o = C.lbm_solve_opts(float(tol), int(max_steps), 0, int(reset))
        slot = ctypes.c_int()
        C.check(self.lib.lbm_batch_admit(self._b, solver._ctx, ctypes.byref(o), ctypes.byref(slot)),
                "lbm_batch_admit")
        return slot.value

    def try_admit(self, solver: Solver, tol: float, max_steps: int, reset: bool):
        """admit, or None when the context does not fit the memory budget now"""
        o = C.lbm_solve_opts(float(tol), int(max_steps), 0, int(reset))
        slot = ctypes.c_int()
        code = self.lib.lbm_batch_admit(self._b, solver._ctx, ctypes.byref(o), ctypes.byref(slot))
        if code == C.LBM_ERR_OOM:
            return None
        C.check(code, "lbm_batch_admit")
        return slot.value

    def release(self, solver: Solver):
        C.check(self.lib.lbm_batch_release(self._b, solver._ctx), "lbm_batch_release")

    def memory(self):
        """(budget, bytes counted now)"""
        b, h = ctypes.c_size_t(), ctypes.c_size_t()
        C.check(self.lib.lbm_batch_memory(self._b, ctypes.byref(b), ctypes.byref(h)), "lbm_batch_memory")
        return b.value, h.value

    def step(self) -> int:
        n = ctypes.c_int()
        C.check(self.lib.lbm_batch_step(self._b, ctypes.byref(n)), "lbm_batch_step")
        return n.value

    def poll(self):
        n = ctypes.c_int()
        C.check(self.lib.lbm_batch_poll(self._b, self._slots, self._ctxs, self._reps,
                                        self.max_slots, ctypes.byref(n)), "lbm_batch_poll")
        out = []
        for k in range(n.value):
            r = self._reps[k]
            out.append((self._slots[k], self._ctxs[k],
                        Report(r.steps, r.residual, r.I, r.J, r.ms, r.status)))
        return out

    def close(self):
        if self._b:
            self.lib.lbm_batch_destroy(self._b)
            self._b = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching server over one GPU."""

    def __init__(self, storage: str = "fp32", budget_bytes: int | None = None,
                 check_every: int = 500, max_slots: int = 32, tol: float = 1e-4,
                 max_steps: int = 20000, keep_designs: bool = True, device=None,
                 max_active_nodes: int = 1_000_000, solo_tiles: int | None = None,
                 host_budget_bytes: int = 32 << 30):
        self.device = torch.device(device) if device else torch.device("cuda", torch.cuda.current_device())
        self.storage = storage
        if budget_bytes is None:
            free, _ = torch.cuda.mem_get_info(self.device)
            budget_bytes = int(free * 0.8)
        self.tol, self.max_steps = tol, max_steps
        self.keep = keep_designs
        # about a million in-flight nodes (one 192x96x48 lattice plus small
        # ones) already keep every SM busy; admitting more only shares the GPU
        # among more requests and lengthens everyone's latency
        self.max_active_nodes = max_active_nodes
        # the library's batch counts every context it admitted until it is
        # destroyed (running or kept for a warm start) against this budget
        self.batch = Batch(storage, check_every, max_slots, solo_tiles, budget_bytes)
        self.max_slots = max_slots
        self.resident = OrderedDict()   # design id -> (solver, lattice, gamma, last sens, bytes)
        self.offloaded = OrderedDict()  # design id -> (lattice, gamma, last sens, host state)
        self.host_used = 0
        self.host_budget = host_budget_bytes
        self.n_restored = 0             # designs brought back from host memory
        self.active = {}                # ctx pointer value -> (request, result, design id)
        self.prep = LatticePrep()

    @property
    def budget(self) -> int:
        return self.batch.memory()[0]

    @property
    def used(self) -> int:
        """device bytes of the resident designs, as the library counts them"""
        return self.batch.memory()[1]

    def _trim_host(self):
        while self.host_used > self.host_budget and self.offloaded:
            self.host_used -= self.offloaded.popitem(last=False)[1][3].numel()

    def _evict_one(self) -> bool:
        """Free the least recently used idle design's device memory; a design
        with a finished solve keeps its state in host memory (export_state) so
        a later optimisation step still warm-starts."""
        busy = {d for (_, _, d) in self.active.values()}
        for d in list(self.resident):
            if d not in busy:
                s, lat, gamma, sens, nb = self.resident.pop(d)
                if self.keep and sens is not None:
                    state = s.export_state()
                    self.offloaded[d] = (lat, gamma.cpu(), sens, state)
                    self.offloaded.move_to_end(d)
                    self.host_used += state.numel()
                    self._trim_host()
                s.close()  # lbm_destroy: the batch stops counting it
                return True
        return False

    def _warm_ready(self, req) -> bool:
        ent = self.resident.get(req.design)
        return req.kind == "opt" and ((ent is not None and ent[3] is not None)
                                      or req.design in self.offloaded)

    def _active_nodes(self) -> int:
        return sum(int(np.prod(r.shape)) for (r, _, _) in self.active.values())

    def _make_room(self, nb: int) -> bool:
        while self.budget and self.used + nb > self.budget:
            if not self._evict_one():
                return False
        return True

    def _admit(self, req: Request, res: Result, now: float) -> bool:
        if len(self.active) >= self.max_slots:
            return False
        if self.active and self._active_nodes() + int(np.prod(req.shape)) > self.max_active_nodes:
            return False
        d = req.design
        warm = False
        if any(dd == d for (_, _, dd) in self.active.values()):
            return False  # that design is still being solved: its next request waits
        if req.kind == "opt" and d in self.resident and self.resident[d][3] is not None:
            s, lat, gamma, sens, nb = self.resident[d]
            self.resident.move_to_end(d)
            gamma = opt_step_gamma(lat, gamma, sens)
            s.set_gamma(gamma)
            self.resident[d] = (s, lat, gamma, sens, nb)
            warm = True
            self.prep.drop(req)
        elif req.kind == "opt" and d in self.offloaded:
            # the design's state was moved to host memory: bring it back
            lat, gamma_h, sens, state = self.offloaded.pop(d)
            self.host_used -= state.numel()
            nb = footprint(lat, self.storage)
            if not self._make_room(nb):
                self.offloaded[d] = (lat, gamma_h, sens, state)
                self.host_used += state.numel()
                self._trim_host()
                return False
            s = Solver.from_lattice(lat, storage=self.storage, device=self.device)
            s.import_state(state)
            self.n_restored += 1
            gamma = opt_step_gamma(lat, gamma_h.to(self.device), sens)
            s.set_gamma(gamma)
            self.resident[d] = (s, lat, gamma, sens, nb)
            warm = True
            self.prep.drop(req)
        else:
            nb = footprint_of(req, self.storage)
            if not self._make_room(nb):
                return False
            lat = self.prep.get(req)
            s = Solver.from_lattice(lat, storage=self.storage, device=self.device)
            gamma = torch.as_tensor(lat.gamma, dtype=s.rdtype, device=self.device)
            if req.kind == "opt":
                # no state of the design is kept any more: replay its update cold
                gamma = gamma.clone()
            if d in self.resident:
                self.resident.pop(d)[0].close()
            self.offloaded.pop(d, None)
            self.resident[d] = (s, lat, gamma, None, nb)
        self.batch.admit(s, self.tol, self.max_steps, reset=not warm)
        res.admitted = now
        res.warm = warm
        self.active[s._ctx.value] = (req, res, d)
        return True

    def run(self, requests, realtime: bool = True):
        """Serve `requests` (arrival times in seconds from now); returns results."""
        order = deque(sorted(requests, key=lambda r: r.arrival))
        waiting = deque()
        results = {r.rid: Result(r.rid, r.kind, r.arrival) for r in requests}
        t0 = time.perf_counter()
        done = 0
        while done < len(requests):
            now = time.perf_counter() - t0 if realtime else float("inf")
            while order and order[0].arrival <= now:
                waiting.append(order.popleft())
            self.prep.want(waiting, skip=self._warm_ready)
            # admission: arrival order, except that a request whose design is
            # still being solved lets later requests for other designs pass;
            # the first request that does not fit in memory stops admission
            blocked = set()
            kept = deque()
            while waiting:
                req = waiting.popleft()
                if req.design in blocked:
                    kept.append(req)
                    continue
                busy = any(dd == req.design for (_, _, dd) in self.active.values())
                if busy:
                    blocked.add(req.design)
                    kept.append(req)
                    continue
                if not self._admit(req, results[req.rid], time.perf_counter() - t0):
                    kept.append(req)
                    kept.extend(waiting)
                    waiting.clear()
                    break
            waiting = kept
            if not self.active:
                if waiting:
                    # nothing runs, so every idle design was evicted, and the
                    # first waiting request still does not fit: it never will
                    req = waiting.popleft()
                    self.prep.drop(req)
                    res = results[req.rid]
                    res.status = C.LBM_ERR_OOM
                    res.admitted = res.done = time.perf_counter() - t0
                    done += 1
                    continue
                if order and realtime:
                    time.sleep(max(0.0, order[0].arrival - (time.perf_counter() - t0)))
                continue
            self.batch.step()
            for slot, ctx, rep in self.batch.poll():
                req, res, d = self.active.pop(ctx)
                s = self.resident[d][0]
                res.status = rep.status
                res.steps = rep.steps
                res.J = rep.J
                if rep.status >= 0:
                    sens = s.sensitivity(dtype=torch.float32)
                    res.sens = sens
                    ent = self.resident[d]
                    self.resident[d] = (ent[0], ent[1], ent[2], sens, ent[4])
                if self.device.type == "cuda":
                    torch.cuda.synchronize(self.device)
                res.done = time.perf_counter() - t0
                done += 1
                if not self.keep or rep.status < 0:
                    self.resident.pop(d)[0].close()
        return [results[r.rid] for r in requests]

    def close(self):
        self.prep.close()
        self.offloaded.clear()
        self.host_used = 0
        for d in list(self.resident):
            self.resident.pop(d)[0].close()
        self.batch.close()


def serve_sequential(requests, storage: str = "fp32", tol: float = 1e-4, max_steps: int = 20000,
                     check_every: int = 500, realtime: bool = True, keep_designs: bool = True,
                     device=None, max_designs: int | None = None):
    """Baseline: one request at a time, in arrival order, through the
    single-context solver (plain path, same tolerance and step caps).
    Finished designs stay resident like the server's (max_designs: LRU cap,
    None = no cap) so optimisation steps warm-start the same way."""
    dev = torch.device(device) if device else torch.device("cuda", torch.cuda.current_device())
    designs = OrderedDict()
    results = []
    prep = LatticePrep()
    ordered = sorted(requests, key=lambda r: r.arrival)
    warm_ready = lambda r: r.kind == "opt" and r.design in designs and designs[r.design][3] is not None
    t0 = time.perf_counter()
    for k, req in enumerate(ordered):
        if realtime:
            wait = req.arrival - (time.perf_counter() - t0)
            if wait > 0:
                time.sleep(wait)
        now = time.perf_counter() - t0 if realtime else float("inf")
        prep.want(itertools.takewhile(lambda r: r.arrival <= now, ordered[k:]), skip=warm_ready)
        res = Result(req.rid, req.kind, req.arrival, admitted=time.perf_counter() - t0)
        warm = False
        if warm_ready(req):
            s, lat, gamma, sens = designs[req.design]
            gamma = opt_step_gamma(lat, gamma, sens)
            s.set_gamma(gamma)
            warm = True
            prep.drop(req)
        else:
            lat = prep.get(req)
            if req.design in designs:
                designs.pop(req.design)[0].close()
            s = Solver.from_lattice(lat, storage=storage, device=dev)
            gamma = torch.as_tensor(lat.gamma, dtype=s.rdtype, device=dev)
        rf = s.forward(tol=tol, max_steps=max_steps, check_every=check_every, reset=not warm,
                       strict=False)
        sens = None
        rep_status, steps = rf.status, rf.steps
        if rf.status >= 0:
            ra = s.adjoint(tol=tol, max_steps=max_steps, check_every=check_every,
                           reset=not warm, strict=False)
            steps += ra.steps
            if ra.status >= 0:
                sens = s.sensitivity(dtype=torch.float32)
                rep_status = max(rf.status, ra.status)
            else:
                rep_status = ra.status
        torch.cuda.synchronize(dev)
        res.done = time.perf_counter() - t0
        res.status, res.steps, res.J, res.sens, res.warm = rep_status, steps, rf.J, sens, warm
        results.append(res)
        if keep_designs and rep_status >= 0:
            designs[req.design] = (s, lat, gamma, sens)
            designs.move_to_end(req.design)
            while max_designs is not None and len(designs) > max_designs:
                designs.popitem(last=False)[1][0].close()
        else:
            designs.pop(req.design, None)  # the design's state is no longer usable
            s.close()
    prep.close()
    for v in designs.values():
        v[0].close()
    return sorted(results, key=lambda r: r.rid)


RE_BANDS = [(10.0, 20.0), (20.0, 50.0), (50.0, 100.0), (100.0, 200.0), (200.0, 500.0)]


def summarize(results, wall: float | None = None, requests=None) -> dict:
    """Throughput and latency of a served run: the count of results per status
    (LBM_OK, LBM_NOT_CONVERGED within the step cap, LBM_ERR_DIVERGED,
    LBM_ERR_OOM) and, with the requests, completed / failed counts per
    lattice shape and per Re band (failed = an error status; a result not
    converged within the step cap counts as completed with its flag)."""
    ok = [r for r in results if r.status >= 0]
    lat = np.array([r.latency for r in results])
    wall = wall if wall is not None else max(r.done for r in results)
    out = {"requests": len(results), "completed": len(ok),
           "failed": len(results) - len(ok),
           "sens_per_s": round(len(ok) / wall, 3), "wall_s": round(wall, 3),
           "p50_s": round(float(np.percentile(lat, 50)), 4),
           "p99_s": round(float(np.percentile(lat, 99)), 4),
           "mean_s": round(float(lat.mean()), 4)}
    by_status = {}
    for r in results:
        name = C.STATUS_NAMES.get(r.status, str(r.status))
        by_status[name] = by_status.get(name, 0) + 1
    out["by_status"] = dict(sorted(by_status.items()))
    if requests is not None:
        by = {r.rid: r for r in requests}
        shapes, bands = {}, {}
        for r in results:
            q = by[r.rid]
            sk = "x".join(str(d) for d in q.shape) + ("/thermal" if q.thermal else "")
            band = next((f"{lo:g}-{hi:g}" for lo, hi in RE_BANDS if lo <= q.re < hi),
                        f">={RE_BANDS[-1][1]:g}" if q.re >= RE_BANDS[-1][1] else f"<{RE_BANDS[0][0]:g}")
            for tab, key in ((shapes, sk), (bands, band)):
                c = tab.setdefault(key, [0, 0])
                c[0 if r.status >= 0 else 1] += 1
        out["by_shape"] = {k: {"completed": v[0], "failed": v[1]} for k, v in sorted(shapes.items())}
        out["by_re"] = {k: {"completed": v[0], "failed": v[1]} for k, v in bands.items()}
    return out
