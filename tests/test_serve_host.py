"""Host-side scheduling of the serving loop, on CPU.

The server's decisions (admission in arrival order, the slot and in-flight
node caps, one request per design at a time, HBM-budget eviction with the
design state moved to host memory and brought back) are plain Python; here
they run against stand-ins for the solver and the batch, so every rule is
checked without a GPU.  The GPU tests check the numbers; these check the
schedule.
"""
import ctypes
import itertools

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2501_02161_gb300 import serve as S
from paper_2501_02161_gb300.solver import Report


@pytest.fixture(scope="module", autouse=True)
def library():
    from paper_2501_02161_gb300 import build as B
    B.build()  # lbm_footprint_bytes is a host function of the library


class FakeSolver:
    _ids = itertools.count(1)
    live = {}

    def __init__(self, lat):
        self.lat = lat
        self.N = lat.n
        self.rdtype = torch.float32
        self._ctx = ctypes.c_void_p(next(FakeSolver._ids))
        self.gamma = None
        self.imported = None
        FakeSolver.live[self._ctx.value] = self

    @classmethod
    def from_lattice(cls, lat, storage="fp32", device=None):
        return cls(lat)

    def set_gamma(self, g):
        self.gamma = g

    def sensitivity(self, dtype=None):
        return torch.full((self.N,), float(self._ctx.value), dtype=dtype or torch.float32)

    def export_state(self):
        return torch.full((64,), self._ctx.value % 251, dtype=torch.uint8)

    def import_state(self, st):
        self.imported = st

    def close(self):
        FakeSolver.live.pop(self._ctx.value, None)
        for b in FakeBatch.instances:  # lbm_destroy releases it from its batch
            b.held.pop(self._ctx.value, None)


class FakeBatch:
    """Completes a context after a number of steps proportional to its nodes
    (one step per 32^3 worth of nodes); records what ran together; counts
    admitted contexts against the memory budget like the library's batch."""
    instances = []

    def __init__(self, storage, check_every, max_slots, solo_tiles=None, budget_bytes=0):
        self.active = {}
        self.log = []
        self.done = []
        self.storage = storage
        self.budget = budget_bytes
        self.held = {}
        FakeBatch.instances.append(self)

    def memory(self):
        return self.budget, sum(self.held.values())

    def try_admit(self, solver, tol, max_steps, reset):
        k = solver._ctx.value
        if k not in self.held:
            fp = S.footprint(solver.lat, self.storage)
            if self.budget and sum(self.held.values()) + fp > self.budget:
                return None
            self.held[k] = fp
        self.active[k] = [solver, max(1, solver.N // 32768), reset]
        return 0

    def admit(self, solver, tol, max_steps, reset):
        slot = self.try_admit(solver, tol, max_steps, reset)
        assert slot is not None, "over the memory budget"
        return slot

    def step(self):
        self.log.append(sorted(self.active))
        for ctx in list(self.active):
            self.active[ctx][1] -= 1
            if self.active[ctx][1] <= 0:
                self.done.append(ctx)
                del self.active[ctx]
        return len(self.active)

    def poll(self):
        out = [(0, ctx, Report(10, 0.0, 0.0, 1.0, 0.0, 0)) for ctx in self.done]
        self.done = []
        return out

    def close(self):
        pass


@pytest.fixture
def fakes(monkeypatch):
    FakeSolver.live.clear()
    FakeBatch.instances.clear()
    monkeypatch.setattr(S, "Solver", FakeSolver)
    monkeypatch.setattr(S, "Batch", FakeBatch)
    return FakeBatch.instances


def _reqs(n=24, seed=3):
    return S.make_requests(n, seed=seed, rate=None, shapes=[(32, 32, 32), (64, 64, 64), (96, 48, 24)],
                           re_range=(10.0, 60.0))


def test_footprint_of_a_request_matches_its_lattice():
    for r in _reqs(12):
        assert S.footprint_of(r, "fp32") == S.footprint(S.lattice_for(r), "fp32")
        assert S.footprint_of(r, "fp16") == S.footprint(S.lattice_for(r), "fp16")


def test_lattice_prefetch_gives_the_same_lattices():
    reqs = _reqs(6)
    prep = S.LatticePrep(workers=2, ahead=4)
    prep.want(reqs)
    for r in reqs:
        a, b = prep.get(r), S.lattice_for(r)
        assert np.array_equal(a.flags, b.flags) and np.array_equal(a.gamma, b.gamma)
        assert np.array_equal(a.bcval, b.bcval) and a.re == b.re
    prep.close()


def test_schedule_respects_slots_node_cap_and_design_order(fakes):
    reqs = _reqs()
    srv = S.Server("fp32", budget_bytes=1 << 60, check_every=500, max_slots=3,
                   max_active_nodes=400_000, device="cpu")
    res = srv.run(reqs, realtime=False)
    log = fakes[0].log
    srv.close()
    assert all(r.status == 0 and r.done >= r.admitted for r in res)
    assert max(len(step) for step in log) <= 3   # slots
    assert max(len(step) for step in log) >= 2   # lattices did share the GPU
    # one request per design at a time, and in arrival order per design
    order = {}
    for r in sorted(res, key=lambda r: r.admitted):
        order.setdefault(reqs[r.rid].design, []).append(r)
    for d, rs in order.items():
        for a, b in zip(rs, rs[1:]):
            assert a.done <= b.admitted and a.rid < b.rid
    # optimisation steps on a finished design warm-start
    assert any(r.kind == "opt" and r.warm for r in res)


def test_node_cap_bounds_the_in_flight_nodes(fakes):
    reqs = _reqs()
    cap = 400_000
    srv = S.Server("fp32", budget_bytes=1 << 60, check_every=500, max_slots=8,
                   max_active_nodes=cap, device="cpu")
    seen = []
    orig = srv.batch.step

    def step():
        seen.append(srv._active_nodes())
        return orig()
    srv.batch.step = step
    srv.run(reqs, realtime=False)
    srv.close()
    biggest = max(int(np.prod(r.shape)) for r in reqs)
    assert max(seen) <= max(cap, biggest)


def test_tight_budget_moves_designs_to_host_and_back(fakes):
    reqs = _reqs(30, seed=4)
    biggest = max(S.footprint_of(r, "fp32") for r in reqs)
    srv = S.Server("fp32", budget_bytes=int(1.5 * biggest), check_every=500, max_slots=4,
                   device="cpu")
    peak = []
    orig = srv.batch.step

    def step():
        peak.append(srv.used)
        return orig()
    srv.batch.step = step
    res = srv.run(reqs, realtime=False)
    restored = srv.n_restored
    srv.close()
    assert max(peak) <= 1.5 * biggest
    assert all(r.status == 0 for r in res)
    warm_opt = [r for r in res if r.kind == "opt" and r.warm]
    assert restored >= 1 and len(warm_opt) >= restored
    assert not FakeSolver.live  # every context was closed


def test_host_budget_drops_the_oldest_offloaded_state(fakes):
    reqs = _reqs(30, seed=4)
    biggest = max(S.footprint_of(r, "fp32") for r in reqs)
    srv = S.Server("fp32", budget_bytes=int(1.5 * biggest), check_every=500, max_slots=4,
                   device="cpu", host_budget_bytes=64)  # room for one fake state
    res = srv.run(reqs, realtime=False)
    held = len(srv.offloaded)
    srv.close()
    assert held <= 1
    assert all(r.status == 0 for r in res)


def test_request_contents_do_not_depend_on_the_arrival_rate():
    """The offline and online streams differ only in arrival times, so their
    results can be compared request by request."""
    a = S.make_requests(64, seed=5, rate=None)
    b = S.make_requests(64, seed=5, rate=3.0)
    key = lambda r: (r.rid, r.shape, r.re, r.thermal, r.kind, r.design, r.seed)
    assert [key(r) for r in a] == [key(r) for r in b]
    assert all(r.arrival == 0.0 for r in a)
    arr = [r.arrival for r in b]
    assert arr == sorted(arr) and arr[-1] > 0
    # an optimisation step refers to an earlier request's design, with its lattice
    for r in a:
        if r.kind == "opt":
            base = a[r.design]
            assert base.rid < r.rid and base.kind == "sens"
            assert (base.shape, base.re, base.thermal, base.seed) == (r.shape, r.re, r.thermal, r.seed)


def test_summary_counts_failures_and_takes_latency_percentiles():
    res = []
    for k in range(100):
        r = S.Result(k, "sens", arrival=0.0, admitted=0.0, done=float(k + 1), status=0 if k % 10 else -4)
        res.append(r)
    s = S.summarize(res)
    assert s["requests"] == 100 and s["completed"] == 90 and s["failed"] == 10
    assert s["wall_s"] == 100.0 and s["sens_per_s"] == 0.9
    assert s["p50_s"] == 50.5 and abs(s["p99_s"] - 99.01) < 1e-9


def test_a_request_larger_than_the_budget_fails_instead_of_waiting_forever(fakes):
    """With nothing running and every idle design evicted, a request that still
    does not fit can never be admitted: it fails with LBM_ERR_OOM and the
    others are served."""
    from paper_2501_02161_gb300 import _capi as C
    reqs = _reqs(20, seed=6)
    sizes = sorted({S.footprint_of(r, "fp32") for r in reqs})
    budget = sizes[-2]  # every shape but the largest fits
    srv = S.Server("fp32", budget_bytes=budget, check_every=500, max_slots=4, device="cpu")
    res = srv.run(reqs, realtime=False)
    srv.close()
    for q, r in zip(reqs, res):
        too_big = S.footprint_of(q, "fp32") > budget
        warm = q.kind == "opt" and r.warm
        assert r.status == (C.LBM_ERR_OOM if too_big and not warm else 0), (q.rid, q.shape, r.status)
    assert any(r.status == C.LBM_ERR_OOM for r in res) and any(r.status == 0 for r in res)


def test_summary_breaks_failures_down_by_shape_and_re():
    reqs = [S.Request(0, 0.0, (32, 32, 32), 15.0, False, "sens", 0, 1),
            S.Request(1, 0.0, (32, 32, 32), 300.0, True, "sens", 1, 2),
            S.Request(2, 0.0, (64, 64, 64), 60.0, False, "sens", 2, 3),
            S.Request(3, 0.0, (64, 64, 64), 499.0, False, "sens", 3, 4)]
    res = [S.Result(0, "sens", 0.0, 0.0, 1.0, status=0), S.Result(1, "sens", 0.0, 0.0, 2.0, status=-4),
           S.Result(2, "sens", 0.0, 0.0, 3.0, status=1), S.Result(3, "sens", 0.0, 0.0, 4.0, status=-4)]
    s = S.summarize(res, requests=reqs)
    assert s["completed"] == 2 and s["failed"] == 2
    assert s["by_shape"] == {"32x32x32": {"completed": 1, "failed": 0},
                             "32x32x32/thermal": {"completed": 0, "failed": 1},
                             "64x64x64": {"completed": 1, "failed": 1}}
    assert s["by_re"]["10-20"] == {"completed": 1, "failed": 0}
    assert s["by_re"]["200-500"] == {"completed": 0, "failed": 2}
    assert s["by_re"]["50-100"] == {"completed": 1, "failed": 0}
    assert s["by_status"] == {"LBM_ERR_DIVERGED": 2, "LBM_NOT_CONVERGED": 1, "LBM_OK": 1}


def test_failed_restore_keeps_the_host_budget(fakes):
    """A design whose state is on the host and that cannot come back (no
    device room) goes back to the host store: the host budget still holds
    afterwards (the oldest states are dropped first)."""
    srv = S.Server("fp32", budget_bytes=1 << 60, check_every=500, max_slots=4, device="cpu",
                   host_budget_bytes=128)
    reqs = _reqs(4, seed=3)
    lat = S.lattice_for(reqs[0])
    st = torch.zeros(64, dtype=torch.uint8)
    for d in (100, 101):
        srv.offloaded[d] = (lat, torch.as_tensor(lat.gamma), torch.zeros(lat.n), st.clone())
        srv.host_used += 64
    req = S.Request(99, 0.0, reqs[0].shape, reqs[0].re, reqs[0].thermal, "opt", 100, reqs[0].seed)
    srv.host_budget = 64            # tightened meanwhile: only one state fits
    srv._make_room = lambda nb: False
    assert not srv._admit(req, S.Result(99, "opt", 0.0), 0.0)
    assert srv.host_used <= srv.host_budget
    assert 100 in srv.offloaded      # the one that could not come back is the newest entry now
    srv.close()
