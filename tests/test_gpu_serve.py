"""Batched solves and the continuous-batching server.

Each context's result must be the same alone and in any mix (the batched
kernels run each lattice's own launch geometry and reductions, so the results
are compared bit for bit), the same as through the single-context calls, and
the server must give the same answers as the one-at-a-time baseline.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2501_02161_gb300 import inputs as I

pytestmark = pytest.mark.gpu

K = 200


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2501_02161_gb300 import build as B
    B.build()


def mix():
    return [I.pipe_bend_3d(n=24, width=6, re=20.0, seed=2),
            I.heat_sink(nx=32, ny=16, nz=12, re=20.0, q_flux=2e-3, seed=4),
            I.six_port_box(),
            I.pipe_bend_3d(n=32, width=8, re=40.0, seed=3, ny=24, nz=20),
            I.heat_sink(nx=40, ny=20, nz=12, re=15.0, q_flux=2e-3, seed=6)]


def solve_batched(lats, storage="fp32", tol=1e-5, max_steps=20000, order=None, solo_tiles=None):
    from paper_2501_02161_gb300.serve import Batch
    from paper_2501_02161_gb300.solver import Solver
    b = Batch(storage, K, 8, solo_tiles)
    solvers = [Solver.from_lattice(l, storage=storage) for l in lats]
    for k in (order or range(len(lats))):
        b.admit(solvers[k], tol, max_steps, reset=True)
    reps = {}
    while len(reps) < len(lats):
        b.step()
        for slot, ctx, rep in b.poll():
            k = [s._ctx.value for s in solvers].index(ctx)
            reps[k] = rep
    out = []
    for k, s in enumerate(solvers):
        out.append((reps[k], s.sensitivity(dtype=torch.float64).cpu(), s.fields(torch.float64)[1].cpu()))
        s.close()
    b.close()
    return out


# solo_tiles: None = library default (every lattice on its own graph), 0 = all
# packed into the persistent launch, 40 = some of each
@pytest.mark.parametrize("solo_tiles", [None, 0, 40])
def test_batched_equals_single_context_bitwise(solo_tiles):
    from paper_2501_02161_gb300.solver import Solver
    lats = mix()
    got = solve_batched(lats, solo_tiles=solo_tiles)
    for lat, (rep, sens, u) in zip(lats, got):
        s = Solver.from_lattice(lat, storage="fp32")
        rf = s.forward(tol=1e-5, max_steps=20000, check_every=K)
        ra = s.adjoint(tol=1e-5, max_steps=20000, check_every=K)
        assert rep.status == 0 and rep.steps == rf.steps + ra.steps
        assert torch.equal(s.sensitivity(dtype=torch.float64).cpu(), sens), lat.name
        assert torch.equal(s.fields(torch.float64)[1].cpu(), u), lat.name
        assert rep.J == rf.J
        s.close()


def test_alone_and_in_the_mix_are_identical():
    lats = mix()
    together = solve_batched(lats, order=[4, 2, 0, 3, 1])
    for k, lat in enumerate(lats):
        alone = solve_batched([lat])[0]
        assert alone[0].steps == together[k][0].steps
        assert torch.equal(alone[1], together[k][1]), lat.name


def _reqs():
    from paper_2501_02161_gb300.serve import make_requests
    return make_requests(14, seed=7, rate=None, shapes=[(24, 24, 24), (32, 16, 16), (40, 20, 12)],
                         re_range=(5.0, 60.0))


def test_server_admission_respects_the_hbm_budget():
    from paper_2501_02161_gb300.serve import Server, footprint, lattice_for, summarize
    reqs = _reqs()
    biggest = max(footprint(lattice_for(r), "fp32") for r in reqs)
    srv = Server("fp32", budget_bytes=int(2.5 * biggest), check_every=K, max_slots=8,
                 tol=1e-5, max_steps=20000)
    peak, conc = [], []
    orig = srv.batch.step

    def step():
        peak.append(srv.used)
        conc.append(len(srv.active))
        return orig()
    srv.batch.step = step
    served = srv.run(reqs, realtime=False)
    srv.close()
    assert max(peak) <= 2.5 * biggest
    assert max(conc) >= 2          # lattices did run together
    summ = summarize(served)
    assert summ["completed"] + summ["failed"] == len(reqs)


def test_server_matches_sequential_bitwise():
    from paper_2501_02161_gb300.serve import Server, serve_sequential
    reqs = _reqs()
    srv = Server("fp32", check_every=K, max_slots=8, tol=1e-5, max_steps=20000)
    served = srv.run(reqs, realtime=False)
    srv.close()
    seq = serve_sequential(reqs, "fp32", tol=1e-5, max_steps=20000, check_every=K, realtime=False)
    assert any(r.kind == "opt" and r.warm for r in served)
    for a, b in zip(served, seq):
        assert (a.status, a.warm) == (b.status, b.warm), (a.rid, a.status, b.status)
        if a.status >= 0:
            assert a.steps == b.steps, (a.rid, a.steps, b.steps)
            assert torch.equal(a.sens.cpu(), b.sens.cpu()), a.rid


def test_tight_budget_offloads_designs_and_still_matches_sequential():
    """With room for about two lattices the server evicts designs; finished
    ones move to host memory (lbm_export_state) and come back for their
    optimisation steps (lbm_import_state), so every result, warm starts
    included, is bit-identical to the baseline that keeps all designs."""
    from paper_2501_02161_gb300.serve import Server, footprint, lattice_for, serve_sequential
    reqs = _reqs()
    biggest = max(footprint(lattice_for(r), "fp32") for r in reqs)
    srv = Server("fp32", budget_bytes=int(2.5 * biggest), check_every=K, max_slots=8,
                 tol=1e-5, max_steps=20000)
    served = srv.run(reqs, realtime=False)
    restored = srv.n_restored
    srv.close()
    seq = serve_sequential(reqs, "fp32", tol=1e-5, max_steps=20000, check_every=K, realtime=False)
    assert restored >= 1
    for a, b in zip(served, seq):
        assert (a.status, a.warm) == (b.status, b.warm), (a.rid, a.status, b.status)
        if a.status >= 0:
            assert a.steps == b.steps, (a.rid, a.steps, b.steps)
            assert torch.equal(a.sens.cpu(), b.sens.cpu()), a.rid


@pytest.mark.parametrize("solo_tiles", [None, 0], ids=["solo", "packed"])
def test_largest_served_shape_matches_oracle(solo_tiles):
    """The largest served lattice (192 x 96 x 48 heat sink, flow + temperature)
    through the batch, on its own graph (solo, the default) and
    inside the packed persistent launch, against the FP64 oracle after the same
    fixed number of steps of every phase: every node compared, FP32 tolerances
    (rel-L2 1e-5 on rho, u, T, J; 1e-4 on f*, g*, dJ/dgamma)."""
    import numpy as np
    from oracle import oracle as O
    from paper_2501_02161_gb300.serve import Batch
    from paper_2501_02161_gb300.solver import Solver
    O.build()
    n = 20
    lat = I.heat_sink(nx=192, ny=96, nz=48, re=50.0, seed=4)
    b = Batch("fp32", 10, 4, solo_tiles)
    s = Solver.from_lattice(lat, storage="fp32")
    b.admit(s, 0.0, n, reset=True)
    reps = []
    while not reps:
        b.step()
        reps = b.poll()
    assert reps[0][2].status == 0 and reps[0][2].steps == 4 * n
    rho, u, T = s.fields(torch.float64)
    fs, gs = s.adjoint_fields(torch.float64)
    g = dict(rho=rho.cpu().numpy(), u=u.cpu().numpy().T, T=T.cpu().numpy(),
             sens=s.sensitivity(dtype=torch.float64).cpu().numpy(),
             fs=fs.cpu().numpy().T, gs=gs.cpu().numpy().T)
    s.close()
    b.close()

    orc = O.Oracle(lat)
    orc.flow_run(n)
    orc.thermal_run(n)
    o = {"T": orc.temperature()}
    orc.thermal_adjoint_run(n)
    orc.finish_thermal_adjoint()
    o["gs"] = orc.thermal_adjoint_post_bc().reshape(orc.N, 7)
    orc.adjoint_run(n)
    o["rho"], o["u"] = orc.macro()
    o.update(sens=orc.sensitivity(), fs=orc.adjoint_post_bc().reshape(orc.N, orc.Q))

    def rel(a, c):
        a, c = np.asarray(a, float), np.asarray(c, float)
        return np.linalg.norm(a - c) / max(np.linalg.norm(c), 1e-300)
    errs = {k: rel(g[k], o[k]) for k in g}
    for k in ("rho", "u", "T"):
        assert errs[k] <= 1e-5, errs
    for k in ("sens", "fs", "gs"):
        assert errs[k] <= 1e-4, errs


@pytest.mark.parametrize("storage", ["fp32", "fp16"])
@pytest.mark.parametrize("solo_tiles", [0, 1], ids=["packed", "solo"])
def test_paper_heat_sink_in_the_batch_equals_single_context(storage, solo_tiles):
    """The paper's heat-sink problem (quarter domain with symmetry planes,
    pressure-driven inlet holding T, heat generation, J_Q) served in the
    batch beside other lattices, packed and solo: bit-identical to the
    single-context solve."""
    from paper_2501_02161_gb300.solver import Solver
    q = I.heat_sink_quarter(nx=32, ny=10, nz=8, re=20.0, beta_max=0.01, plenum=3, seed=3)
    lats = [q, I.pipe_bend_3d(n=24, width=6, re=20.0, seed=2)]
    got = solve_batched(lats, storage=storage, solo_tiles=solo_tiles)
    rep, sens, u = got[0]
    s = Solver.from_lattice(q, storage=storage)
    rf = s.forward(tol=1e-5, max_steps=20000, check_every=K)
    ra = s.adjoint(tol=1e-5, max_steps=20000, check_every=K)
    assert rep.status >= 0 and rep.steps == rf.steps + ra.steps
    assert torch.equal(s.sensitivity(dtype=torch.float64).cpu(), sens)
    assert torch.equal(s.fields(torch.float64)[1].cpu(), u)
    assert rep.J == rf.J
    s.close()
