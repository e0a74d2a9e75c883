"""Checkpoint / resume of a context's solver state (lbm_export_state /
lbm_import_state): a state moved to another context continues exactly as the
original would, bit for bit, through warm-started solves, the sensitivity and
the fields; mismatched contexts and short buffers are refused."""
import pytest

torch = pytest.importorskip("torch")

from paper_2501_02161_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2501_02161_gb300 import build as B
    B.build()


def _solver(lat, storage):
    from paper_2501_02161_gb300.solver import Solver
    return Solver.from_lattice(lat, storage=storage)


@pytest.mark.parametrize("storage", ["fp32", "fp16"])
def test_resumed_forward_is_bitwise_the_same(storage):
    lat = I.pipe_bend_3d(n=24, width=6, re=20.0, seed=2)
    a = _solver(lat, storage)
    a.forward(tol=0, max_steps=1000, check_every=500)
    state = a.export_state()
    ra = a.forward(tol=0, max_steps=1000, check_every=500, reset=False)
    b = _solver(lat, storage)
    b.import_state(state)
    rb = b.forward(tol=0, max_steps=1000, check_every=500, reset=False)
    assert ra.J == rb.J and ra.I == rb.I
    for x, y in zip(a.fields(torch.float64)[:2], b.fields(torch.float64)[:2]):
        assert torch.equal(x, y)
    a.close()
    b.close()


def test_resumed_thermal_adjoint_and_sensitivity_are_bitwise_the_same():
    lat = I.heat_sink(nx=32, ny=16, nz=12, re=20.0, q_flux=2e-3, seed=4)
    a = _solver(lat, "fp32")
    a.forward(tol=1e-6, max_steps=20000, check_every=500)
    a.adjoint(tol=0, max_steps=600, check_every=200)
    mid = a.export_state()
    a.adjoint(tol=0, max_steps=600, check_every=200, reset=False)
    done = a.export_state(torch.empty(a.state_bytes(), dtype=torch.uint8, device="cuda"))
    sa = a.sensitivity(dtype=torch.float64)
    b = _solver(lat, "fp32")
    b.import_state(mid)
    b.adjoint(tol=0, max_steps=600, check_every=200, reset=False)
    assert torch.equal(b.sensitivity(dtype=torch.float64), sa)
    c = _solver(lat, "fp32")
    c.import_state(done)  # a completed solve: the sensitivity needs no further steps
    assert torch.equal(c.sensitivity(dtype=torch.float64), sa)
    assert torch.equal(c.fields(torch.float64)[2], a.fields(torch.float64)[2])
    for s in (a, b, c):
        s.close()


def test_import_refuses_other_lattices_and_short_buffers():
    from paper_2501_02161_gb300._capi import LBMError
    a = _solver(I.pipe_bend_3d(n=24, width=6, re=20.0, seed=2), "fp32")
    a.forward(tol=0, max_steps=200, check_every=200)
    st = a.export_state()
    other = _solver(I.pipe_bend_3d(n=32, width=8, re=20.0, seed=2), "fp32")
    with pytest.raises(LBMError, match="another lattice"):
        other.import_state(st)
    same = _solver(I.pipe_bend_3d(n=24, width=6, re=20.0, seed=2), "fp32")
    with pytest.raises(LBMError, match="smaller"):
        same.import_state(st[: st.numel() // 2])
    with pytest.raises(LBMError, match="not a state"):
        same.import_state(torch.zeros_like(st))
    for s in (a, other, same):
        s.close()
