"""The seeded synthetic input generators (shared by the oracle and the CUDA
path): named workload presets build the stated lattices."""
import pytest


def test_named_workloads_build_with_their_stated_shapes():
    """The named workload presets: shape, a valid flag field, gamma in [0, 1],
    an inlet and an outlet, and the temperature lattice where stated."""
    from paper_2501_02161_gb300 import inputs as I
    want = {"pipe_bend_2d_64x64": ((64, 64, 1), False), "pipe_bend_3d_64cubed": ((64, 64, 64), False),
            "heat_sink_128x64x32": ((128, 64, 32), True), "heat_sink_96x48x24": ((96, 48, 24), True)}
    assert set(want) == set(I.WORKLOADS)
    for name, (shape, thermal) in want.items():
        lat = I.workload(name)
        assert (lat.nx, lat.ny, lat.nz) == shape and lat.thermal == thermal, name
        kinds = lat.flags & 7
        assert kinds.max() <= 3 and (kinds == I.VEL).any() and (kinds == I.PRES).any(), name
        assert 0.0 <= lat.gamma.min() and lat.gamma.max() <= 1.0, name
    with pytest.raises(ValueError):
        I.workload("no such workload")

