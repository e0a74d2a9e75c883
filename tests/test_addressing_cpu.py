"""The kernels' pull addressing, run on the host (lbm_check_addressing).

Every global-memory read of a population goes to node n + offset, with the
offset built from the six per-node neighbour offsets (periodic wrap folded in).
The library runs that same code on the CPU over every node and direction and
counts sources that differ from a plain modular wrap of x -/+ e_i or leave the
lattice: zero on every shape here, including one-node-wide and ragged ones.
"""
import ctypes

import pytest

from paper_2501_02161_gb300 import _capi as C


@pytest.fixture(scope="module", autouse=True)
def library():
    from paper_2501_02161_gb300 import build as B
    B.build()


def mismatches(stencil, nx, ny, nz):
    bad = ctypes.c_longlong(-1)
    C.check(C.lib().lbm_check_addressing(stencil, nx, ny, nz, ctypes.byref(bad)), "lbm_check_addressing")
    return bad.value


@pytest.mark.parametrize("shape", [(1, 1, 1), (2, 2, 2), (1, 5, 3), (7, 1, 1), (3, 2, 1), (33, 17, 9),
                                   (64, 64, 64), (96, 48, 24), (129, 3, 2)])
@pytest.mark.parametrize("stencil", [1, 2], ids=["D3Q19", "D3Q7"])
def test_3d_pull_sources_are_the_periodic_neighbours(stencil, shape):
    assert mismatches(stencil, *shape) == 0


@pytest.mark.parametrize("shape", [(1, 1), (64, 64), (37, 29), (5, 1), (1, 7)])
def test_2d_pull_sources_are_the_periodic_neighbours(shape):
    assert mismatches(0, shape[0], shape[1], 1) == 0


def test_bad_arguments_are_refused():
    bad = ctypes.c_longlong()
    L = C.lib()
    assert L.lbm_check_addressing(1, 0, 4, 4, ctypes.byref(bad)) == C.LBM_ERR_ARG
    assert L.lbm_check_addressing(5, 4, 4, 4, ctypes.byref(bad)) == C.LBM_ERR_ARG
    assert L.lbm_check_addressing(1, 512, 512, 512, ctypes.byref(bad)) == C.LBM_ERR_ARG
    assert L.lbm_check_addressing(1, 4, 4, 4, None) == C.LBM_ERR_ARG
