"""GB300-native discrete adjoint lattice Boltzmann solver (arXiv 2501.02161).

The solver lives in the CUDA library liblbmadj.so (C-ABI: include/lbmadj.h);
`Solver` is its Python face.  Submodules load lazily so that the seeded input
generators (`inputs`) import without the library.
"""
__all__ = ["Solver", "inputs"]


def __getattr__(name):
    if name == "Solver":
        from .solver import Solver
        return Solver
    raise AttributeError(name)
