"""The pins must catch plausible mistakes in the oracle.

Each case compiles a copy of the oracle with one planted mistake (a flipped
sign, a dropped factor, a transposed Jacobian, a reversed adjoint stream, a
wrong derivative) and runs a set of pins against it; at least one must fail.
Only the oracle is mutated, on the CPU.
"""
import os

import pytest

import test_oracle_continuous as CA
import test_oracle_heatgen as H
import test_oracle_pins as T
import test_oracle_symmetry as SY
from paper_2501_02161_gb300 import inputs as I

MUTATIONS = {
    1: "Zou-He tangential correction with the wrong sign",
    2: "boundary Jacobian without the 1/2 of the tangential term",
    3: "adjoint collision with C instead of C^T",
    4: "adjoint streaming in the forward direction",
    5: "Eq. 12 collision Jacobian with gamma instead of gamma^2",
    6: "fixed-density outlet Jacobian with 3 w instead of 6 w",
    7: "adjoint objective source with the wrong sign",
    8: "thermal-to-flow coupling with the wrong sign",
    9: "heat-generation objective source with the wrong sign",
    10: "continuous adjoint boundaries with the printed bottom-outlet / left-inlet indices on every face",
    11: "symmetry plane that moves the image node but does not reflect the population",
}


def pins(O):
    lat2 = I.pipe_bend_2d(nx=12, ny=12, width=4, tau=0.8, gamma_value=0.6)
    lat3 = I.pipe_bend_3d(n=8, width=2, re=2.0, seed=3)
    yield lambda: T.test_inlet_matches_eq7_values(O)
    yield lambda: T.test_inlet_jacobian_is_eq58(O)
    yield lambda: T.test_adjoint_inlet_is_eq59(O)
    yield lambda: T.test_adjoint_outlet_is_eq60(O)
    yield lambda: T.test_zou_he_moments_every_face(O, 1, I.VEL)
    yield lambda: T.test_zou_he_moments_every_face(O, 1, I.PRES)
    yield lambda: T.test_collision_jacobian_exact_central_difference(O, 1, 0)
    yield lambda: T.test_tangent_equals_central_difference_of_step(O, lat3)
    yield lambda: T.test_dot_product_adjoint_of_step(O, lat2)
    yield lambda: T.test_thermal_tangent_and_dot_product(O)
    yield lambda: T.test_sensitivity_vs_finite_difference_2d(O, I.GAMMA_EQ12)
    yield lambda: H.test_sensitivity_with_heat_generation_vs_finite_difference(O)
    yield lambda: CA.test_boundary_term_of_eq25_vanishes_on_every_face(O, (0, -1, 0), I.PRES)
    yield lambda: SY.test_quarter_equals_the_unfolded_full_domain(O, "qgen")


@pytest.mark.parametrize("k", sorted(MUTATIONS), ids=lambda k: MUTATIONS[k])
def test_pins_catch_planted_mistake(oracle_mod, tmp_path, k):
    O = oracle_mod
    path = O.build(target=str(tmp_path / f"liblbm_oracle_m{k}.so"), mutation=k)
    O.use_library(path)
    caught = []
    try:
        for check in pins(O):
            try:
                check()
            except AssertionError:
                caught.append(check)
                break
    finally:
        O.use_library(None)
    assert caught, f"no pin caught mutation {k}: {MUTATIONS[k]}"
