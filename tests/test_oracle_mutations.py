"""Planted mistakes in the oracle (on the CPU) must each be caught by at least one pin.

The oracle has a test-only switch that introduces one plausible mistake at a time: a dropped
mass term, a transposed Jacobian inverse, a signed determinant, two swapped local nodes, a
dropped Duffy factor in the quadrature, a Dirichlet lift with the wrong sign, boundary columns
left in place, a CG search direction built from the unpreconditioned residual, a CG step length
from r.r instead of r.z, a wave p update with the wrong sign, full phi steps instead of halves,
and three in the per-entry error scale that every parity test uses as its tolerance (the
absolute-term sums multiplied by the point count, the Cauchy-Schwarz floor taken from one
diagonal twice, signed coefficient terms in the linear form's scale).  Each must make some pin
fail; otherwise the pins would not be strong enough to trust the oracle.  (Signed terms in the
bilinear forms' off-diagonal sums, mistake 14, provably change no scale; the scale tests show
that instead.)
"""
import pytest

import oracle as O
from tests import test_oracle_pins as P
from tests import test_oracle_scale as SC
from tests import test_oracle_solve as S
from tests import test_oracle_wave as W

PINS = [
    ("reference_elements", lambda: P.pin_reference_elements()),
    ("p1_interior_row", lambda: P.pin_p1_interior_row(16)),
    ("mass_sum_3d", lambda: P.pin_mass_sum_and_stiffness_rows(3, 2, 2, 0.2)),
    ("poly_repro_2d_p2", lambda: P.pin_polynomial_reproduction(2, 2, 4, 0.2)),
    ("poly_repro_3d_p2", lambda: P.pin_polynomial_reproduction(3, 2, 2, 0.2)),
    ("exact_rational_3d_p2", lambda: P.pin_exact_rational(3, 2, 1)),
    ("quadrature_2d", lambda: P.pin_quadrature_monomials(2, 4)),
    ("reduced_system", lambda: S.pin_reduced_system()),
    ("harmonic_p2", lambda: S.pin_harmonic_reproduction(2)),
    ("cg_dense_spd", lambda: S.pin_cg_dense_spd()),
    ("cg_diagonal", lambda: S.pin_cg_diagonal()),
    ("wave_modes", lambda: W.pin_modes()),
    ("scale_reference_triangle", lambda: SC.pin_scale_reference_triangle()),
    ("scale_element_3d_p2", lambda: SC.pin_scale_element(3, 2, cells=1)),
    ("scale_vector_p1", lambda: SC.pin_scale_vector_p1(2)),
]


@pytest.mark.parametrize("code,what", [(1, "drop mass term"), (2, "transposed J^-1"), (3, "signed detJ"),
                                       (4, "swapped edge nodes"), (5, "dropped Duffy factor"),
                                       (6, "Dirichlet lift with the wrong sign"),
                                       (7, "boundary columns kept"), (8, "CG direction from r, not z"),
                                       (9, "CG step length from r.r"),
                                       (10, "wave: p update with the wrong sign"),
                                       (11, "wave: full phi steps instead of halves"),
                                       (12, "error scale times the point count"),
                                       (13, "Cauchy-Schwarz floor from one diagonal twice"),
                                       (15, "linear-form scale from signed terms")])
def test_planted_mistake_is_caught(code, what):
    O.set_mutation(code)
    caught = []
    try:
        for name, pin in PINS:
            try:
                pin()
            except AssertionError:
                caught.append(name)
    finally:
        O.set_mutation(0)
    assert caught, f"planted mistake '{what}' passed every pin"


def test_pins_pass_without_mistake():
    for name, pin in PINS:
        pin()
