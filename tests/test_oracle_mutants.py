"""Each planted mistake in a copy of the oracle must fail at least one pin.

This shows the pins are sensitive to the plausible errors they guard
against: a dropped field term, a flipped sign, the wrong triangle of J, the
diagonal included, reversed or inverted bit encoding, reversed tie order, a
lost record, a wrong gradient factor, single-precision accumulation and, for the
QUBO form, the diagonal or the lower triangle of a read, and for the Potts model an
inverted pair indicator or a transposed field table.
"""
import pytest

import oracle
import oracle_pins

PLANTS = {
    1: "field term dropped",
    2: "pair term sign flipped",
    3: "lower triangle of J read",
    4: "diagonal of J included",
    5: "bit order reversed",
    6: "spin mapping inverted",
    7: "ties ordered by descending c",
    8: "first record lost in selection",
    9: "gradient uses s_i instead of s_i s_j",
    10: "energy accumulated in single precision",
    11: "QUBO pair sum includes the diagonal",
    12: "QUBO pairs read from the lower triangle",
    13: "Potts pair term counts unequal states",
    14: "Potts field table transposed",
}


@pytest.mark.parametrize("plant", sorted(PLANTS), ids=lambda k: PLANTS[k].replace(" ", "_"))
def test_plant_is_caught(plant):
    lib = oracle.Oracle(oracle.build(plant=plant))
    assert lib.lib.oracle_plant() == plant
    failed = []
    for pin in oracle_pins.ALL_PINS:
        try:
            pin(lib)
        except (AssertionError, ValueError):
            failed.append(pin.__name__)
    assert failed, f"plant {plant} ({PLANTS[plant]}) passed every pin"
