"""Plant one plausible mistake at a time in the oracle (on the CPU, through a
compile-time switch of its C source) and check that some pin catches it."""
import pytest

from tests import oracle_pins as pins


@pytest.mark.parametrize("mutant", [1, 2, 3, 4, 5])
def test_pins_catch_planted_mistake(mutant):
    failures = pins.run_all(mutant=mutant, fast=True)
    assert failures, f"mutant {mutant} passed every pin"
