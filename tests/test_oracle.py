"""The CPU oracle against its pins (brute force, golden trace, invariants,
closed forms, library reductions).  See tests/oracle_pins.py."""
import pytest

import oracle_pins as pins


@pytest.mark.parametrize("pin", pins.ALL_PINS, ids=lambda f: f.__name__)
def test_oracle_pin(pin):
    pin(mutant=0)
