"""Every planted oracle mistake must be caught by at least one pin.

Each mutant is the oracle rebuilt with -DORACLE_MUTANT=n, one plausible
mistake each: 1 insert overwrites an existing value, 2 heap free writes at the
wrong top, 3 a key coordinate is dropped, 4 quantisation truncates instead of
flooring, 5 rehash drops an entry, 6 erase leaks the freed index, 7 growth
adds one instead of doubling, 8 TSDF integration replaces the running mean
by the newest value, 9 ray casting returns the sample depth instead of the
interpolated crossing, 10 the double hash map stores the local index instead
of the global one, 11 unprojection adds the camera centre with the wrong
sign.
"""
import pytest

import oracle_pins as pins

MUTANTS = [1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11]


@pytest.mark.parametrize("mutant", MUTANTS)
def test_mutant_is_caught(mutant):
    caught = []
    for pin in pins.ALL_PINS:
        try:
            pin(mutant=mutant)
        except AssertionError as e:
            caught.append((pin.__name__, str(e)[:80]))
    assert caught, f"no pin caught oracle mutant {mutant}"
