"""Each plausible mistake planted in the oracle (compiled with ORACLE_MUTANT=k)
must fail at least one pin: the pins are strong enough to catch a dropped row,
swapped MIN/MAX, equal keys not combined across runs, unsigned key order, a
dropped first count, a 32-bit SUM accumulator, a dropped final table, and a
wrong MIN identity."""
import pytest

import _pins
import oracle as oracle_mod

MUTANTS = {
    1: "last row dropped",
    2: "MIN and MAX swapped",
    3: "equal keys of different runs not combined",
    4: "unsigned key order",
    5: "first row of a group not counted",
    6: "32-bit SUM accumulator",
    7: "final in-memory table dropped",
    8: "MIN starts from 0",
}


@pytest.mark.parametrize("k", sorted(MUTANTS), ids=lambda k: MUTANTS[k].replace(" ", "_"))
def test_mutant_is_caught(k):
    m = oracle_mod.mutant(k)
    failed = []
    for pin in _pins.ALL_PINS:
        try:
            pin(m)
        except AssertionError:
            failed.append(pin.__name__)
    assert failed, f"mutant {k} ({MUTANTS[k]}) passed every pin"
