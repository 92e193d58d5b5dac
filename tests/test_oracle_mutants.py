"""Planted mistakes in the oracle (built on the CPU with -DORACLE_MUTANT=k):
each one must make at least one pin fail, so the pins can see that kind of
mistake.  Mutants: 1 natural instead of bit-reversed order in the definition,
2 swapped operands of the subtraction in Algorithm 1, 3 twiddle zeta^(k+1)
instead of zeta^k, 4 inverse run with omega instead of omega^-1, 5 an index
error in the schoolbook product, 6 the batched forms stepping by L instead of
the stride."""
import pytest

import oracle
from tests import oracle_pins


@pytest.mark.parametrize("mutant", [1, 2, 3, 4, 5, 6])
def test_mutant_is_caught(mutant):
    o = oracle.Oracle(mutant)
    caught = []
    for pin in oracle_pins.ALL_PINS:
        try:
            pin(o)
        except AssertionError:
            caught.append(pin.__name__)
    assert caught, f"planted mistake {mutant} passed every pin"
