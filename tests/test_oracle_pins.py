"""The CPU oracle against the paper's worked examples, brute force,
independent algorithms, invariants and the stream-format cases."""
import pytest

import oracle
import oracle_pins


@pytest.mark.parametrize("pin", oracle_pins.ALL_PINS, ids=lambda f: f.__name__)
def test_oracle_pin(pin):
    pin(oracle.load())
