"""The FP64 oracle against closed forms, identities, brute force and invariants (no GPU)."""
import pytest

from oracle import ftcg_oracle as O
from tests.oracle_pins import PINS


@pytest.mark.parametrize("pin", PINS, ids=[p.__name__ for p in PINS])
def test_pin(pin):
    ok, detail = pin(O)
    assert ok, detail
