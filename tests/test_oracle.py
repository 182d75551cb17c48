"""The FP64 oracle against its pins (see tests/oracle_pins.py)."""
import pytest

from tests import oracle_pins


@pytest.mark.parametrize("pin", oracle_pins.ALL, ids=lambda f: f.__name__)
def test_oracle_pin(pin):
    pin()
