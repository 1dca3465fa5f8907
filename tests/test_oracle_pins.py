"""The FP64 oracle against its pins (CPU only)."""
import pytest

from oracle_pins import PINS


@pytest.mark.parametrize("name", sorted(PINS))
def test_pin(orc, name):
    PINS[name](orc)
