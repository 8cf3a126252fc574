"""The CPU oracle against facts fixed by the paper's definitions and by
arithmetic (see oracle_pins.py for what each pin rests on)."""
import pytest

import oracle_pins as pins


@pytest.mark.parametrize("check", pins.ALL_PINS, ids=lambda f: f.__name__)
def test_oracle_pin(check):
    check()
