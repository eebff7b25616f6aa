"""The oracle against its pins (CPU only)."""

import pytest

import oracle
import oracle_pins


@pytest.mark.parametrize("pin", oracle_pins.ALL_PINS, ids=lambda f: f.__name__)
def test_pin(pin):
    pin(oracle.Oracle())


def test_star_margin_report():
    """Records the objlim margin of the FWHM-2 star (script form below 1, article form above)."""
    rs, _ = oracle_pins.star_margin(oracle.Oracle(), 0)
    ra, _ = oracle_pins.star_margin(oracle.Oracle(), 1)
    print(f"star R max: script form {rs:.3f}, article form {ra:.3f} (objlim 1.0)")
    assert rs < 1.0 < ra
