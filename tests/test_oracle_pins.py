"""The oracle against the paper's printed values, closed forms and brute force."""
import pytest

import oracle_pins as P

pytestmark = pytest.mark.timeout(600) if hasattr(pytest.mark, "timeout") else []


@pytest.mark.parametrize("pin", P.PINS, ids=lambda f: f.__name__)
def test_pin(orc, pin):
    pin(orc)
