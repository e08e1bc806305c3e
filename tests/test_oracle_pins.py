"""The oracle against the paper's examples, closed forms and invariants (CPU only)."""
import pytest

import oracle
import oracle_pins


@pytest.fixture(scope="module")
def o():
    return oracle.get()


@pytest.mark.parametrize("pin", oracle_pins.ALL_PINS, ids=lambda f: f.__name__)
def test_pin(o, pin):
    pin(o)


def test_invalid_arguments(o):
    import numpy as np
    J = np.zeros((4, 4))
    h = np.zeros(4)
    with pytest.raises(ValueError):
        o.low_spectrum(J, h, 17)          # S > 2^n
    with pytest.raises(ValueError):
        o.low_spectrum(J, h, 0)
    with pytest.raises(ValueError):
        o.low_spectrum(J, h, 2, fixed_bits=2, fixed_value=4)  # value does not fit
