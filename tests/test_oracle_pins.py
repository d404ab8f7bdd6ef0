"""The FP64 oracle against what the paper and the mathematics fix (CPU only).

Each check is documented in ``pins.py`` with the passage it follows."""
import pytest

from . import pins


@pytest.mark.parametrize("check", pins.FAST_CHECKS, ids=lambda f: f.__name__)
def test_pin(check):
    check()


@pytest.mark.parametrize("check", pins.LATTICE_CHECKS, ids=lambda f: f.__name__)
def test_lattice_pin(check):
    check()
