"""The CPU oracle pinned to the paper and to mathematics (no GPU needed)."""
import pytest

import oracle
import oracle_pins as pins


@pytest.fixture(scope="module")
def o():
    return oracle.default()


@pytest.mark.parametrize("check", pins.ALL_CHECKS, ids=lambda c: c.__name__)
def test_oracle_pin(o, check):
    check(o)
