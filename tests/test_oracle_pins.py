"""The CPU oracle against what the paper and mathematics fix (no GPU)."""
import pytest

import oracle
import pins


@pytest.fixture(scope="module")
def orc():
    return oracle.get()


@pytest.mark.parametrize("pin", pins.PINS, ids=[p.__name__ for p in pins.PINS])
def test_pin(orc, pin):
    pin(orc)


def test_hand_cases_are_well_formed():
    from paper_1801_09809_gb300 import gen  # noqa: F401
    cases = pins.load_hand_cases()
    assert len(cases) >= 5
    for c in cases:
        assert "cite" in c and len(c["mate"]) == c["n"] == len(c["expect_mate"])
