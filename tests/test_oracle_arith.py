"""Pins of the oracle's DD/QD arithmetic against exact rationals (CPU only)."""

import pytest

import pins


def test_selfcheck(orc):
    assert orc.selfcheck()
    assert orc.plant() == 0


def test_error_free_transforms(orc):
    pins.pin_error_free_transforms(orc)


@pytest.mark.parametrize("L", [1, 2, 4, 8])
def test_real_ops(orc, L):
    pins.pin_real_ops(orc, L)


@pytest.mark.parametrize("L", [1, 2, 4, 8])
def test_complex_ops(orc, L):
    pins.pin_complex_ops(orc, L)
