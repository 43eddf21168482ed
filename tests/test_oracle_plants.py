"""Every planted mistake in the oracle is caught by at least one pin."""

import pytest

import oracle
import pins

PLANTS = {
    1: "two-product drops its rounding error",
    2: "inner product does not conjugate",
    3: "back substitution reads R transposed",
    4: "square root without Newton refinement",
    5: "division keeps one quotient digit",
    6: "update adds r_kj q_k instead of subtracting",
    7: "rounding never fills the last limb",
    8: "column norm drops the imaginary part",
    9: "adjoint product A^H v does not conjugate A in the real part",
    10: "matrix-vector product flips the sign of the imaginary cross term",
}


@pytest.mark.parametrize("plant", sorted(PLANTS))
def test_plant_is_caught(plant, tmp_path):
    path = oracle.build(plant=plant, out=str(tmp_path / f"liboracle_plant{plant}.so"))
    o = oracle.Oracle(path)
    assert o.plant() == plant
    with pytest.raises(AssertionError):
        pins.quick_battery(o)


def test_unplanted_passes_quick_battery(orc):
    pins.quick_battery(orc)
