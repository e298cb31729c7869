"""The FP64 oracle against what the paper and the mathematics fix (CPU only)."""
import pytest

import pins


@pytest.mark.parametrize("check", pins.ALL, ids=lambda f: f.__name__)
def test_pin(check):
    check()


def test_a_b_with_lambda():
    pins.check_a_b_finite_differences(lam=0.3)


def test_w_a_b_with_rho():
    pins.check_w_a_b_finite_differences(rho=0.2)


def test_transpose_symmetry_regularised():
    pins.check_transpose_symmetry(reg=0.15)
