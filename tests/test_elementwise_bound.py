"""The element-wise parity check of the GPU tests (gpu_helpers.step_elementwise), on the
CPU: the oracle's own half-step passes it exactly, and a planted error in one entry
(10 % of its value, in an entry that matters for its column) fails it in the FP32 forms."""
import dataclasses

import numpy as np
import pytest

import pins
from gpu_helpers import step_elementwise
from oracle import dna as o


def _case(which):
    V, W, H = pins.rand_problem(30, 40, 5, 77)
    W, H = o.normalize_w_columns(W, H)
    W, H, _, _ = o.dna_iteration(V, W, H)
    half = (o.h_half_step if which == 0 else o.w_half_step)(V, W, H)
    W2, H2, _ = (o.dna_step_h if which == 0 else o.dna_step_w)(V, W, H, choice=half.choice)
    return half, W, H, W2, H2


@pytest.mark.parametrize("which", [0, 1])
@pytest.mark.parametrize("kind", ["f64", "f32", "f32t", "bf16"])
def test_exact_step_passes(which, kind):
    half, W, H, W2, H2 = _case(which)
    assert step_elementwise(half, which, W, H, W2, H2, kind) == 0.0


@pytest.mark.parametrize("which", [0, 1])
@pytest.mark.parametrize("kind", ["f64", "f32", "f32t"])
def test_planted_entry_error_fails(which, kind):
    half, W, H, W2, H2 = _case(which)
    X = (H2 if which == 0 else W2).copy()
    i = np.unravel_index(np.argmax(X), X.shape)     # the largest entry
    X[i] *= 1.1
    if which == 0:
        assert step_elementwise(half, 0, W, H, W2, X, kind) > 1.0
    else:
        assert step_elementwise(half, 1, W, H, X, H2, kind) > 1.0


def test_wrong_choice_fails():
    """Taking the other candidate for one column with a clear cost margin fails too."""
    half, W, H, W2, H2 = _case(0)
    t = int(np.argmax(half.margin))
    flipped = half.choice.copy()
    flipped[t] = not flipped[t]
    V, _, _ = pins.rand_problem(30, 40, 5, 77)
    _, Hf, _ = o.dna_step_h(V, W, H, choice=flipped)
    Wf = W2
    assert step_elementwise(dataclasses.replace(half), 0, W, H, Wf, Hf, "f32") > 1.0
