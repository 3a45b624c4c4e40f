"""Each pin set must reject a plausible slip planted in the oracle (CPU only).

`oracle.mutant(k)` swaps in a build of the same C source compiled with
ORACLE_MUTANT = k, which plants exactly one mistake: a stored-index map off by
one, a dropped c(kt) weight, a wrong sign of the t exponent, a missing 1/N, a
transposed bypass weight, a conjugate dropped in the weight gradient, a
GELU derivative missing its second term, a bias dropped in the pointwise
encoder/decoder layer, a loss gradient missing its factor 2, or the pointwise
layer's GELU derivative taken at GELU(A) instead of A, or Adam's second moment
fed g instead of g^2.  For every mutant at
least one pin of tests/test_oracle_pins.py or tests/test_oracle_stack_pins.py
must fail; the unmutated oracle passes them all.
"""
import pytest

import oracle
import test_oracle_pins as pins
import test_oracle_stack_pins as spins

PINS = {
    "rfftn corners": lambda: pins.test_spectrum_equals_numpy_rfftn_kept_corners(pins.TINY[1]),
    "irfftn padded": lambda: pins.test_synthesis_equals_numpy_irfftn_of_zero_padded(pins.TINY[1]),
    "identity": pins.test_identity_with_all_modes_kept,
    "plane waves": pins.test_plane_wave_closed_forms,
    "adjoint dot products": lambda: pins.test_spectral_adjoint_dot_products(pins.TINY[0]),
    "finite differences": pins.test_block_gradient_central_finite_differences,
    "linear+gelu special case": pins.test_zero_spectral_weight_reduces_to_torch_linear_gelu,
    "gelu values": pins.test_gelu_textbook_values,
    "pointwise vs torch": lambda: spins.test_pointwise_forward_equals_torch_linear_and_gelu(1),
    "pointwise grad vs torch": lambda: spins.test_pointwise_gradient_equals_torch_autograd(1),
    "mse vs torch": spins.test_mse_equals_torch_mse_loss_and_its_gradient,
    "stack finite differences": spins.test_stack_gradient_central_finite_differences,
    "adam vs torch": spins.test_adam_matches_torch_optim_adam,
}

MUTANTS = {
    1: "stored-index map off by one",
    2: "dropped c(kt)",
    3: "wrong sign of the t exponent",
    4: "missing 1/N in the synthesis",
    5: "transposed W_l in the forward",
    6: "conjugate dropped in dW",
    7: "GELU' without its second term",
    8: "bias dropped in the pointwise layer",
    9: "loss gradient without its factor 2",
    10: "pointwise GELU' taken at GELU(A)",
    11: "Adam's second moment fed g instead of g^2",
}


def _failing_pins():
    failed = []
    for name, fn in PINS.items():
        try:
            fn()
        except AssertionError:
            failed.append(name)
    return failed


def test_unmutated_oracle_passes_every_pin():
    assert _failing_pins() == []


@pytest.mark.parametrize("k", sorted(MUTANTS), ids=[MUTANTS[k] for k in sorted(MUTANTS)])
def test_planted_slip_fails_some_pin(k):
    with oracle.mutant(k):
        failed = _failing_pins()
    print(MUTANTS[k], "->", failed)
    assert failed, f"no pin caught mutant {k} ({MUTANTS[k]})"
