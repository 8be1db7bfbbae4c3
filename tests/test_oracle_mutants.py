"""Plant plausible mistakes in copies of the oracle (built on the CPU with a
mutation define) and check that the pin suite rejects every one of them:
    1  g(j+k) instead of g(j-k) in Eq. 1
    2  w^(-ut) instead of w^(ut) in Eq. 2
    3  the 1/N of Eq. 3 dropped
    4  w^(ut) instead of w^(-ut) in Eq. 3
    5  the last term of the sum in Eq. 1 dropped
    6  g(j+k) instead of g(j-k) in the exact integer convolution
    7  the modulus-free transform not truncated to alpha bits
    8  the sampled Eq. 1 evaluated at the list position instead of the listed index
    9  the sampled Eq. 1 evaluated one output index too far
"""
import os

import pytest

import oracle
import oracle_pins as P
import test_oracle_exact_modfree as X


@pytest.mark.parametrize("mutant", [1, 2, 3, 4, 5])
def test_mutant_is_caught(tmp_path, mutant):
    so = oracle.build(out=os.path.join(tmp_path, f"mut{mutant}.so"), defines={"ORACLE_MUTANT": mutant})
    o = oracle.Oracle(oracle.load(so))
    fast = [P.pin_hand_example, P.pin_impulses, P.pin_roundtrip_linear,
            P.pin_conv_closed_forms, P.pin_theorem]
    failed = P.run_pins(o, fast)
    assert failed, f"mutant {mutant} passed every pin"


@pytest.mark.parametrize("mutant", [6, 7])
def test_exact_and_modulus_free_mutant_is_caught(tmp_path, mutant):
    so = oracle.build(out=os.path.join(tmp_path, f"mut{mutant}.so"), defines={"ORACLE_MUTANT": mutant})
    o = oracle.Oracle(oracle.load(so))
    pins = [X.test_int_conv_brute_force, X.test_int_conv_library_linear_convolution,
            X.test_int_conv_closed_forms, X.test_dyadic_ntt_brute_force, X.test_dyadic_conv_brute_force]
    failed = 0
    for pin in pins:
        try:
            pin(o)
        except AssertionError:
            failed += 1
    assert failed, f"mutant {mutant} passed every pin"


@pytest.mark.parametrize("mutant", [8, 9])
def test_sampler_mutant_is_caught(tmp_path, mutant):
    so = oracle.build(out=os.path.join(tmp_path, f"mut{mutant}.so"), defines={"ORACLE_MUTANT": mutant})
    o = oracle.Oracle(oracle.load(so))
    assert P.run_pins(o, [P.pin_conv_sample]), f"mutant {mutant} passed the sampler pin"
    # the mutation touches the sampler only: the full convolution pins still pass
    assert P.run_pins(o, [P.pin_hand_example, P.pin_conv_closed_forms]) == []


def test_real_oracle_passes_fast_subset(orc):
    assert P.run_pins(orc, [P.pin_hand_example, P.pin_impulses]) == []
