"""Planted mistakes: each one is switched on inside the oracle (on the CPU) and one of
the pins must catch it, which shows the pins would catch that kind of error in the
oracle itself (a bound off by one bit, a dropped or extra bit, a wrong code cap, a
transposed operand, a wrong sign, a dropped term)."""
import json
import os

import numpy as np
import pytest

import oracle as O
from paper_1911_04034_gb300 import circuits as Cc

from test_oracle_codec import GOLDEN, _expected_image, np_truncate
from test_oracle_sim import full_unitary, random_gate


def sigbits_pin() -> bool:
    return [O.sig_bits(e) for e in (1e-1, 1e-2, 1e-3, 1e-4, 1e-5)] == [16, 19, 22, 26, 29]


def truncation_pin() -> bool:
    rng = np.random.default_rng(1)
    bits = rng.integers(1 << 60, 1 << 62, size=200, dtype=np.uint64)
    t = np.array([O.truncate(int(b), 26) for b in bits], dtype=np.uint64)
    return bool(np.array_equal(t, np_truncate(bits, 26)))


def golden_pin() -> bool:
    for case in json.load(open(GOLDEN))["cases"]:
        vals = np.array([int(v, 16) for v in case["values_hex"]], dtype=np.uint64)
        try:
            if O.encode_chunk(vals, case["kc"], case["S"], modes=case.get("modes", O.DEFAULT_MODES)) != _expected_image(case):
                return False
        except O.OracleError:
            return False
    return True


def unitary_pin() -> bool:
    n = 4
    rng = np.random.default_rng(4)
    gates = Cc.to_array([random_gate(rng, n) for _ in range(25)])
    psi0 = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
    ref = psi0.copy()
    for g in gates:
        ref = full_unitary(g, n) @ ref
    got = psi0.copy()
    O.sv_run(got, n, gates)
    return bool(np.max(np.abs(got - ref)) < 1e-13)


PINS = [sigbits_pin, truncation_pin, golden_pin, unitary_pin]


def test_pins_hold_without_mutant():
    O.set_mutant(0)
    assert all(p() for p in PINS)


@pytest.mark.parametrize("mutant", [1, 2, 3, 4, 5, 6])
def test_each_planted_mistake_is_caught(mutant):
    try:
        O.set_mutant(mutant)
        caught = [p.__name__ for p in PINS if not p()]
    finally:
        O.set_mutant(0)
    assert caught, f"planted mistake {mutant} passed every pin"
