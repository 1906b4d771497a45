"""The arithmetic forms of the streaming kernel against the kept-term chains the oracle
defines (each output part: terms with a zero coefficient left out, the first kept term
one rounded product, each later one a fused multiply-add), checked on the host in
float64 with an exact fused multiply-add (no GPU): the equalities the kernel relies on."""
from fractions import Fraction

import numpy as np


def truncate_hi(x: np.ndarray, S: int) -> np.ndarray:
    """Keep the top S bits of each binary64 value (S <= 32: the low word is cut)."""
    u = np.ascontiguousarray(x).view(np.uint64)
    mask = np.uint64(((1 << S) - 1) << (64 - S))
    return (u & mask).view(np.float64)


def fma(a: float, b: float, c: float) -> float:
    """a * b + c rounded once (exact rational arithmetic, then one correct rounding)."""
    return float(Fraction(a) * Fraction(b) + Fraction(c))


def kept_chain(coefs, xs) -> float:
    acc, have = 0.0, False
    for c, x in zip(coefs, xs):
        if c == 0.0:
            continue
        acc = fma(c, x, acc) if have else c * x
        have = True
    return acc


def all_terms_chain(coefs, xs) -> float:
    """The dense form: every term, zero coefficients included."""
    acc = coefs[0] * xs[0]
    for c, x in zip(coefs[1:], xs[1:]):
        acc = fma(c, x, acc)
    return acc


def bits(v: float) -> int:
    return int(np.float64(v + 0.0).view(np.uint64))  # + 0.0 stores a zero as +0, as the encoder does


def test_dense_and_real_forms_equal_the_kept_chain():
    """Adding the terms of zero coefficients (the dense form) or leaving them out (the real
    form) gives the kept chain's value: a zero coefficient adds an exact zero."""
    rng = np.random.default_rng(7)
    rows = [(0.7071067811865476, 0.0, -0.7071067811865476, 0.0),     # a real row (H)
            (0.9238795325112867, -0.0, 0.0, 0.3826834323650898),     # RX-like: two kept terms
            (0.5, -0.5, 0.5, 0.5), (0.0, 0.0, 0.8, -0.6)]
    for _ in range(400):
        xs = [float(truncate_hi(np.array([rng.standard_normal() * 2.0 ** rng.integers(-30, 2)]), 26)[0])
              for _ in range(4)]
        for c in rows:
            assert bits(all_terms_chain(c, xs)) == bits(kept_chain(c, xs))


def test_power_of_two_chain_is_the_scaled_signed_chain():
    """Coefficient parts +-1/2 (sqrt(X), sqrt(Y)): the kept chain equals 1/2 times the chain
    of the signed inputs in the same order, bit for bit (zeros stored as +0)."""
    rng = np.random.default_rng(11)
    for S in (19, 22, 26, 29, 32):
        x = [truncate_hi(rng.standard_normal(400) * 2.0 ** rng.integers(-40, 2, 400), S) for _ in range(4)]
        for signs in ((1, -1, 1, 1), (1, 1, 1, -1), (-1, -1, 1, 1), (1, 1, -1, -1)):
            for i in range(400):
                xs = [float(v[i]) for v in x]
                want = kept_chain([0.5 * s for s in signs], xs)
                signed = ((signs[0] * xs[0] + signs[1] * xs[1]) + signs[2] * xs[2]) + signs[3] * xs[3]
                assert bits(0.5 * signed) == bits(want)


def test_power_of_two_identity_holds_below_the_kernel_floor():
    """Inputs truncated to at most 32 bits near the bottom of the normal range (exponents
    -1022..-960): the identity still holds wherever the output is normal, so the kernel's
    check (inputs of at least 2^-959) is conservative."""
    rng = np.random.default_rng(3)
    n = 300
    x = [truncate_hi(np.ldexp(rng.uniform(1, 2, n) * rng.choice([-1.0, 1.0], n), rng.integers(-1022, -960, n)), 26)
         for _ in range(4)]
    checked = 0
    for i in range(n):
        xs = [float(v[i]) for v in x]
        for signs in ((1, -1, 1, 1), (-1, 1, 1, -1)):
            want = kept_chain([0.5 * s for s in signs], xs)
            if abs(want) < np.ldexp(1.0, -1022):
                continue  # a subnormal output goes to the general kernel either way
            signed = ((signs[0] * xs[0] + signs[1] * xs[1]) + signs[2] * xs[2]) + signs[3] * xs[3]
            assert bits(0.5 * signed) == bits(want)
            checked += 1
    assert checked > n
