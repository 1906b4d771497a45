"""Pins of the oracle's codec against facts that do not come from the oracle.

Section 4.2 (Solution C): bit-plane truncation to Sig_Bit_Count = 12 - EXP(eps) bits
(Eq. sigbits), XOR leading-zero coding with a 2-bit code; Section 3.7: the decoded
value lies in (|D(1 - delta)|, |D|]; Section 4.2 worked example (3.9921875 -> 3.96875).
"""
import json
import math
import os

import numpy as np
import pytest

import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "codec_hand_streams.json")
LEVELS = [1e-1, 1e-2, 1e-3, 1e-4, 1e-5]


def np_truncate(bits: np.ndarray, S: int) -> np.ndarray:
    """Independent numpy restatement used only to check the oracle: keep the S
    leading bits, store -0 as +0."""
    bits = bits.astype(np.uint64)
    if S < 64:
        mask = np.uint64((0xFFFFFFFFFFFFFFFF << (64 - S)) & 0xFFFFFFFFFFFFFFFF)
        bits = bits & mask
    bits = np.where(bits == np.uint64(0x8000000000000000), np.uint64(0), bits)
    return bits


# ----------------------------------------------------------- Eq. sigbits --- #

def test_exp_of_paper_example():
    # Section 4.2: "EXP(0.01) = -7"
    assert O.exp_of(0.01) == -7


@pytest.mark.parametrize("eps", LEVELS)
def test_sig_bits_matches_frexp(eps):
    # frexp gives eps = f 2^e with f in [0.5, 1): the IEEE exponent is e - 1.
    f, e = math.frexp(eps)
    assert 0.5 <= f < 1.0
    assert O.exp_of(eps) == e - 1
    assert O.sig_bits(eps) == 12 - (e - 1)


def test_sig_bits_table_and_lossless():
    # 12 sign+exponent bits for binary64 (Eq. sigbits): S = 16, 19, 22, 26, 29.
    assert [O.sig_bits(e) for e in LEVELS] == [16, 19, 22, 26, 29]
    assert O.sig_bits(0.0) == 64
    for bad in (1.0, 2.0, -1e-3, float("nan"), float("inf"), 1e-300):
        assert O.sig_bits(bad) < 0


def test_worked_example_float32():
    # Section 4.2: 3.9921875 kept to 15 leading bits -> 3.96875, relative error 0.005871.
    # Read in float32 (9 sign+exponent bits): 15 bits = 6 mantissa bits.  numpy only:
    f = np.array([3.9921875], dtype=np.float32).view(np.uint32)
    t = (f & np.uint32(0xFFFFFFFF << (32 - 15) & 0xFFFFFFFF)).view(np.float32)[0]
    assert float(t) == 3.96875
    assert round((3.9921875 - 3.96875) / 3.9921875, 6) == 0.005871


def test_worked_example_oracle():
    # The same value in binary64 keeps the same 6 mantissa bits with S = 12 + 6.
    t6 = O.truncate_double(3.9921875, 12 + 6)
    assert t6 == 3.96875
    assert round((3.9921875 - t6) / 3.9921875, 6) == 0.005871
    # Eq. sigbits itself gives S = 12 - EXP(0.01) = 19 (7 mantissa bits): within the bound.
    t7 = O.truncate_double(3.9921875, O.sig_bits(0.01))
    assert t7 == 3.984375
    assert (3.9921875 - t7) / 3.9921875 < 0.01


# --------------------------------------------------- truncation interval --- #

def _random_doubles(rng, n):
    mant = rng.integers(0, 1 << 52, size=n, dtype=np.uint64)
    expo = rng.integers(1, 2047, size=n).astype(np.uint64)
    sign = rng.integers(0, 2, size=n).astype(np.uint64)
    return (sign << np.uint64(63)) | (expo << np.uint64(52)) | mant


@pytest.mark.parametrize("eps", LEVELS)
def test_truncation_interval(eps):
    rng = np.random.default_rng(7)
    S = O.sig_bits(eps)
    bits = _random_doubles(rng, 4000)
    edge = np.array([0x0010000000000000, 0x7FEFFFFFFFFFFFFF, 0x3FFFFFFFFFFFFFFF, 0x3FF0000000000000,
                     0xBFF0000000000001], dtype=np.uint64)
    bits = np.concatenate([bits, edge])
    t = np.array([O.truncate(int(b), S) for b in bits], dtype=np.uint64)
    assert np.array_equal(t, np_truncate(bits, S))
    x = bits.view(np.float64)
    tv = t.view(np.float64)
    assert np.all(np.signbit(x) == np.signbit(tv))
    assert np.all(np.abs(tv) <= np.abs(x))
    # |x - t| < 2^(12-S) |x| <= eps |x|   (Section 3.7: D' in (|D(1-delta)|, |D|])
    rel = np.abs(x - tv) / np.abs(x)
    assert np.all(rel < 2.0 ** (12 - S))
    assert np.all(rel < eps)


def test_truncation_float32_sweep():
    # every float32 exponent with random and extreme mantissas, widened to binary64
    rng = np.random.default_rng(3)
    exps = np.arange(1, 255, dtype=np.uint32)
    mant = np.concatenate([rng.integers(0, 1 << 23, size=(254, 6), dtype=np.uint32),
                           np.full((254, 1), (1 << 23) - 1, dtype=np.uint32),
                           np.zeros((254, 1), dtype=np.uint32)], axis=1)
    f32 = ((exps[:, None] << np.uint32(23)) | mant).ravel().view(np.float32)
    x = f32.astype(np.float64)
    for eps in LEVELS:
        S = O.sig_bits(eps)
        t = np.array([O.truncate(int(b), S) for b in x.view(np.uint64)], dtype=np.uint64).view(np.float64)
        rel = np.abs(x - t) / np.abs(x)
        assert np.all(rel < eps) and np.all(np.abs(t) <= np.abs(x))


@pytest.mark.parametrize("eps", LEVELS)
def test_truncation_every_float32_mantissa(eps):
    """Every float32 mantissa, with both signs, in the smallest, the unit and the largest
    float32 binade, widened to binary64 and sent through the oracle's whole codec
    (encode, then decode).  Truncation toward zero to m = S - 12 mantissa bits has
    exactly one result: the value t with |t| a multiple of 2^(E-m) (E the binade of x,
    from frexp) and |x| - 2^(E-m) < |t| <= |x|, sign kept.  Checked without the oracle's
    formula for every value."""
    kc = 11
    S = O.sig_bits(eps)
    m = S - 12
    mant = np.arange(1 << 23, dtype=np.uint32)
    for e32 in (1, 127, 254):
        f = ((np.uint32(e32) << np.uint32(23)) | mant).view(np.float32).astype(np.float64)
        x = np.concatenate([f, -f])
        t = np.empty_like(x)
        step = 2 << kc
        for i in range(0, x.size, step):
            t[i:i + step] = O.decode_chunk(O.encode_chunk(x[i:i + step], kc, S), kc).view(np.float64)
        ax, at = np.abs(x), np.abs(t)
        _, ex = np.frexp(ax)
        ulp = np.ldexp(1.0, ex - 1 - m)
        assert np.array_equal(np.signbit(t), np.signbit(x)), e32
        assert np.all(at <= ax) and np.all(ax - at < ulp), e32
        q = at / ulp
        assert np.array_equal(q, np.floor(q)), e32


def test_zero_and_negative_zero():
    for S in (16, 26, 64):
        assert O.truncate(0, S) == 0
        assert O.truncate(0x8000000000000000, S) == 0


# ---------------------------------------------------- hand-derived images --- #

def _expected_image(case) -> bytes:
    h = case["header"]
    head = bytes([h["mode"], h["S"], h["log2P"], 0]) + h["payload_bytes"].to_bytes(4, "little") + \
        h["n_values"].to_bytes(4, "little") + h["resid_bits"].to_bytes(4, "little")
    payload = b""
    if "codes_byte_bits" in case or "codes_bytes_bits" in case:
        cb = case.get("codes_bytes_bits", [case.get("codes_byte_bits")])
        codes = bytes([int(b, 2) for b in cb]).ljust(16, b"\0")
        bits = "".join(case["residual_bits"])
        nwords = (len(bits) + 127) // 128 * 2
        bits = bits.ljust(64 * nwords, "0")
        words = [int(bits[64 * k: 64 * (k + 1)], 2) for k in range(nwords)]
        payload = codes + b"".join(w.to_bytes(8, "little") for w in words)
    elif "payload_hex_le_words" in case:
        payload = b"".join(int(w, 16).to_bytes(8, "little") for w in case["payload_hex_le_words"])
    assert len(payload) == h["payload_bytes"]
    return head + payload


@pytest.mark.parametrize("case", json.load(open(GOLDEN))["cases"], ids=lambda c: c["name"])
def test_hand_derived_image(case):
    vals = np.array([int(v, 16) for v in case["values_hex"]], dtype=np.uint64)
    img = O.encode_chunk(vals, case["kc"], case["S"], modes=case.get("modes", O.DEFAULT_MODES))
    assert img[0] == case["expect_mode"]
    assert img == _expected_image(case)
    dec = O.decode_chunk(img, case["kc"]).view(np.uint64)
    assert np.array_equal(dec, np_truncate(vals, case["S"] if case["expect_mode"] else 64))


# ------------------------------------------------------------ round trips --- #

def _chunks(rng, kc):
    A = 1 << kc
    yield "normal", (rng.standard_normal(A) + 1j * rng.standard_normal(A)) * 2.0 ** -8
    yield "sparse", np.where(rng.random(A) < 0.1, rng.standard_normal(A) + 1j * rng.standard_normal(A), 0)
    yield "const", np.full(A, 0.25 - 0.125j)
    yield "zero", np.zeros(A, dtype=np.complex128)
    if kc >= 2:
        P = 1 << int(rng.integers(1, kc))
        base = rng.standard_normal(P) + 1j * rng.standard_normal(P)
        yield "period", np.tile(base, A // P)
    yield "phases", np.exp(1j * rng.uniform(0, 2 * np.pi, A)) / np.sqrt(A)
    sub = rng.standard_normal(A) + 0j
    sub[rng.integers(0, A)] = 5e-320
    yield "subnormal", sub
    neg = rng.standard_normal(A) + 0j
    neg[::3] = -0.0
    yield "negzero", neg
    # a few-valued state (the Grover diffusion's +-c pattern): PALETTE territory
    lv = np.array([0.125, -0.125, 0.5, -0.0625])
    yield "few", lv[rng.integers(0, 4, A)] + 1j * lv[rng.integers(0, 4, A)] * (rng.random(A) < 0.5)


@pytest.mark.parametrize("kc", [0, 1, 2, 3, 5, 8, 10])
def test_roundtrip(kc):
    rng = np.random.default_rng(100 + kc)
    for name, a in _chunks(rng, kc):
        bits = np.ascontiguousarray(a, dtype=np.complex128).view(np.uint64)
        has_sub = np.any(((bits >> np.uint64(52)) & np.uint64(0x7FF) == 0) & (bits & np.uint64((1 << 52) - 1) != 0))
        for S in (64, 29, 26, 22, 19, 16):
          for force in (-1, 5, 6):
            t = np_truncate(bits, 64 if has_sub else S)
            if force == 6 and np.unique(t).size > 256:
                continue
            img = O.encode_chunk(a, kc, S, force_mode=force, modes=O.ALL_MODES)
            assert len(img) % 16 == 0
            eff = 64 if has_sub else S
            if img[0] != 0:
                assert img[1] == eff, (name, S)
            dec = O.decode_chunk(img, kc).view(np.uint64)
            assert np.array_equal(dec, np_truncate(bits, eff)), (name, kc, S, force)


def _smallest_period(t: np.ndarray, kc: int):
    amps = t.reshape(-1, 2)
    for p in range(1, kc):
        P = 1 << p
        if all(np.array_equal(amps[i], amps[i % P]) for i in range(1 << kc)):
            return p
    return None


def _palette_size(t: np.ndarray):
    """PALETTE image size from the format rule: header, the distinct values (8 bytes
    each, padded to 16), then N indices of k = max(1, ceil(log2 P)) bits padded to 16
    bytes; None above 256 distinct values."""
    P = np.unique(t).size
    if P > 256:
        return None
    k = max(1, (P - 1).bit_length())
    return 16 + (8 * P + 15) // 16 * 16 + (t.size * k + 127) // 128 * 16


@pytest.mark.parametrize("kc", [1, 2, 4, 6, 9])
@pytest.mark.parametrize("modes", [O.DEFAULT_MODES, 0x3F, 0x7F])
def test_selector_is_minimal_and_modes_apply(kc, modes):
    rng = np.random.default_rng(kc)
    for name, a in _chunks(rng, kc):
        for S in (64, 26, 16):
            bits = np.ascontiguousarray(a, dtype=np.complex128).view(np.uint64)
            t = np_truncate(bits, S if name != "subnormal" else 64)
            applicable = {
                0: bool(np.all(t == 0)),
                1: bool(np.all(t.reshape(-1, 2) == t[:2])),
                2: _smallest_period(t, kc) is not None,
                3: True,
                4: True,
                5: True,
                6: _palette_size(t) is not None,
            }
            sizes = {}
            for m in range(7):
                if not (modes >> m) & 1:
                    continue
                if applicable[m]:
                    sizes[m] = len(O.encode_chunk(a, kc, S, force_mode=m))
                else:
                    with pytest.raises(O.OracleError):
                        O.encode_chunk(a, kc, S, force_mode=m)
            auto = O.encode_chunk(a, kc, S, modes=modes)
            best = min(sizes.values())
            assert len(auto) == best
            assert auto[0] == min(m for m, s in sizes.items() if s == best)
            if applicable[2]:
                assert O.encode_chunk(a, kc, S, force_mode=2)[2] == _smallest_period(t, kc)
            assert sizes[4] == 16 + 16 * (1 << kc)
            if 6 in sizes:
                assert sizes[6] == _palette_size(t)


def test_subnormal_forces_full_width():
    a = np.full(8, 0.5 + 0.25j)
    a[3] = 1e-310 + 0j
    img = O.encode_chunk(a, 3, 26)
    assert img[1] == 64
    assert np.array_equal(O.decode_chunk(img, 3), a)


def test_nonfinite_rejected():
    for bad in (np.inf, np.nan):
        a = np.zeros(4, dtype=np.complex128)
        a[1] = bad
        with pytest.raises(O.OracleError):
            O.encode_chunk(a, 2, 26)


def test_corrupt_images_rejected():
    rng = np.random.default_rng(5)
    a = rng.standard_normal(64) + 1j * rng.standard_normal(64)
    img = bytearray(O.encode_chunk(a, 6, 26))
    for pos, val in ((0, 9), (1, 5), (3, 1), (4, 16), (8, 7), (12, 3)):
        bad = bytearray(img)
        bad[pos] = (bad[pos] + val) & 0xFF
        with pytest.raises(O.OracleError):
            O.decode_chunk(bytes(bad), 6)
    with pytest.raises(O.OracleError):
        O.decode_chunk(bytes(img[:-16]), 6)


def test_palette_index_width_and_limit():
    """k = max(1, ceil(log2 P)) for P distinct values; above 256 the mode does not apply."""
    for P, k in ((1, 1), (2, 1), (3, 2), (4, 2), (5, 3), (17, 5), (128, 7), (129, 8), (256, 8)):
        vals = np.arange(1, P + 1, dtype=np.float64)
        a = np.resize(vals, 512)  # 256 amplitudes, kc = 8: P distinct values
        img = O.encode_chunk(a, 8, 64, force_mode=6, modes=O.ALL_MODES)
        assert img[0] == 6 and img[2] == k and int.from_bytes(img[12:16], "little") == P
        assert np.array_equal(O.decode_chunk(img, 8).view(np.float64), a)
    with pytest.raises(O.OracleError):
        O.encode_chunk(np.arange(1, 258, dtype=np.float64).tolist() + [0.0] * 255, 8, 64, force_mode=6)


def test_palette_corrupt_images_rejected():
    lv = np.array([0.5, -0.25, 0.125, 2.0, 3.0])
    rng = np.random.default_rng(3)
    a = lv[rng.integers(0, 5, 256)]
    img = bytearray(O.encode_chunk(a, 7, 26, force_mode=6, modes=O.ALL_MODES))
    assert img[0] == 6 and img[2] == 3
    P = int.from_bytes(img[12:16], "little")
    assert P == 5
    bad = bytearray(img)
    bad[16:24], bad[24:32] = img[24:32], img[16:24]  # palette no longer ascending
    with pytest.raises(O.OracleError):
        O.decode_chunk(bytes(bad), 7)
    bad = bytearray(img)
    bad[2] = 4  # wrong index width
    with pytest.raises(O.OracleError):
        O.decode_chunk(bytes(bad), 7)
    bad = bytearray(img)
    pa = (8 * P + 15) // 16 * 16
    bad[16 + pa + 7] = 0xFF  # first index 0b111 = 7 >= P
    with pytest.raises(O.OracleError):
        O.decode_chunk(bytes(bad), 7)


@pytest.mark.parametrize("kc", [2, 7, 10])
def test_reencoding_at_the_same_width_is_the_identity(kc):
    """Encoding the decoded values of an image again at the same S gives the same bytes
    (truncation is idempotent and the smallest-image choice sees the same values).  The
    streaming kernel relies on it to leave untouched a chunk whose gate row is an exact copy
    when the chunk is already coded at the gate's S."""
    rng = np.random.default_rng(40 + kc)
    for name, a in _chunks(rng, kc):
        for S in (19, 26, 32, 64):
            for modes in (O.DEFAULT_MODES, O.ALL_MODES):
                img = O.encode_chunk(a, kc, S, modes=modes)
                again = O.encode_chunk(O.decode_chunk(img, kc), kc, S, modes=modes)
                assert again == img, (name, S, modes)
