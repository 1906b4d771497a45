"""GPU codec parity: the device encoder writes the same bytes as the CPU oracle for the
same chunk, every mode and bound; the device decoder returns the oracle's values bit
for bit (Section 4.2, Solution C; Eq. sigbits)."""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

EPS = [0.0, 1e-5, 1e-4, 1e-3, 1e-2, 1e-1]


def qc():
    from paper_1911_04034_gb300 import qcsim

    return qcsim


def chunk_families(rng, kc, count):
    """Seeded chunks with the structures a state vector shows: dense random, sparse,
    constant, zero, periodic, unit-modulus phases, +-0, subnormals, tiny and huge."""
    A = 1 << kc
    out = []
    for k in range(count):
        f = k % 10
        if f == 0:
            a = (rng.standard_normal(A) + 1j * rng.standard_normal(A)) * 2.0 ** -int(rng.integers(1, 20))
        elif f == 1:
            a = np.where(rng.random(A) < 0.05, rng.standard_normal(A) + 1j * rng.standard_normal(A), 0)
        elif f == 2:
            a = np.full(A, complex(rng.standard_normal(), rng.standard_normal()))
        elif f == 3:
            a = np.zeros(A, dtype=np.complex128)
        elif f == 4 and kc >= 2:
            P = 1 << int(rng.integers(1, kc))
            a = np.tile(rng.standard_normal(P) + 1j * rng.standard_normal(P), A // P)
        elif f == 5:
            a = np.exp(1j * rng.uniform(0, 2 * np.pi, A)) / np.sqrt(A)
        elif f == 6:
            a = rng.standard_normal(A) + 0j
            a[::2] = -0.0
        elif f == 7:
            a = rng.standard_normal(A) + 1j * rng.standard_normal(A)
            a[int(rng.integers(0, A))] = complex(3e-320, 0)
        elif f == 8:
            a = (rng.standard_normal(A) + 1j * rng.standard_normal(A)) * 1e-300
        else:
            v = rng.choice([0.5, -0.25, 0.125], size=A) + 1j * rng.choice([0.0, 0.5], size=A)
            a = v.astype(np.complex128)
        out.append(np.asarray(a, dtype=np.complex128))
    return out


@pytest.mark.parametrize("modes", [0x1F, 0x3F, 0x5F, 0x7F])
@pytest.mark.parametrize("kc", [0, 1, 2, 3, 5, 7, 8, 9, 10, 11])
def test_encode_bytes_match_oracle(kc, modes):
    rng = np.random.default_rng(1000 + kc)
    chunks = chunk_families(rng, kc, 40)
    x = np.concatenate(chunks)
    for eps in EPS:
        S = O.sig_bits(eps)
        imgs, lens = qc().codec_encode(x, kc, eps, modes=modes)
        for k, a in enumerate(chunks):
            ref = O.encode_chunk(a, kc, S, modes=modes)
            assert imgs[k] == ref, (kc, eps, k, imgs[k][:16].hex(), ref[:16].hex())


@pytest.mark.parametrize("e32", [1, 127, 254])
def test_every_float32_mantissa_matches_oracle(e32):
    """All 2^23 float32 mantissas of one binade with both signs (the smallest, the unit
    and the largest float32 binade), widened to binary64, in index order and in a seeded
    shuffle: 4096 chunks of 2^11 amplitudes per bound, the device's images byte for byte
    the oracle's."""
    kc = 11
    mant = np.arange(1 << 23, dtype=np.uint32)
    f = ((np.uint32(e32) << np.uint32(23)) | mant).view(np.float32).astype(np.float64)
    x = np.concatenate([f, -np.random.default_rng(e32).permutation(f)])
    step = 2 << kc
    for eps in EPS:
        S = O.sig_bits(eps)
        imgs, _ = qc().codec_encode(x.view(np.complex128), kc, eps)
        assert len(imgs) == x.size // step
        for k in range(len(imgs)):
            assert imgs[k] == O.encode_chunk(x[k * step:(k + 1) * step], kc, S), (eps, k)


@pytest.mark.parametrize("kc", [1, 4, 8, 10])
def test_forced_modes_match_oracle(kc):
    rng = np.random.default_rng(kc)
    chunks = chunk_families(rng, kc, 20)
    for eps in (0.0, 1e-4):
        S = O.sig_bits(eps)
        for m in range(6):
            for a in chunks:
                try:
                    ref = O.encode_chunk(a, kc, S, force_mode=m)
                except O.OracleError:
                    with pytest.raises(qc().SimError):
                        qc().codec_encode(a, kc, eps, force_mode=m)
                    continue
                imgs, _ = qc().codec_encode(a, kc, eps, force_mode=m)
                assert imgs[0] == ref


@pytest.mark.parametrize("kc", [0, 2, 6, 8, 10, 11])
def test_decode_matches_oracle(kc):
    rng = np.random.default_rng(77 + kc)
    chunks = chunk_families(rng, kc, 30)
    for eps in EPS:
        S = O.sig_bits(eps)
        imgs = [O.encode_chunk(a, kc, S) for a in chunks] + [O.encode_chunk(a, kc, S, force_mode=5) for a in chunks]
        got = qc().codec_decode(imgs, kc)
        want = np.concatenate([O.decode_chunk(b, kc) for b in imgs])
        assert np.array_equal(got.view(np.uint64), want.view(np.uint64))


def test_device_buffers_round_trip():
    torch = pytest.importorskip("torch")
    kc = 10
    rng = np.random.default_rng(3)
    x = np.concatenate(chunk_families(rng, kc, 64))
    dx = torch.from_numpy(x.view(np.float64).copy()).cuda()
    buf, lens, stride = qc().codec_encode(dx, kc, 1e-4)
    host_imgs, _ = qc().codec_encode(x, kc, 1e-4)
    b = buf.cpu().numpy()
    ln = lens.cpu().numpy()
    for k in range(len(host_imgs)):
        assert b[k * stride: k * stride + ln[k]].tobytes() == host_imgs[k]


def test_corrupt_images_are_reported_not_trapped():
    kc = 6
    rng = np.random.default_rng(9)
    a = rng.standard_normal(1 << kc) + 1j * rng.standard_normal(1 << kc)
    good = O.encode_chunk(a, kc, O.sig_bits(1e-4))
    for pos, val in ((0, 9), (1, 5), (3, 1), (4, 16), (8, 7), (12, 3)):
        bad = bytearray(good)
        bad[pos] = (bad[pos] + val) & 0xFF
        with pytest.raises(qc().SimError) as ei:
            qc().codec_decode([bytes(bad)], kc)
        assert ei.value.code == qc().ERR_CORRUPT
    # the decoder keeps working afterwards
    assert np.array_equal(qc().codec_decode([good], kc), O.decode_chunk(good, kc))


def test_nonfinite_input_rejected():
    a = np.zeros(16, dtype=np.complex128)
    a[3] = np.nan
    with pytest.raises(qc().SimError) as ei:
        qc().codec_encode(a, 4, 1e-4)
    assert ei.value.code == qc().ERR_INVALID


@pytest.mark.parametrize("kc", [0, 2, 6, 8, 10, 11])
def test_palette_mode_forced_and_decoded_like_the_oracle(kc):
    """PALETTE forced on few-valued chunks (the distinct-value count from 1 to 256, and
    257, where it does not apply): the device's images are the oracle's byte for byte
    and decode to the oracle's values."""
    rng = np.random.default_rng(77 + kc)
    A = 1 << kc
    q = qc()
    for P in (1, 2, 3, 5, 16, 100, 256, 257):
        if P > 2 * A:
            continue
        lv = rng.standard_normal(P)
        vals = np.resize(rng.permutation(lv), 2 * A)  # every one of the P values occurs
        rng.shuffle(vals)
        a = vals.view(np.complex128)
        for eps in (0.0, 1e-4):
            S = O.sig_bits(eps)
            t = np.unique(vals.view(np.uint64) & np.uint64(~((1 << (64 - S)) - 1) & (2**64 - 1)))
            if t.size > 256:
                with pytest.raises(q.SimError):
                    q.codec_encode(a, kc, eps, force_mode=6, modes=0x7F)
                continue
            imgs, _ = q.codec_encode(a, kc, eps, force_mode=6, modes=0x7F)
            ref = O.encode_chunk(a, kc, S, force_mode=6, modes=0x7F)
            assert imgs[0] == ref, (P, eps)
            dec = q.codec_decode([ref], kc)
            assert np.array_equal(dec.view(np.uint64), O.decode_chunk(ref, kc).view(np.uint64))
