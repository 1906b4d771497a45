"""sim_codec_encode_noalloc: the encoder for callers that cannot allocate device memory
(their device memory belongs to another allocator, e.g. a framework's caching
allocator that already holds the free memory, or to a fixed budget that an allocation
in mid-run could break).  It must write exactly what sim_codec_encode writes for the
same chunks -- the images are integer data, so the tolerance is bit-for-bit -- on
consecutive calls that reuse the library's fixed scratch array, and what the CPU
oracle's encoder writes.  Kept in a file of its own that pytest collects last."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

SCRATCH = 8 << 20


def _chunks(rng, kc, count):
    A = 1 << kc
    out = []
    for k in range(count):
        if k % 4 == 0:
            a = (rng.standard_normal(A) + 1j * rng.standard_normal(A)) * 2.0 ** -10
        elif k % 4 == 1:
            a = np.full(A, complex(0.25, -0.5))
        elif k % 4 == 2:
            a = np.where(rng.random(A) < 0.2, rng.standard_normal(A) + 0j, 0)
        else:
            a = np.tile(rng.standard_normal(4) + 1j * rng.standard_normal(4), max(1, A // 4))[:A]
        out.append(np.asarray(a, dtype=np.complex128))
    return np.concatenate(out)


def _fits(n, kc, stride):
    """The library's layout: [error word, padded to 256][inputs][images][lengths], each
    region rounded up to 256 bytes."""
    r = lambda x: (x + 255) // 256 * 256
    return 256 + r(n * (16 << kc)) + r(n * stride) + 4 * n <= SCRATCH


def _largest_fitting(kc, stride):
    n = SCRATCH // ((16 << kc) + stride + 4)
    while _fits(n + 1, kc, stride):
        n += 1
    while not _fits(n, kc, stride):
        n -= 1
    return n


def test_noalloc_matches_allocating_encoder_on_two_calls():
    from paper_1911_04034_gb300 import qcsim

    rng = np.random.default_rng(123)
    for kc, eps, count in ((10, 1e-4, 96), (8, 0.0, 64), (11, 1e-3, 40), (0, 1e-4, 64)):
        first = _chunks(rng, kc, count)
        second = _chunks(rng, kc, count // 2)  # smaller: stale bytes from call 1 must not leak
        for x in (first, second):
            want, wl = qcsim.codec_encode(x, kc, eps)
            got, gl = qcsim.codec_encode_noalloc(x, kc, eps)
            assert np.array_equal(np.asarray(gl), np.asarray(wl))
            assert got == want


def test_noalloc_forced_mode_matches_allocating_encoder():
    from paper_1911_04034_gb300 import qcsim

    rng = np.random.default_rng(5)
    x = (rng.standard_normal(16 << 9) + 1j * rng.standard_normal(16 << 9)).astype(np.complex128)
    for mode in (3, 4):  # STREAM and RAW apply to any chunk
        want, _ = qcsim.codec_encode(x, 9, 1e-4, force_mode=mode)
        got, _ = qcsim.codec_encode_noalloc(x, 9, 1e-4, force_mode=mode)
        assert got == want


def test_noalloc_matches_the_oracle_directly():
    import oracle as O
    from paper_1911_04034_gb300 import qcsim

    rng = np.random.default_rng(77)
    kc, eps = 10, 1e-4
    x = _chunks(rng, kc, 8)
    got, _ = qcsim.codec_encode_noalloc(x, kc, eps)
    S = O.sig_bits(eps)
    for k in range(8):
        assert got[k] == O.encode_chunk(x[k << kc: (k + 1) << kc], kc, S)


def test_noalloc_at_the_limit_and_one_past_it():
    from paper_1911_04034_gb300 import qcsim

    kc = 10
    stride = qcsim.codec_stride(kc)
    n = _largest_fitting(kc, stride)
    rng = np.random.default_rng(9)
    x = _chunks(rng, kc, n)
    want, _ = qcsim.codec_encode(x, kc, 1e-4)
    got, _ = qcsim.codec_encode_noalloc(x, kc, 1e-4)
    assert got == want
    x1 = np.concatenate([x, np.zeros(1 << kc, dtype=np.complex128)])
    with pytest.raises(qcsim.SimError) as ei:
        qcsim.codec_encode_noalloc(x1, kc, 1e-4)
    assert ei.value.code == qcsim.ERR_INVALID
    assert "8 MiB" in str(ei.value)


def test_noalloc_rejects_requests_beyond_its_scratch():
    from paper_1911_04034_gb300 import qcsim

    x = np.zeros(600 << 10, dtype=np.complex128)  # 600 chunks of 2^10 amplitudes: > 8 MiB staged
    with pytest.raises(qcsim.SimError) as ei:
        qcsim.codec_encode_noalloc(x, 10, 1e-4)
    assert ei.value.code == qcsim.ERR_INVALID
    assert "8 MiB" in str(ei.value)


def test_noalloc_reserves_no_device_memory():
    import torch

    from paper_1911_04034_gb300 import qcsim

    rng = np.random.default_rng(11)
    x = _chunks(rng, 10, 64)
    qcsim.codec_encode_noalloc(x, 10, 1e-4)  # the first call on the device does its set-up
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        qcsim.codec_encode_noalloc(x, 10, 1e-4)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
