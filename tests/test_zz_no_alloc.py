"""sim_codec_encode_noalloc: the encoder for callers that cannot allocate device memory
(their device memory belongs to another allocator or to a fixed budget).  It must
write exactly what sim_codec_encode writes for the same chunks -- the images are
integer data, so the tolerance is bit-for-bit -- on consecutive calls that reuse the
library's fixed scratch array.  Kept in a file of its own that pytest collects last."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


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
            a = np.tile(rng.standard_normal(4) + 1j * rng.standard_normal(4), A // 4)
        out.append(np.asarray(a, dtype=np.complex128))
    return np.concatenate(out)


def test_noalloc_matches_allocating_encoder_on_two_calls():
    from paper_1911_04034_gb300 import qcsim

    rng = np.random.default_rng(123)
    for kc, eps, count in ((10, 1e-4, 96), (8, 0.0, 64)):
        first = _chunks(rng, kc, count)
        second = _chunks(rng, kc, count // 2)  # smaller: stale bytes from call 1 must not leak
        for x in (first, second):
            want, wl = qcsim.codec_encode(x, kc, eps)
            got, gl = qcsim.codec_encode_noalloc(x, kc, eps)
            assert np.array_equal(np.asarray(gl), np.asarray(wl))
            assert got == want


def test_noalloc_rejects_requests_beyond_its_scratch():
    from paper_1911_04034_gb300 import qcsim

    x = np.zeros(600 << 10, dtype=np.complex128)  # 600 chunks of 2^10 amplitudes: > 8 MiB staged
    with pytest.raises(qcsim.SimError) as ei:
        qcsim.codec_encode_noalloc(x, 10, 1e-4)
    assert ei.value.code == qcsim.ERR_INVALID
    assert "8 MiB" in str(ei.value)
