"""Checkpoint / resume (Section 3.5): a state saved mid-circuit and loaded into a fresh
handle continues exactly like the uninterrupted run -- same images, same controller,
same counters -- and both agree with the oracle's compressed simulator."""
import numpy as np
import pytest

import oracle as O
from paper_1911_04034_gb300 import circuits as Cc

pytestmark = pytest.mark.gpu


def qc():
    from paper_1911_04034_gb300 import qcsim

    return qcsim


def images(sim):
    return [sim.chunk_image(c) for c in range(sim.n_chunks)]


def make(n, kc, eps, ladder=0):
    return qc().Sim(n, min(n, 10), eps, chunk_log2=kc, budget=(16 << n) // 4, ladder=ladder,
                    pool_bytes=2 * (16 << n) + (32 << 20))


KEYS = ("gates", "encoded_bytes", "max_encoded_bytes", "eps_switch_gate", "level", "sig_bits_current",
        "fidelity_lb_sum", "fidelity_lb_prod", "amp_updates", "chunks_by_mode", "pages_in_use_bytes")


@pytest.mark.parametrize("split", [5, 40, 120])  # before, around and after the switch to lossy
@pytest.mark.parametrize("kc", [6, 10])
def test_resume_continues_bit_identically(split, kc):
    n, eps = 14, 1e-4
    gates = Cc.rcs_n(n, 10, seed=31)
    a = make(n, kc, eps)
    a.apply_circuit(gates[:split])
    ck = a.checkpoint()
    b = make(n, kc, eps)
    b.apply_circuit(Cc.h_all(n))  # some other state first: the load replaces it
    b.restore(ck)
    assert images(b) == images(a)
    a.apply_circuit(gates[split:])
    b.apply_circuit(gates[split:])
    assert images(b) == images(a)
    sa, sb = a.stats(), b.stats()
    for k in KEYS:
        assert sa[k] == sb[k], k
    orc = O.CSim(n, min(n, 10), kc, eps, (16 << n) // 4)
    orc.apply(gates)
    assert images(b) == [orc.image(c) for c in range(orc.nchunks)]


def test_checkpoint_in_device_memory_and_guarded_ladder():
    torch = pytest.importorskip("torch")
    n, kc, eps = 14, 8, 1e-3
    gates, _ = Cc.qaoa_maxcut(n, 2, 3, seed=4)
    a = make(n, kc, eps, ladder=2)
    a.apply_circuit(gates[:60])
    host = a.checkpoint()
    dev = torch.zeros(host.size, dtype=torch.uint8, device="cuda")
    a.checkpoint(out=dev)
    assert np.array_equal(dev.cpu().numpy(), host)
    b = make(n, kc, eps, ladder=2)
    b.restore(dev)
    a.apply_circuit(gates[60:])
    b.apply_circuit(gates[60:])
    assert images(b) == images(a)
    assert a.stats()["level"] == b.stats()["level"]


def test_checkpoint_layout_and_rejections():
    n, kc = 12, 6
    a = make(n, kc, 1e-4)
    a.apply_circuit(Cc.rcs_n(n, 4, seed=2))
    ck = a.checkpoint()
    assert bytes(ck[:8]) == b"QCSIMCK1"
    nch = 1 << (n - kc)
    lens = ck[256:256 + 4 * nch].view(np.uint32)
    assert ck.size == 256 + 4 * nch + int(lens.sum())
    imgs = images(a)
    assert [int(x) for x in lens] == [len(b) for b in imgs]
    assert bytes(ck[256 + 4 * nch:]) == b"".join(imgs)
    bad = ck.copy()
    bad[0] ^= 1
    with pytest.raises(qc().SimError) as ei:
        make(n, kc, 1e-4).restore(bad)
    assert ei.value.code == qc().ERR_INVALID
    with pytest.raises(qc().SimError):
        make(n, kc, 1e-4).restore(ck[:-16])
    with pytest.raises(qc().SimError):
        make(n + 1, kc, 1e-4).restore(ck)
    with pytest.raises(qc().SimError):
        make(n, kc, 1e-3).restore(ck)
    bad = ck.copy()
    bad[256:260] = np.frombuffer(np.uint32(17).tobytes(), dtype=np.uint8)
    with pytest.raises(qc().SimError):
        make(n, kc, 1e-4).restore(bad)
