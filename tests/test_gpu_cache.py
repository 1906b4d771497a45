"""Compressed block cache (Section 3.4): work items whose two input images were seen
earlier in the same gate take the cached outputs.  The result must be byte-identical
to computing them (and to the oracle), hits must happen on redundant states, and the
cache must pause itself when it never hits."""
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


def make(n, kc, eps, budget_div=4, cache=False, ladder=0):
    s = qc().Sim(n, n, eps, chunk_log2=kc, budget=(16 << n) // budget_div, ladder=ladder,
                 pool_bytes=2 * (16 << n) + (32 << 20))
    if cache:
        s.set_block_cache(True)
    return s


@pytest.mark.parametrize("kc", [5, 7])
def test_cache_gives_the_same_images_on_grover(kc):
    """18 qubits: a gate has thousands of work items, several per CTA, so later items
    find the lines that earlier ones of the same gate published."""
    n, eps = 18, 1e-4
    gates, _ = Cc.grover(n, 2, seed=6)
    a, b = make(n, kc, eps, cache=True), make(n, kc, eps)
    for k in range(0, len(gates), 40):
        a.apply_circuit(gates[k:k + 40])
        b.apply_circuit(gates[k:k + 40])
        assert images(a) == images(b), k
    sa, sb = a.stats(), b.stats()
    for key in ("gates", "encoded_bytes", "max_encoded_bytes", "eps_switch_gate", "level", "fidelity_lb_sum"):
        assert sa[key] == sb[key], key
    assert sa["cache_hits"] > 0 and sa["cache_lookups"] > sa["cache_hits"]
    assert sb["cache_lookups"] == 0
    orc = O.CSim(n, n, kc, eps, (16 << n) // 4)
    orc.apply(gates)
    assert images(a) == [orc.image(c) for c in range(orc.nchunks)]


def test_cache_on_qaoa_matches_the_oracle():
    n, kc, eps = 14, 6, 1e-3
    gates, _ = Cc.qaoa_maxcut(n, 2, 3, seed=8)
    a = make(n, kc, eps, cache=True, ladder=1)
    a.apply_circuit(gates)
    orc = O.CSim(n, n, kc, eps, (16 << n) // 4, ladder=1)
    orc.apply(gates)
    assert images(a) == [orc.image(c) for c in range(orc.nchunks)]


def test_cache_pauses_when_it_never_hits():
    """A deep random circuit: every chunk pair is distinct, so after 16 gates with
    lookups and no hit the cache sits out the next 64 gates."""
    n, kc = 12, 5
    gates = Cc.rcs_n(n, 12, seed=4)
    s = make(n, kc, 1e-4)
    s.apply_circuit(gates[:60])  # scramble first, without the cache
    s.set_block_cache(True)
    s.apply_circuit(gates[60:60 + 16])
    st = s.stats()
    assert st["cache_hits"] == 0 and st["cache_lookups"] > 0
    s.apply_circuit(gates[76:76 + 40])
    assert s.stats()["cache_lookups"] == st["cache_lookups"]


def test_batched_launch_with_caches():
    kc, eps = 6, 1e-4
    sizes = (14, 16, 17)
    circuits = [Cc.grover(n, 1, seed=n)[0] for n in sizes]
    batch = [make(n, kc, eps, cache=True) for n in sizes]
    qc().batch_apply(batch, circuits)
    for k, n in enumerate(sizes):
        solo = make(n, kc, eps)
        solo.apply_circuit(circuits[k])
        assert images(batch[k]) == images(solo)
    assert sum(s.stats()["cache_hits"] for s in batch) > 0
