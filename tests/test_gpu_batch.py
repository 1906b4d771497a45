"""Batched launches (many circuits of uneven size in one persistent launch per gate
step, captured in a CUDA graph) and the chunk-size autotuner.  Each circuit must end
in exactly the state -- chunk images, counters, controller -- that running it alone
gives, and the oracle's compressed simulator agrees with both."""
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


def make(n, kc, eps):
    budget = (16 << n) // 3
    return qc().Sim(n, min(n, 9), eps, chunk_log2=kc, budget=budget, pool_bytes=2 * (16 << n) + (32 << 20))


@pytest.mark.parametrize("use_graph", [True, False])
def test_batch_equals_individual_runs(use_graph):
    rng = np.random.default_rng(7)
    kc, eps = 6, 1e-3
    specs = [(int(rng.integers(7, 14)), int(rng.integers(3, 9))) for _ in range(12)]
    circuits = [Cc.rcs_n(n, d, seed=100 + k) for k, (n, d) in enumerate(specs)]
    batch = [make(n, kc, eps) for n, _ in specs]
    qc().batch_apply(batch, circuits, use_graph=use_graph)
    for k, (n, _) in enumerate(specs):
        solo = make(n, kc, eps)
        solo.apply_circuit(circuits[k])
        assert images(batch[k]) == images(solo), k
        a, b = batch[k].stats(), solo.stats()
        for key in ("gates", "encoded_bytes", "max_encoded_bytes", "eps_switch_gate", "level", "amp_updates"):
            assert a[key] == b[key], (k, key)
    # two of them against the oracle's compressed simulator as well
    for k in (0, 5):
        n = specs[k][0]
        orc = O.CSim(n, min(n, 9), kc, eps, (16 << n) // 3)
        orc.apply(circuits[k])
        assert images(batch[k]) == [orc.image(c) for c in range(orc.nchunks)]


def test_batch_rejects_mixed_chunk_sizes_and_duplicates():
    a = make(8, 4, 1e-3)
    b = make(8, 5, 1e-3)
    g = Cc.h_all(8)
    with pytest.raises(qc().SimError):
        qc().batch_apply([a, b], [g, g])
    with pytest.raises(qc().SimError):
        qc().batch_apply([a, a], [g, g])


def test_autotune_returns_fastest_candidate():
    n = 14
    probe = Cc.rcs_n(n, 4, seed=3)
    best, rates = qc().autotune_chunk(n, 12, 1e-4, probe, candidates=(6, 8, 10))
    assert best in (6, 8, 10)
    assert all(r > 0 for r in rates.values())
    assert rates[best] == max(rates.values())


def test_batch_run_matches_individual_runs():
    """sim_batch_run: handles created, run batched and destroyed inside the call; each
    circuit's statistics equal those of the same circuit run alone with the same
    settings (chunk size as the call reports it)."""
    rng = np.random.default_rng(11)
    eps = 1e-4
    sizes = [int(rng.integers(9, 14)) for _ in range(6)]
    circuits = [Cc.rcs_n(n, int(rng.integers(3, 7)), seed=200 + k) for k, n in enumerate(sizes)]
    stats = qc().batch_run(circuits, sizes, eps)
    for k, n in enumerate(sizes):
        kc = stats[k]["chunk_log2"]
        raw = 16 << n
        solo = qc().Sim(n, min(n, 20), eps, chunk_log2=kc, budget=raw // 4, pool_bytes=raw + raw // 8 + (8 << 20))
        solo.apply_circuit(circuits[k])
        st = solo.stats()
        for key in ("gates", "encoded_bytes", "max_encoded_bytes", "eps_switch_gate", "level", "amp_updates"):
            assert stats[k][key] == st[key], (k, key)


def test_budget_and_named_options():
    n, kc = 12, 6
    gates = Cc.rcs_n(n, 6, seed=5)
    raw = 16 << n
    a = qc().Sim(n, n, 1e-4, chunk_log2=kc, budget=raw // 4, pool_bytes=2 * raw + (16 << 20))
    b = qc().Sim(n, n, 1e-4, chunk_log2=kc, budget=raw // 4, pool_bytes=2 * raw + (16 << 20))
    b.set_budget(4 * raw)  # lossless fits: never switches
    a.apply_circuit(gates)
    b.apply_circuit(gates)
    assert a.stats()["eps_switch_gate"] >= 0 and b.stats()["eps_switch_gate"] == -1
    c = qc().Sim(n, n, 1e-4, chunk_log2=kc, budget=raw // 4, pool_bytes=2 * raw + (16 << 20))
    c.set_option("tau_ppm", 100000)  # tau 0.1: switches no later than at tau 0.9
    c.set_option("ladder", 1)
    c.apply_circuit(gates)
    assert 0 <= c.stats()["eps_switch_gate"] <= a.stats()["eps_switch_gate"]
    with pytest.raises(qc().SimError):
        c.set_option("ladder", 0)  # only before the first gate
    for key, val in (("chunk_log2", 5), ("no_such_option", 1), ("selector", 2), ("tau_ppm", 0)):
        with pytest.raises(qc().SimError) as ei:
            c.set_option(key, val)
        assert ei.value.code == qc().ERR_INVALID
    d = qc().Sim(n, n, 1e-4, chunk_log2=kc, budget=raw // 4, pool_bytes=2 * raw + (16 << 20))
    e = qc().Sim(n, n, 1e-4, chunk_log2=kc, budget=raw // 4, pool_bytes=2 * raw + (16 << 20))
    d.set_option("modes", 0x3F)
    e.set_modes(0x3F)
    d.apply_circuit(gates)
    e.apply_circuit(gates)
    assert images(d) == images(e)
