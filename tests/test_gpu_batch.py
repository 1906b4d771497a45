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


def test_autotune_searches_block_tile_and_schedule():
    """Coordinate descent over block size, chunk size, ladder and mode set: every
    measured point is a distinct setting as the handle applies it (blocks clamped to n,
    chunks to the block), every rate is positive, and the winner has the highest rate
    measured."""
    n = 14
    probe = Cc.rcs_n(n, 6, seed=8)
    best, tried = qc().autotune(n, 1e-4, probe, block_log2s=(16, 10, 12, 14), chunk_log2s=(9, 8, 7),
                                ladders=(0, 1, 2), mode_sets=(0x1F, 0x5F))
    keys = [(p["block_log2"], p["chunk_log2"], p["ladder"], p["modes"]) for p in tried]
    assert len(keys) == len(set(keys)) >= 1 + 2 + 2 + 2 + 1
    for b, kc, lad, m in keys:
        assert b <= n and kc <= b and lad in (0, 1, 2) and m in (0x1F, 0x5F)
    assert all(p["rate"] > 0 and p["ratio"] > 1 for p in tried)
    assert best["rate"] == max(p["rate"] for p in tried)
    assert (best["block_log2"], best["chunk_log2"], best["ladder"], best["modes"]) in keys


def test_reset_then_rerun_is_a_fresh_run():
    """sim_reset returns the handle to |0...0> with zero statistics; the same circuit
    run again (block cache on) gives the bytes of a fresh handle."""
    n, kc, eps = 13, 8, 1e-4
    gates = Cc.rcs_n(n, 6, seed=9)
    s = make(n, kc, eps)
    s.set_block_cache(True)
    s.apply_circuit(Cc.qft(n, seed=3)[0])
    s.reset()
    fresh = make(n, kc, eps)
    assert images(s) == images(fresh)
    st = s.stats()
    assert st["gates"] == 0 and st["amp_updates"] == 0 and st["eps_switch_gate"] == -1 and st["level"] == 0
    s.apply_circuit(gates)
    fresh.apply_circuit(gates)
    assert images(s) == images(fresh)
    for key in ("gates", "encoded_bytes", "max_encoded_bytes", "eps_switch_gate", "amp_updates", "pages_in_use_bytes"):
        assert s.stats()[key] == fresh.stats()[key], key


def test_batch_graph_is_kept_and_replayed():
    """The graph of a batched call stays with the first handle: after sim_reset the same
    call replays it (same bytes as the first run); a changed circuit is captured anew
    and still equals the circuits run alone."""
    kc, eps = 7, 1e-4
    specs = [(11, 5), (13, 4), (12, 6), (10, 3)]
    circuits = [Cc.rcs_n(n, d, seed=300 + k) for k, (n, d) in enumerate(specs)]
    batch = [make(n, kc, eps) for n, _ in specs]
    qc().batch_apply(batch, circuits, use_graph=True)
    first = [images(s) for s in batch]
    for s in batch:
        s.reset()
    qc().batch_apply(batch, circuits, use_graph=True)
    assert batch[0].stats()["graph_replays"] == 1
    assert [images(s) for s in batch] == first
    for s in batch:
        s.reset()
    circuits[2] = Cc.rcs_n(12, 6, seed=399)
    qc().batch_apply(batch, circuits, use_graph=True)
    assert batch[0].stats()["graph_replays"] == 1
    for k, (n, _) in enumerate(specs):
        solo = make(n, kc, eps)
        solo.apply_circuit(circuits[k])
        assert images(batch[k]) == images(solo), k


def test_batch_run_matches_individual_runs():
    """sim_batch_run: handles created, run batched and destroyed inside the call; each
    circuit's statistics equal those of the same circuit run alone with the same
    settings (block and chunk size, ladder and mode set as the call reports them)."""
    rng = np.random.default_rng(11)
    eps = 1e-4
    sizes = [int(rng.integers(9, 14)) for _ in range(6)]
    circuits = [Cc.rcs_n(n, int(rng.integers(3, 7)), seed=200 + k) for k, n in enumerate(sizes)]
    stats = qc().batch_run(circuits, sizes, eps)
    for k, n in enumerate(sizes):
        kc, b = stats[k]["chunk_log2"], stats[k]["block_log2"]
        raw = 16 << n
        solo = qc().Sim(n, b, eps, chunk_log2=kc, budget=raw // 4, ladder=stats[k]["ladder"],
                        pool_bytes=raw + raw // 8 + (8 << 20))
        solo.set_modes(stats[k]["modes"])
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
