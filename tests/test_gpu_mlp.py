"""Learned chunk-mode selector (not from the paper): the GPU training kernels against
the oracle's gradients, selector decisions reproduced bit for bit by the oracle's
compressed simulator, and what the trained network gains over the method without it.

Selectors: 0 = Solution C modes only (the paper's choice); 1 = Solution C and D, every
chunk trying both orders (exhaustive); 2 = C and D, the network deciding which chunks
try the Solution D order.  The codec enforces the bound under all three."""
import numpy as np
import pytest

import oracle as O
from oracle import mlp as M
from paper_1911_04034_gb300 import circuits as Cc

pytestmark = pytest.mark.gpu


def qc():
    from paper_1911_04034_gb300 import qcsim

    return qcsim


def bf16_bits(flat32: np.ndarray) -> np.ndarray:
    return (M.bf16_round(flat32).view(np.uint32) >> 16).astype(np.uint16)


def random_params(seed):
    rng = np.random.default_rng(seed)
    p = M.init_params(seed)
    for k in ("b1", "b2", "b3"):
        p[k] = M.bf16_round(rng.standard_normal(M.SHAPES[k]).astype(np.float32) * 0.5)
    return M.flatten(p)


def test_gpu_gradient_matches_oracle():
    rng = np.random.default_rng(1)
    n = 3000
    flat = random_params(2)
    x = rng.random((n, 16)).astype(np.float32)
    mode = rng.integers(0, 6, size=n).astype(np.int32)
    sizes = rng.random((n, 2)).astype(np.float32)
    loss, g = qc().mlp_grad(flat, x, mode, sizes)
    p = {k: v.astype(np.float64) for k, v in M.unflatten(M.bf16_round(flat)).items()}
    want_loss, want = M.loss_and_grads(p, x.astype(np.float64), mode, sizes.astype(np.float64))
    gw = M.flatten({k: want[k].astype(np.float32) for k in M.ORDER})
    assert loss == pytest.approx(want_loss, rel=1e-4)
    scale = np.max(np.abs(gw))
    assert np.max(np.abs(g - gw)) <= 2e-4 * scale


def test_gpu_training_reduces_the_loss():
    rng = np.random.default_rng(3)
    n = 4096
    x = rng.random((n, 16)).astype(np.float32)
    mode = np.where(x[:, 9] > 0.5, 5, 3).astype(np.int32)
    sizes = np.stack([0.3 + 0.2 * x[:, 6], 0.2 + 0.3 * x[:, 7]], axis=1).astype(np.float32)
    p0 = random_params(4)
    l0, _ = qc().mlp_grad(p0, x, mode, sizes)
    p1, wb, l1 = qc().mlp_train(x, mode, sizes, p0, epochs=30, batch=256, lr=3e-3, seed=5)
    lf, _ = qc().mlp_grad(p1, x, mode, sizes)
    assert lf < 0.3 * l0
    acc = np.mean(M.wants_split(M.unflatten(M.bf16_round(p1)), x) == (mode == 5))
    assert acc > 0.95
    assert np.array_equal(wb, bf16_bits(p1))


@pytest.mark.parametrize("circuit", ["grover", "rcs"])
def test_selector_decisions_bit_exact_with_oracle(circuit):
    n, kc, eps = 12, 7, 1e-4
    if circuit == "grover":
        gates, _ = Cc.grover(n, 3, seed=5)
    else:
        gates = Cc.rcs(3, 4, 4, seed=5)
    flat = random_params(9)
    budget = (16 << n) // 6
    orc = O.CSim(n, 9, kc, eps, budget)
    orc.set_mlp(M.bf16_round(flat))
    gpu = qc().Sim(n, 9, eps, chunk_log2=kc, budget=budget, pool_bytes=64 << 20)
    gpu.set_selector(2, bf16_bits(flat))
    gpu.apply_circuit(gates)
    orc.apply(gates)
    assert [gpu.chunk_image(c) for c in range(gpu.n_chunks)] == [orc.image(c) for c in range(orc.nchunks)]
    st = gpu.stats()
    assert 0 < st["split_trials"]


@pytest.mark.parametrize("n,kc", [(10, 5), (12, 9)])
def test_trace_records_match_oracle_features(n, kc):
    """Every training record the device writes (exhaustive selector) is the oracle's
    feature row for one of the chunks the gate re-encoded, with the exhaustive mode and
    the STREAM / SPLIT sizes of that chunk."""
    eps = 1e-4
    gates = list(Cc.grover(n, 1, seed=3)[0][: 3 * n]) + list(Cc.rcs_n(n, 3, seed=4))
    gpu = qc().Sim(n, n, eps, chunk_log2=kc, budget=1, pool_bytes=(16 << n) + (64 << 20))
    gpu.set_selector(1)
    gpu.trace(1 << 16)
    orc = O.CSim(n, n, kc, eps, 1, modes=0x3F)
    raw = np.float32(16 + (16 << kc))
    prev = [orc.image(c) for c in range(orc.nchunks)]
    seen = 0
    for g in gates:
        gpu.apply_circuit([g])
        orc.apply([g])
        cur = [orc.image(c) for c in range(orc.nchunks)]
        S = orc.stats()["S_current"]
        want = set()
        for c in range(orc.nchunks):
            vals = O.decode_chunk(cur[c], kc)
            f = M.features(prev[c], kc, g["u"], int(g["target"]), S, vals)
            sz = O.mode_sizes(vals, kc, cur[c][1] if cur[c][0] else S)
            row = np.concatenate([f, np.array([cur[c][0], np.float32(sz[3]) / raw, np.float32(sz[5]) / raw, 0],
                                              dtype=np.float32)])
            want.add(row.astype(np.float32).tobytes())
        recs = gpu.trace_read()
        assert recs.shape[0] >= seen
        for r in recs[seen:]:
            assert r.astype(np.float32).tobytes() in want
        seen = recs.shape[0]
        prev = cur
    assert seen > len(gates)


def _run(gates, n, kc, eps, selector, params=None):
    s = qc().Sim(n, n, eps, chunk_log2=kc, budget=1, pool_bytes=(16 << n) + (64 << 20))  # lossy from gate 0
    if selector == 2:
        s.set_selector(2, params)
    else:
        s.set_selector(selector)
    s.apply_circuit(gates)
    return s.stats()


def test_trained_selector_gain():
    """Traces from exhaustive runs (a real-valued Grover search and a complex random
    circuit) train the network on the GPU; on fresh circuits of both kinds it must keep
    almost all of the exhaustive ratio while running far fewer Solution D trials, and
    beat Solution C alone on the real-valued state."""
    n, kc, eps = 14, 8, 1e-4
    train_sets = [Cc.grover(n, 3, seed=11)[0], Cc.rcs_n(n, 6, seed=12)]
    recs = []
    for g in train_sets:
        s = qc().Sim(n, n, eps, chunk_log2=kc, budget=1, pool_bytes=(16 << n) + (64 << 20))
        s.set_selector(1)
        s.trace(1 << 20)
        s.apply_circuit(g)
        recs.append(s.trace_read())
    tr = np.concatenate(recs)
    assert tr.shape[0] > 1000
    x, mode, sizes = tr[:, :16], tr[:, 16].astype(np.int32), tr[:, 17:19]
    p, wb, loss = qc().mlp_train(x, mode, sizes, random_params(13), epochs=40, batch=256, lr=3e-3, seed=14)
    for g in (Cc.grover(n, 3, seed=21)[0], Cc.rcs_n(n, 6, seed=22)):
        c_only = _run(g, n, kc, eps, 0)
        exh = _run(g, n, kc, eps, 1)
        net = _run(g, n, kc, eps, 2, wb)
        assert exh["max_encoded_bytes"] <= c_only["max_encoded_bytes"]
        # the network keeps >= 98 % of the exhaustive compression ...
        assert net["max_encoded_bytes"] <= 1.02 * exh["max_encoded_bytes"]
        # ... with fewer Solution D trials than the exhaustive selector runs
        assert net["split_trials"] < exh["split_trials"]
    # on the real-valued Grover state Solution D pays: the network beats Solution C alone
    g = Cc.grover(n, 3, seed=21)[0]
    assert _run(g, n, kc, eps, 2, wb)["max_encoded_bytes"] < 0.9 * _run(g, n, kc, eps, 0)["max_encoded_bytes"]
