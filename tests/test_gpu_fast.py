"""The streaming gate kernel (one warp pair per work item, values kept in registers from
decoder to encoder) against the oracle and against the general kernel.

Every gate of a lossy run at chunk sizes 2^7..2^11 goes through the streaming kernel
first; items it cannot finish as STREAM images go to the general kernel.  Both must give
the oracle's bytes.  The circuits cover every work-item kind of the streaming kernel:
cross-chunk targets, in-chunk targets 0-1 (partner in the lane), 2-6 (partner in another
lane of the warp), diagonal gates on any in-chunk target, in-chunk controls, and targets
7..kc-1 (general kernel only).
"""
import numpy as np
import pytest

import oracle as O
from paper_1911_04034_gb300 import circuits as Cc

pytestmark = pytest.mark.gpu


def qc():
    from paper_1911_04034_gb300 import qcsim

    return qcsim


def all_images(s):
    return [s.chunk_image(c) for c in range(s.n_chunks)]


def every_target_circuit(n, seed):
    """A random layer to leave the lossless stage, then on every qubit a dense gate,
    T, a gate under an in-chunk control and CZ to the next qubit, in a seeded order."""
    rng = np.random.default_rng(seed)
    g = []
    for q in range(n):
        g.append(Cc.gate(q, Cc.H))
    for q in range(n):
        g.append(Cc.gate(q, [Cc.SX, Cc.SY, Cc.T][int(rng.integers(3))]))
    for q in rng.permutation(n):
        q = int(q)
        g.append(Cc.gate(q, Cc.SY))
        g.append(Cc.gate(q, Cc.T))
        c = (q + 3) % n
        g.append(Cc.gate(q, Cc.SX, {c: 1}))
        g.append(Cc.gate((q + 1) % n, Cc.Z, {q: 1}))
        g.append(Cc.gate(q, Cc.X, {(q + 5) % n: 0}))
    return Cc.to_array(g)


@pytest.mark.parametrize("kc,n", [(7, 12), (8, 13), (10, 14), (11, 14)])
def test_streaming_kernel_every_gate_bit_exact(kc, n):
    """Every gate's images equal the oracle's, with the streaming kernel on."""
    gates = every_target_circuit(n, seed=kc)
    eps = 1e-4
    budget = (16 << n) // 4
    orc = O.CSim(n, n, kc, eps, budget)
    gpu = qc().Sim(n, n, eps, chunk_log2=kc, budget=budget, pool_bytes=2 * (16 << n) + (64 << 20))
    for k in range(len(gates)):
        gpu.apply_gate(gates[k])
        orc.apply(gates[k])
        assert all_images(gpu) == [orc.image(c) for c in range(orc.nchunks)], f"gate {k} target {int(gates[k]['target'])}"
    st = gpu.stats()
    assert st["fast_items"] > 0
    assert st["encoded_bytes"] == orc.stats()["encoded_bytes"]


@pytest.mark.parametrize("eps", [1e-5, 1e-4, 1e-3])
@pytest.mark.parametrize("kc", [7, 9, 10])
def test_streaming_and_general_kernels_write_the_same_bytes(eps, kc):
    """Random circuit, QAOA, QFT and Grover: the same run with the streaming kernel on
    and off gives identical images, counters and amplitudes, and both the oracle's."""
    n = 14
    circuits = [Cc.rcs_n(n, 8, seed=3 + kc), Cc.qaoa_maxcut(n, 2, 3, seed=4)[0], Cc.qft(n, seed=5)[0],
                Cc.grover(n, 2, seed=6)[0]]
    for ci, gates in enumerate(circuits):
        budget = (16 << n) // 4
        sims = []
        for fast in (1, 0):
            s = qc().Sim(n, n, eps, chunk_log2=kc, budget=budget, pool_bytes=2 * (16 << n) + (64 << 20))
            s.set_option("fast_path", fast)
            sims.append(s)
        for k in range(0, len(gates), 17):
            for s in sims:
                s.apply_circuit(gates[k:k + 17])
            assert all_images(sims[0]) == all_images(sims[1]), (ci, k)
        a, b = (s.stats() for s in sims)
        for key in ("encoded_bytes", "max_encoded_bytes", "eps_switch_gate", "chunks_by_mode", "fidelity_lb_sum"):
            assert a[key] == b[key], key
        assert b["fast_items"] == 0
        if ci == 0:
            assert a["fast_items"] > 0
        orc = O.CSim(n, n, kc, eps, budget)
        orc.apply(gates)
        assert all_images(sims[0]) == [orc.image(c) for c in range(orc.nchunks)]
        assert np.array_equal(sims[0].amplitudes().view(np.uint64), orc.amplitudes().view(np.uint64))


def test_streaming_kernel_takes_the_lossy_random_circuit():
    """On a lossy random-circuit state nearly every work item is a STREAM pair the
    streaming kernel finishes; the general kernel sees the rest."""
    n, kc = 16, 10
    gates = Cc.rcs(4, 4, 6, seed=11)
    s = qc().Sim(n, n, 1e-4, chunk_log2=kc, budget=(16 << n) // 4, pool_bytes=2 * (16 << n) + (64 << 20))
    s.apply_circuit(gates[: len(gates) // 2])
    st0 = s.stats()
    s.apply_circuit(gates[len(gates) // 2:])
    st = s.stats()
    done = st["fast_items"] - st0["fast_items"]
    left = st["fast_deferred"] - st0["fast_deferred"]
    assert done > 0 and left <= done // 20
    orc = O.CSim(n, n, kc, 1e-4, (16 << n) // 4)
    orc.apply(gates)
    assert all_images(s) == [orc.image(c) for c in range(orc.nchunks)]


def test_power_of_two_gates_near_the_bottom_of_the_normal_range():
    """sqrt(X) and sqrt(Y) (every coefficient part +-1/2) run as signed sums scaled by
    1/2.  With qubit 3 at |0>, a rotation on it with cos = 1e-300 puts c * a, near
    1e-300 (normal, exponent field below 64), beside every amplitude a: items holding
    such values go to the general kernel, the rest stay on the streaming kernel; the
    images equal the oracle's gate by gate."""
    n, kc, eps = 13, 8, 1e-4
    c = 1e-300
    s_ = np.sqrt(1.0 - c * c)
    g = [Cc.gate(q, Cc.H) for q in range(n) if q != 3]
    g.append(Cc.gate(3, np.array([[c, -s_], [s_, c]], dtype=np.complex128)))
    rng = np.random.default_rng(5)
    for q in rng.permutation(n):
        g.append(Cc.gate(int(q), Cc.SX))
        g.append(Cc.gate(int(q), Cc.SY))
    gates = Cc.to_array(g)
    budget = (16 << n) // 4
    orc = O.CSim(n, n, kc, eps, budget)
    gpu = qc().Sim(n, n, eps, chunk_log2=kc, budget=budget, pool_bytes=2 * (16 << n) + (64 << 20))
    for k in range(len(gates)):
        gpu.apply_gate(gates[k])
        orc.apply(gates[k])
        assert all_images(gpu) == [orc.image(q) for q in range(orc.nchunks)], k
    st = gpu.stats()
    assert st["fast_items"] > 0 and st["fast_deferred"] > 0
