"""GPU simulator parity with the CPU oracle.

* compressed path: every chunk image bit-exact with the oracle's compressed simulator
  after every gate (same controller, Section 3.7; same codec, Section 4.2; same gate
  arithmetic, Eq. matrix1/matrix2), so decoded amplitudes are identical too;
* uncompressed complex128 path: within 1e-12 per amplitude of the oracle's state
  vector (the arithmetic is the same, so in practice equal);
* fidelity (Section 3.8) against the oracle's exact state;
* edge cases: one chunk, the top qubit, many controls, invalid gates.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_1911_04034_gb300 import circuits as Cc

pytestmark = pytest.mark.gpu


def qc():
    from paper_1911_04034_gb300 import qcsim

    return qcsim


def images_equal(gpu, orc):
    bad = [c for c in range(orc.nchunks) if gpu.chunk_image(c) != orc.image(c)]
    return bad


def stats_match(gs, os_):
    assert gs["gates"] == os_["gates"]
    assert gs["encoded_bytes"] == os_["encoded_bytes"]
    assert gs["max_encoded_bytes"] == os_["max_encoded_bytes"]
    assert gs["eps_switch_gate"] == os_["eps_switch_gate"]
    assert gs["sig_bits_current"] == os_["S_current"]
    assert gs["level"] == os_["level"]
    assert gs["fidelity_lb_sum"] == pytest.approx(os_["fid_lb_sum"], abs=1e-12)
    assert gs["fidelity_lb_prod"] == pytest.approx(os_["fid_lb_prod"], rel=1e-12)
    assert gs["chunks_by_mode"][:7] == os_["chunks_by_mode"][:7]
    assert gs["wide_images"] == os_["wide_images"]


@pytest.mark.parametrize("kc", [0, 1, 4, 7, 8, 9, 10, 11])
def test_initial_state_images_match_oracle(kc):
    """|0...0>: chunk 0 holds amplitude 1 coded losslessly, every other chunk is ZERO."""
    n = max(kc + 2, 6)
    gpu = qc().Sim(n, n, 1e-4, chunk_log2=kc, budget=16 << n, pool_bytes=(32 << n) + (16 << 20))
    orc = O.CSim(n, n, kc, 1e-4, 16 << n)
    assert images_equal(gpu, orc) == []


def test_grover_12q_every_gate_bit_exact():
    """Grover search, 12 qubits, one marked item, 50 iterations; blocks of 2^8
    amplitudes; lossless, then lossy at 1e-4 once the budget (raw/4) is reached."""
    n, b, eps = 12, 8, 1e-4
    gates, marked = Cc.grover(n, 50, seed=1)
    budget = (16 << n) // 4
    orc = O.CSim(n, b, 8, eps, budget)
    gpu = qc().Sim(n, b, eps, chunk_log2=8, budget=budget, pool_bytes=2 * (16 << n) + (64 << 20))
    assert images_equal(gpu, orc) == []
    for k in range(len(gates)):
        gpu.apply_gate(gates[k])
        orc.apply(gates[k])
        if k % 7 == 0 or k == len(gates) - 1:
            assert images_equal(gpu, orc) == [], f"after gate {k}"
    stats_match(gpu.stats(), orc.stats())
    st = gpu.stats()
    assert st["eps_switch_gate"] >= 0 and st["eps_current"] == eps
    # fidelity against the exact state (Section 3.8) and the provable bound
    psi = O.sv_init(n)
    O.sv_run(psi, n, gates)
    f = gpu.fidelity(psi)
    a = gpu.amplitudes()
    assert np.array_equal(a, orc.amplitudes())
    assert f["F"] == pytest.approx(O.fidelity(psi, a, n), abs=1e-12)
    assert f["F"] >= st["fidelity_lb_sum"]
    theta = math.asin(2.0 ** (-n / 2))
    assert abs(psi[marked]) ** 2 == pytest.approx(math.sin(101 * theta) ** 2, abs=1e-12)


@pytest.mark.parametrize("eps", [1e-5, 1e-4, 1e-3])
@pytest.mark.parametrize("kc", [4, 7, 10])
def test_random_circuit_bit_exact(eps, kc):
    n = 14
    gates = Cc.rcs(2, 7, 8, seed=int(eps * 1e6) + kc)
    budget = (16 << n) // 3
    orc = O.CSim(n, 10, kc, eps, budget)
    gpu = qc().Sim(n, 10, eps, chunk_log2=kc, budget=budget, pool_bytes=2 * (16 << n) + (64 << 20))
    gpu.apply_circuit(gates)
    orc.apply(gates)
    assert images_equal(gpu, orc) == []
    stats_match(gpu.stats(), orc.stats())
    assert np.array_equal(gpu.amplitudes().view(np.uint64), orc.amplitudes().view(np.uint64))


@pytest.mark.parametrize("kc,n", [(0, 8), (1, 9), (2, 10), (11, 14), (11, 16)])
def test_extreme_chunk_sizes_bit_exact(kc, n):
    """One- to four-amplitude chunks (one value per thread, most threads idle) and the
    largest chunks (16 values per thread, one CTA per SM), over a circuit with both
    in-chunk and cross-chunk targets and a lossy switch."""
    gates = Cc.rcs_n(n, 6, seed=40 + kc)
    budget = (16 << n) // 4
    b = min(n, max(kc, 6))
    orc = O.CSim(n, b, kc, 1e-4, budget)
    gpu = qc().Sim(n, b, 1e-4, chunk_log2=kc, budget=budget, pool_bytes=4 * (16 << n) + (64 << 20))
    gpu.apply_circuit(gates)
    orc.apply(gates)
    assert images_equal(gpu, orc) == []
    stats_match(gpu.stats(), orc.stats())
    assert gpu.stats()["eps_switch_gate"] >= 0


def test_subnormal_amplitudes_in_the_fused_kernel():
    """Chunks holding subnormal amplitudes are coded at 64 bits in a lossy run, the
    others at the bound; the images equal the oracle's."""
    from test_oracle_sim import subnormal_circuit

    n, kc = 10, 4
    gates = subnormal_circuit()
    orc = O.CSim(n, n, kc, 1e-4, 1)
    gpu = qc().Sim(n, n, 1e-4, chunk_log2=kc, budget=1, pool_bytes=4 * (16 << n) + (16 << 20))
    for k in range(len(gates)):
        gpu.apply_circuit(gates[k:k + 1])
        orc.apply(gates[k:k + 1])
        assert images_equal(gpu, orc) == [], k
    stats_match(gpu.stats(), orc.stats())
    widths = {gpu.chunk_image(q)[1] for q in range(gpu.n_chunks)}
    assert widths == {0, 26, 64}  # 0: ZERO chunks (qubit 9 is never touched)


def paired_subnormal_circuit():
    """Like test_oracle_sim.subnormal_circuit, for chunks of 2^7 amplitudes: the rotation
    with cos = 1e-310 runs under a control on qubit 7 (bit 0 of the chunk index), so in a
    work item of an in-chunk gate one chunk holds subnormal amplitudes and its partner
    none, while a cross-chunk gate on qubits 8-11 pairs two chunks of the same kind.
    Qubit 0 is not touched again, so the subnormals survive."""
    c = 1e-310
    U = np.array([[c, -1.0], [1.0, c]], dtype=np.complex128)
    g = [Cc.gate(7, Cc.H), Cc.gate(0, U, {7: 1}), Cc.gate(1, Cc.H), Cc.gate(8, Cc.H), Cc.gate(2, Cc.H),
         Cc.gate(9, Cc.SX), Cc.gate(3, Cc.H), Cc.gate(4, Cc.SX), Cc.gate(10, Cc.H), Cc.gate(5, Cc.T),
         Cc.gate(6, Cc.SY), Cc.gate(11, Cc.H), Cc.gate(2, Cc.SY), Cc.gate(9, Cc.T)]
    return Cc.to_array(g)


def test_subnormal_chunk_beside_a_normal_one_in_a_work_item():
    """Chunks of 2^7 amplitudes, where both chunks of a work item decode and encode in one
    pass: an item holding a subnormal chunk falls back to chunk-by-chunk coding (the
    subnormal chunk at 64 bits, its partner at the bound), and every image equals the
    oracle's after every gate."""
    n, kc = 12, 7
    gates = paired_subnormal_circuit()
    orc = O.CSim(n, n, kc, 1e-4, 1)
    gpu = qc().Sim(n, n, 1e-4, chunk_log2=kc, budget=1, pool_bytes=4 * (16 << n) + (16 << 20))
    for k in range(len(gates)):
        gpu.apply_circuit(gates[k:k + 1])
        orc.apply(gates[k:k + 1])
        assert images_equal(gpu, orc) == [], k
    stats_match(gpu.stats(), orc.stats())
    widths = [gpu.chunk_image(q)[1] for q in range(gpu.n_chunks)]
    assert {w for q, w in enumerate(widths) if q & 1} == {64}
    assert {w for q, w in enumerate(widths) if not q & 1} == {O.sig_bits(1e-4)}


@pytest.mark.parametrize("kc", [8, 10])
def test_paired_and_chunk_by_chunk_coding_agree(kc):
    """Tracing selector records switches the fused kernel to chunk-by-chunk encoding (one
    record per chunk encode, here with the Solution C modes); the images must not
    change.  Random circuit, Grover and QAOA states (STREAM, CONST, PERIOD, ZERO chunks
    side by side)."""
    n, eps = 14, 1e-4
    circuits = [Cc.rcs_n(n, 6, seed=70 + kc), Cc.grover(n, 1, seed=71)[0], Cc.qaoa_maxcut(n, 1, 3, seed=72)[0]]
    for gates in circuits:
        sims = []
        for tracing in (False, True):
            s = qc().Sim(n, n, eps, chunk_log2=kc, budget=(16 << n) // 4, pool_bytes=2 * (16 << n) + (32 << 20))
            if tracing:
                s.trace(1 << 10)
            sims.append(s)
        for k in range(0, len(gates), 25):
            for s in sims:
                s.apply_circuit(gates[k:k + 25])
            a, b = sims
            assert [a.chunk_image(c) for c in range(a.n_chunks)] == [b.chunk_image(c) for c in range(b.n_chunks)], k
        recs = sims[1].trace_read()
        assert 0 < recs.shape[0] <= 1 << 10
        assert set(np.unique(recs[:, 16]).astype(int)) <= {0, 1, 2, 3, 4}
        orc = O.CSim(n, n, kc, eps, (16 << n) // 4)
        orc.apply(gates)
        assert images_equal(sims[0], orc) == []


def test_loschmidt_echo_matches_oracle_and_bound():
    """QAOA then its inverse, compressed at 1e-4 (guarded ladder, budget raw/4): the
    images equal the oracle's, and the amplitude of |0...0> is at least 1 - sum(delta)
    (Section 3.8 reading) but below 1.  The benchmark runs the same check at 34 qubits."""
    n, kc, eps = 16, 8, 1e-4
    gates, _ = Cc.qaoa_maxcut(n, 2, 3, seed=12)
    echo = np.concatenate([gates, Cc.inverse(gates)])
    budget = (16 << n) // 4
    gpu = qc().Sim(n, n, eps, chunk_log2=kc, budget=budget, ladder=2, pool_bytes=2 * (16 << n) + (32 << 20))
    gpu.apply_circuit(echo)
    orc = O.CSim(n, n, kc, eps, budget, ladder=2)
    orc.apply(echo)
    assert images_equal(gpu, orc) == []
    stats_match(gpu.stats(), orc.stats())
    a0 = abs(gpu.amplitudes(0, 1)[0])
    assert gpu.stats()["fidelity_lb_sum"] - 1e-12 <= a0 < 1.0


@pytest.mark.parametrize("ladder", [0, 1, 2])
def test_qaoa_and_qft_bit_exact(ladder):
    n = 12
    qa, _ = Cc.qaoa_maxcut(n, 2, 3, seed=5)
    qf, _ = Cc.qft(n, seed=4)
    for gates, eps in ((qa, 1e-2), (qf, 1e-3)):
        budget = (16 << n) // 5
        orc = O.CSim(n, 7, 6, eps, budget, ladder=ladder)
        gpu = qc().Sim(n, 7, eps, chunk_log2=6, budget=budget, ladder=ladder, pool_bytes=2 * (16 << n) + (64 << 20))
        gpu.apply_circuit(gates)
        orc.apply(gates)
        assert images_equal(gpu, orc) == []
        stats_match(gpu.stats(), orc.stats())


def test_guarded_ladder_switches_mid_run_like_the_oracle():
    """Ladder 2 with a budget that admits the lossless stage at first: the level rises
    when a gate's worst case (controlled gates rewrite half the chunks) stops fitting;
    every gate's images and the controller state match the oracle's."""
    n, kc = 14, 6
    gates, _ = Cc.qaoa_maxcut(n, 2, 3, seed=9)
    nch = 1 << (n - kc)
    raw_img = 16 + 8 * (2 << kc)
    budget = -(-nch * raw_img * 10 // 9) + 1
    orc = O.CSim(n, n, kc, 1e-3, budget, ladder=2)
    gpu = qc().Sim(n, n, 1e-3, chunk_log2=kc, budget=budget, ladder=2, pool_bytes=2 * (16 << n) + (64 << 20))
    levels = []
    for k in range(0, len(gates), 16):
        gpu.apply_circuit(gates[k:k + 16])
        orc.apply(gates[k:k + 16])
        assert images_equal(gpu, orc) == []
        stats_match(gpu.stats(), orc.stats())
        levels.append(gpu.stats()["level"])
    assert levels[0] == 0 and levels[-1] > 0


@pytest.mark.parametrize("thresh", [12000, 15000, 17500])
def test_guarded_ladder_counts_subnormal_chunks_like_the_oracle(thresh):
    """Ladder 2 on a random state whose chunks all come to hold subnormals (coded at 64
    bits at any level): the gate with the subnormal coefficient and every later gate
    count the 64-bit images at RAW size, as the oracle does; images, the 64-bit image
    count and the controller state match gate by gate."""
    from test_oracle_sim import wide_chunk_circuit

    n, kc = 10, 4
    gates = wide_chunk_circuit()
    budget = -(-thresh * 10 // 9)
    orc = O.CSim(n, n, kc, 1e-4, budget, ladder=2)
    gpu = qc().Sim(n, n, 1e-4, chunk_log2=kc, budget=budget, ladder=2, pool_bytes=64 << 20)
    for g in gates:
        gpu.apply_circuit([g])
        orc.apply([g])
        assert images_equal(gpu, orc) == []
        stats_match(gpu.stats(), orc.stats())
    assert gpu.stats()["wide_images"] == 1 << (n - kc)


def test_solution_d_mode_bit_exact():
    """SPLIT (Solution D) enabled on both sides: real-valued Grover states favour it."""
    n = 11
    gates, _ = Cc.grover(n, 6, seed=3)
    rc = Cc.rcs(1, 11, 4, seed=2)
    for circ, eps in ((gates, 1e-4), (rc, 1e-3)):
        budget = (16 << n) // 5
        orc = O.CSim(n, 8, 7, eps, budget, modes=0x3F)
        gpu = qc().Sim(n, 8, eps, chunk_log2=7, budget=budget, pool_bytes=64 << 20)
        gpu.set_modes(0x3F)
        gpu.apply_circuit(circ)
        orc.apply(circ)
        assert images_equal(gpu, orc) == []
        stats_match(gpu.stats(), orc.stats())


def test_lossless_equals_exact_state():
    n = 13
    gates = Cc.rcs(1, 13, 6, seed=3)
    psi = O.sv_init(n)
    O.sv_run(psi, n, gates)
    gpu = qc().Sim(n, 13, 0.0, chunk_log2=9)
    gpu.apply_circuit(gates)
    a = gpu.amplitudes()
    assert np.array_equal(a, psi)  # values equal; a -0 may be stored as +0
    assert gpu.stats()["sig_bits_current"] == 64
    assert gpu.fidelity(psi)["F"] == pytest.approx(1.0, abs=1e-12)


@pytest.mark.parametrize("n", [10, 16])
def test_uncompressed_path_within_1e12(n):
    """The uncompressed comparator equals the oracle's state vector bit for bit: random
    circuit (T and CZ leave one or three amplitudes of four untouched, which the kernel
    neither reads nor writes), Grover (multi-controlled Z, X) and QAOA (RZ, CNOT, RX)."""
    for gates in (Cc.rcs_n(n, 8, seed=n), Cc.grover(n, 2, seed=n)[0], Cc.qaoa_maxcut(n, 1, 3, seed=n)[0]):
        psi = O.sv_init(n)
        O.sv_run(psi, n, gates)
        sv = qc().StateVector(n)
        sv.apply_circuit(gates)
        got = sv.amplitudes()
        assert np.max(np.abs(got - psi)) <= 1e-12
        assert np.array_equal(got, psi)


def test_edge_shapes_and_controls():
    rng = np.random.default_rng(2)
    # single chunk (n == kc), one and two qubits, the top qubit, multi-controls with
    # controls below and above the chunk boundary
    for n, kc in ((1, 1), (2, 2), (3, 1), (5, 5), (9, 3), (11, 4)):
        gs = []
        for _ in range(30):
            t = int(rng.integers(0, n))
            others = [q for q in range(n) if q != t]
            ctrl = {int(q): int(rng.integers(0, 2)) for q in rng.choice(others, size=min(len(others), int(rng.integers(0, 4))), replace=False)} if others else {}
            z = rng.standard_normal((2, 2)) + 1j * rng.standard_normal((2, 2))
            q, r = np.linalg.qr(z)
            U = [q * (np.diag(r) / np.abs(np.diag(r))), Cc.H, Cc.X, Cc.T, Cc.Z][int(rng.integers(0, 5))]
            gs.append(Cc.gate(t, U, ctrl))
        gs.append(Cc.gate(n - 1, Cc.H, {q: 1 for q in range(n - 1)}))
        gates = Cc.to_array(gs)
        for eps in (0.0, 1e-3):
            # eps > 0: threshold 0, so both sides run every gate lossy
            orc = O.CSim(n, n, kc, eps, 1 if eps else 1 << 40)
            gpu = qc().Sim(n, n, eps, chunk_log2=kc, budget=1 if eps else 1 << 40, pool_bytes=64 << 20)
            gpu.apply_circuit(gates)
            orc.apply(gates)
            assert images_equal(gpu, orc) == [], (n, kc, eps)


def test_invalid_gates_rejected_state_unchanged():
    n = 6
    gpu = qc().Sim(n, 6, 1e-4, chunk_log2=3)
    gpu.apply_circuit(Cc.h_all(n))
    before = gpu.amplitudes().copy()
    bad = [Cc.gate(6, Cc.H), Cc.gate(1, Cc.H, {1: 1}), Cc.gate(0, 2 * Cc.H), Cc.gate(0, Cc.H, {9: 1})]
    g = Cc.gate(0, Cc.H)
    g["u"][3] = np.inf
    bad.append(g)
    for b in bad:
        with pytest.raises(qc().SimError) as ei:
            gpu.apply_gate(b)
        assert ei.value.code == qc().ERR_INVALID
    # a batch with one bad gate applies none of them
    with pytest.raises(qc().SimError):
        gpu.apply_circuit(Cc.to_array([Cc.gate(0, Cc.X), bad[0]]))
    assert np.array_equal(gpu.amplitudes(), before)


def test_measure_matches_oracle():
    n = 10
    gates = Cc.rcs(2, 5, 6, seed=11)
    psi = O.sv_init(n)
    O.sv_run(psi, n, gates)
    gpu = qc().Sim(n, 10, 0.0, chunk_log2=6)
    gpu.apply_circuit(gates)
    p = np.abs(psi) ** 2
    cum = np.cumsum(p)
    agree = 0
    for seed in range(300):
        o_gpu, pr_gpu = gpu.measure(seed)
        o_orc, pr_orc = O.sv_measure(psi, n, seed)
        u = (O.splitmix64(seed) >> 11) * 2.0 ** -53
        near = np.min(np.abs(cum - u * cum[-1])) < 1e-12
        if not near:
            assert o_gpu == o_orc
            assert pr_gpu == pytest.approx(pr_orc, rel=1e-12)
            agree += 1
    assert agree > 290


def test_oom_poisons_handle():
    n = 16
    gpu = qc().Sim(n, 16, 0.0, chunk_log2=10, budget=1 << 20, pool_bytes=256 << 10)  # lossless, 256 KiB pool
    with pytest.raises(qc().SimError) as ei:
        gpu.apply_circuit(Cc.rcs_n(n, 4, seed=1))
    assert ei.value.code == qc().ERR_OOM
    with pytest.raises(qc().SimError) as ei:
        gpu.apply_gate(Cc.gate(0, Cc.H))
    assert ei.value.code == qc().ERR_STATE


def test_oom_in_the_lossy_stage_poisons_handle():
    """A lossy random circuit whose state outgrows a 4 MiB pool: the streaming kernel runs
    (one CTA fits the pool's page-cache cap) and the pool runs dry in one of the gate
    kernels; the failed reservation is given back, the bookkeeping kernel skips the stack,
    and the call reports SIM_ERR_OOM, later calls SIM_ERR_STATE."""
    n = 20
    gpu = qc().Sim(n, n, 1e-4, chunk_log2=10, budget=1, pool_bytes=4 << 20)
    with pytest.raises(qc().SimError) as ei:
        gpu.apply_circuit(Cc.rcs_n(n, 6, seed=2))
    assert ei.value.code == qc().ERR_OOM
    with pytest.raises(qc().SimError) as ei:
        gpu.apply_gate(Cc.gate(0, Cc.H))
    assert ei.value.code == qc().ERR_STATE
    ok = qc().Sim(12, 12, 1e-4, chunk_log2=8)  # the context is still usable
    ok.apply_circuit(Cc.rcs_n(12, 3, seed=3))


def _oracle_pair_check(gpu, gate, before_imgs, chunks, eps, kc):
    """Oracle applied to the sampled chunks alone: a state of kc+1 qubits made of the
    two chunks, the gate's target and controls remapped onto it."""
    t = int(gate["target"])
    mask, vals = int(gate["ctrl_mask"]), int(gate["ctrl_vals"])
    lo = (1 << kc) - 1
    if t >= kc:
        tt = kc
    else:
        tt = t
    g2 = Cc.gate(tt, Cc.matrix_of(gate), {q: (vals >> q) & 1 for q in range(kc) if (mask >> q) & 1})
    orc = O.CSim(kc + 1, kc + 1, kc, eps, budget=1 if eps else (1 << 40))
    for k, c in enumerate(chunks):
        orc.set_image(k, before_imgs[c])
    orc.apply(g2)
    return [orc.image(k) for k in range(len(chunks))]


@pytest.mark.parametrize("modes", [0x5F, 0x7F])
def test_palette_mode_bit_exact(modes):
    """PALETTE (and with 0x7F also SPLIT) enabled on both sides: Grover's few-valued
    states take PALETTE images in the lossless and the lossy stage; random-circuit and
    QAOA states mostly do not.  Every image equals the oracle's."""
    n = 12
    grover, _ = Cc.grover(n, 4, seed=8)
    rc = Cc.rcs(3, 4, 4, seed=9)
    qa, _ = Cc.qaoa_maxcut(n, 1, 3, seed=10)
    seen = set()
    for circ, eps, kc in ((grover, 1e-4, 8), (grover, 0.0, 10), (rc, 1e-3, 7), (qa, 1e-4, 9)):
        budget = (16 << n) // 5
        orc = O.CSim(n, 10, kc, eps, budget, modes=modes)
        gpu = qc().Sim(n, 10, eps, chunk_log2=kc, budget=budget, pool_bytes=64 << 20)
        gpu.set_modes(modes)
        for k in range(0, len(circ), 9):
            gpu.apply_circuit(circ[k:k + 9])
            orc.apply(circ[k:k + 9])
            assert images_equal(gpu, orc) == [], k
            seen |= {gpu.chunk_image(c)[0] for c in range(gpu.n_chunks)}
        stats_match(gpu.stats(), orc.stats())
    assert 6 in seen


def test_full_size_30q_sampled_chunks():
    """Random circuit on 30 qubits (5 x 6 grid) with blocks of 2^20 amplitudes at
    1e-4, the configuration the benchmark times: after the Hadamard layer and two
    random layers, sampled chunk pairs of the next gates are recomputed by the oracle
    from their pre-gate images and must match the GPU's post-gate images bit for bit."""
    n, b, eps = 30, 20, 1e-4
    gates = Cc.rcs(5, 6, 4, seed=2024)
    raw = 16 << n
    gpu = qc().Sim(n, b, eps, chunk_log2=10, budget=raw // 4, pool_bytes=raw + raw // 8)
    kc = gpu.chunk_log2
    warm = 30 + 2 * (30 + 12)
    gpu.apply_circuit(gates[:warm])
    st = gpu.stats()
    assert st["sig_bits_current"] in (64, O.sig_bits(eps))
    rng = np.random.default_rng(5)
    checked = 0
    for g in gates[warm: warm + 6]:
        t = int(g["target"])
        hi_mask, hi_vals = int(g["ctrl_mask"]) >> kc, int(g["ctrl_vals"]) >> kc
        S_before = gpu.stats()
        picks = []
        while len(picks) < 3:
            q = int(rng.integers(0, gpu.n_chunks))
            if (q & hi_mask) != hi_vals:
                continue
            if t >= kc:
                q &= ~(1 << (t - kc))
                picks.append((q, q | (1 << (t - kc))))
            else:
                picks.append((q, q ^ 1) if ((q ^ 1) & hi_mask) == hi_vals else (q,))
        before = {c: gpu.chunk_image(c) for p in picks for c in p}
        gpu.apply_gate(g)
        st = gpu.stats()
        eps_used = st["eps_current"]
        for p in picks:
            want = _oracle_pair_check(gpu, g, before, list(p), eps_used, kc)
            for k, c in enumerate(p):
                assert gpu.chunk_image(c) == want[k], (int(g["target"]), c)
                checked += 1
        del S_before
    assert checked >= 18
