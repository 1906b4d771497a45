"""Pins of the oracle's simulators against mathematics that does not come from it.

* gate semantics (Section 3.1, Eq. matrix1/matrix2; Eq. psi3) against full 2^n x 2^n
  Kronecker-product unitaries built with numpy, n <= 6;
* Grover's success probability sin^2((2k+1) theta), theta = asin(2^(-n/2));
* QFT of a basis state |x> -> sum_k exp(2 pi i x k / 2^n) |k> / 2^(n/2);
* norm conservation (Eq. psi), the truncation interval after every gate (Section 3.7),
  the fidelity lower bound (Section 3.8), the controller rule (Section 3.7 with
  Eq. totalnbBytes), the error statistics of Section 4.2 (bounded, uncorrelated);
* QAOA gate counts of Table 2 (42 and 43 qubits, p = 1, 4-regular graphs).
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_1911_04034_gb300 import circuits as Cc


def kron_all(factors):
    out = np.array([[1.0 + 0j]])
    for f in factors:
        out = np.kron(out, f)
    return out


def full_unitary(g, n):
    """A = I (x) ... (x) U (x) ... (x) I (Eq. psi3, qubit n-1 leftmost), generalised to
    controls as A = I + K(U) - K(I), where K(V) puts the projector |v><v| on every
    control qubit, V on the target and I elsewhere."""
    U = Cc.matrix_of(g)
    t, mask, vals = int(g["target"]), int(g["ctrl_mask"]), int(g["ctrl_vals"])
    P = [np.diag([1.0, 0.0]).astype(complex), np.diag([0.0, 1.0]).astype(complex)]
    I2 = np.eye(2, dtype=complex)

    def K(V):
        fs = []
        for q in reversed(range(n)):
            if q == t:
                fs.append(V)
            elif (mask >> q) & 1:
                fs.append(P[(vals >> q) & 1])
            else:
                fs.append(I2)
        return kron_all(fs)

    return np.eye(1 << n, dtype=complex) + K(U) - K(I2)


def random_unitary(rng):
    z = rng.standard_normal((2, 2)) + 1j * rng.standard_normal((2, 2))
    q, r = np.linalg.qr(z)
    return q * (np.diag(r) / np.abs(np.diag(r)))


def random_gate(rng, n):
    t = int(rng.integers(0, n))
    others = [q for q in range(n) if q != t]
    nc = int(rng.integers(0, min(3, len(others)) + 1))
    ctrl = {int(q): int(rng.integers(0, 2)) for q in rng.choice(others, size=nc, replace=False)} if nc else {}
    kind = rng.integers(0, 4)
    U = [random_unitary(rng), Cc.H, Cc.T, Cc.X][kind]
    return Cc.gate(t, U, ctrl)


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6])
def test_bruteforce_unitary(n):
    rng = np.random.default_rng(n)
    gates = Cc.to_array([random_gate(rng, n) for _ in range(25)])
    psi0 = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
    psi0 /= np.linalg.norm(psi0)
    ref = psi0.copy()
    for g in gates:
        ref = full_unitary(g, n) @ ref
    got = psi0.copy()
    O.sv_run(got, n, gates)
    assert np.max(np.abs(got - ref)) < 1e-13


def test_grover_closed_form_n12_k50():
    n, k = 12, 50
    gates, marked = Cc.grover(n, k, seed=1)
    assert len(gates) == n + k * (4 * n + 2) == 2512
    psi = O.sv_init(n)
    O.sv_run(psi, n, gates)
    theta = math.asin(2.0 ** (-n / 2))
    p = math.sin((2 * k + 1) * theta) ** 2
    assert abs(p - 0.99994535) < 1e-8
    assert abs(abs(psi[marked]) ** 2 - p) < 1e-12
    assert abs(O.sv_norm2(psi, n) - 1.0) < 1e-12


@pytest.mark.parametrize("k", [1, 3, 7])
def test_grover_amplitudes_every_item(k):
    n = 8
    gates, marked = Cc.grover(n, k, seed=11)
    psi = O.sv_init(n)
    O.sv_run(psi, n, gates)
    theta = math.asin(2.0 ** (-n / 2))
    # the diffusion H X MCZ X H equals -(2|s><s| - I): amplitudes carry (-1)^k
    sgn = (-1) ** k
    a_m = sgn * math.sin((2 * k + 1) * theta)
    a_o = sgn * math.cos((2 * k + 1) * theta) / math.sqrt((1 << n) - 1)
    expect = np.full(1 << n, a_o, dtype=complex)
    expect[marked] = a_m
    assert np.max(np.abs(psi - expect)) < 1e-12


@pytest.mark.parametrize("n,seed", [(5, 1), (8, 2), (10, 3)])
def test_qft_of_basis_state(n, seed):
    gates, x = Cc.qft(n, seed)
    psi = O.sv_init(n)
    O.sv_run(psi, n, gates)
    N = 1 << n
    k = np.arange(N)
    expect = np.exp(2j * np.pi * x * k / N) / math.sqrt(N)
    assert np.max(np.abs(psi - expect)) < 1e-12


def test_norm_conservation_rcs():
    n = 12
    gates = Cc.rcs(3, 4, 10, seed=5)
    psi = O.sv_init(n)
    O.sv_run(psi, n, gates)
    assert abs(O.sv_norm2(psi, n) - 1.0) < 1e-12


@pytest.mark.parametrize("family", ["rcs", "qaoa", "qft"])
def test_inverse_circuit_returns_to_the_start(family):
    """circuits.inverse: U then U^dagger on the exact state vector gives back |0...0>
    (Loschmidt echo without compression) up to rounding."""
    n = 10
    gates = {"rcs": lambda: Cc.rcs(2, 5, 8, seed=3), "qaoa": lambda: Cc.qaoa_maxcut(n, 2, 3, seed=3)[0],
             "qft": lambda: Cc.qft(n, seed=3)[0]}[family]()
    psi = O.sv_init(n)
    O.sv_run(psi, n, gates)
    assert abs(psi[0]) < 0.5  # the forward circuit leaves |0...0>
    O.sv_run(psi, n, Cc.inverse(gates))
    assert abs(psi[0] - 1.0) < 1e-12
    assert np.max(np.abs(psi[1:])) < 1e-12


@pytest.mark.parametrize("eps", [1e-4, 1e-3])
def test_compressed_echo_bound(eps):
    """Section 3.8 reading: each lossy encode moves the state by at most delta, and the
    inverse circuit is unitary, so after U and U^dagger run compressed the amplitude of
    |0...0> is at least 1 - sum(delta) over both halves; it is below 1 because the
    compression did lose something."""
    n, kc = 12, 6
    gates, _ = Cc.qaoa_maxcut(n, 2, 3, seed=5)
    cs = O.CSim(n, n, kc, eps, budget=1)
    cs.apply(gates)
    cs.apply(Cc.inverse(gates))
    a0 = abs(cs.amplitudes()[0])
    st = cs.stats()
    assert st["fid_lb_sum"] == pytest.approx(1.0 - 2 * len(gates) * 2.0 ** O.exp_of(eps), rel=1e-12)
    assert st["fid_lb_sum"] - 1e-12 <= a0 < 1.0


def test_qaoa_gate_counts_table2():
    # Table 2: QAOA with 42 and 43 qubits uses 336 and 344 gates; one round (p = 1)
    # on a 4-regular graph with CNOT-RZ-CNOT cost terms gives n + 3 (2n) + n.
    for n, expect in ((42, 336), (43, 344)):
        gates, edges = Cc.qaoa_maxcut(n, 1, 4, seed=n)
        assert len(edges) == 2 * n
        assert len(gates) == expect


def test_gate_check_rejects():
    n = 4
    good = Cc.gate(1, Cc.H, {2: 1})
    assert O.gate_check(good, n) == 0
    bad = [Cc.gate(4, Cc.H), Cc.gate(1, Cc.H, {1: 1}), Cc.gate(0, 2 * Cc.H), Cc.gate(0, Cc.H, {7: 0})]
    g = Cc.gate(0, Cc.H)
    g["u"][0] = np.nan
    bad.append(g)
    g = Cc.gate(0, Cc.H, {1: 1})
    g["ctrl_vals"] = 1 << 3
    bad.append(g)
    for b in bad:
        assert O.gate_check(b, n) < 0


# ------------------------------------------------- compressed simulator --- #

def run_lossless_vs_sv(n, gates, b, kc):
    psi = O.sv_init(n)
    O.sv_run(psi, n, gates)
    cs = O.CSim(n, b, kc, 0.0, budget=1 << 40)
    cs.apply(gates)
    a = cs.amplitudes()
    return psi, a, cs


@pytest.mark.parametrize("kc", [2, 4, 6])
def test_lossless_equals_state_vector(kc):
    n = 9
    gates = Cc.rcs(3, 3, 6, seed=9)
    psi, a, cs = run_lossless_vs_sv(n, gates, b=7, kc=kc)
    # same arithmetic, lossless codec: equal values (a -0 may be stored as +0)
    assert np.array_equal(psi, a)
    assert cs.stats()["S_current"] == 64
    assert abs(O.fidelity(psi, a, n) - 1.0) < 1e-12


def test_lossy_interval_after_every_gate():
    """Section 3.7: each decoded value is the truncation of the value the gate
    produced; |x - t| < 2^(12-S) |x|, |t| <= |x|."""
    n, kc = 8, 4
    gates = Cc.rcs(2, 4, 4, seed=3)
    cs = O.CSim(n, 6, kc, 1e-3, budget=1)  # tiny budget: lossy from the first gate
    S = O.sig_bits(1e-3)
    prev = cs.amplitudes()
    for g in gates:
        x = prev.copy()
        O.sv_run(x, n, g)
        cs.apply(g)
        cur = cs.amplitudes()
        xb, tb = x.view(np.float64), cur.view(np.float64)
        nz = xb != 0
        assert np.all(np.abs(tb) <= np.abs(xb))
        assert np.all(np.abs(xb - tb)[nz] < 2.0 ** (12 - S) * np.abs(xb)[nz])
        assert np.all(tb[~nz] == 0)
        prev = cur
    st = cs.stats()
    assert st["eps_switch_gate"] == 0 and st["S_current"] == S


@pytest.mark.parametrize("eps", [1e-5, 1e-3, 1e-1])
def test_fidelity_lower_bound(eps):
    n = 10
    gates = Cc.rcs(2, 5, 8, seed=4)
    psi = O.sv_init(n)
    O.sv_run(psi, n, gates)
    cs = O.CSim(n, 8, 6, eps, budget=1)
    cs.apply(gates)
    a = cs.amplitudes()
    F = O.fidelity(psi, a, n)
    st = cs.stats()
    delta = 2.0 ** O.exp_of(eps)
    assert st["fid_lb_sum"] == pytest.approx(1.0 - len(gates) * delta, rel=1e-12)
    assert F >= st["fid_lb_sum"] - 1e-12
    assert F <= 1.0 + 1e-12
    assert O.sv_norm2(a, n) <= 1.0 + 1e-12  # truncation never grows a magnitude


def test_controller_switch_rule():
    """Before each gate: relax when E + 2 * (raw block bytes) > floor(tau * B)."""
    n, b, kc = 10, 6, 4
    gates = Cc.rcs(2, 5, 6, seed=8)
    B = (16 << n) // 4
    thresh = math.floor(0.9 * B)
    W = 2 * (16 << b)
    cs = O.CSim(n, b, kc, 1e-4, budget=B)
    expect_switch = None
    for k, g in enumerate(gates):
        E = cs.stats()["encoded_bytes"]
        if expect_switch is None and E + W > thresh:
            expect_switch = k
        cs.apply(g)
        st = cs.stats()
        if expect_switch is None:
            assert st["S_current"] == 64
        else:
            assert st["S_current"] == O.sig_bits(1e-4)
    assert expect_switch is not None
    assert cs.stats()["eps_switch_gate"] == expect_switch


def test_paper_ladder_one_level_per_gate():
    n = 8
    gates = Cc.rcs(2, 4, 4, seed=2)
    cs = O.CSim(n, 6, 4, 1e-2, budget=1, ladder=O.LADDER_PAPER)
    seen = []
    for g in gates[:5]:
        cs.apply(g)
        seen.append(cs.stats()["eps_current"])
    assert seen == [1e-5, 1e-4, 1e-3, 1e-2, 1e-2]


def _format_max_image(kc, S):
    """Largest image the format allows at S bits: 16-byte header, one 2-bit code per
    value padded to 16 bytes, S residual bits per value padded to 16 bytes -- or the
    verbatim values (RAW) when that is smaller."""
    N = 2 << kc
    codes = -(-(-(-N // 4)) // 16) * 16
    resid = -(-(S * N) // 128) * 16
    return min(16 + codes + resid, 16 + 8 * N)


@pytest.mark.parametrize("kc", [2, 6, 10])
def test_largest_image_bound_is_attained_and_never_exceeded(kc):
    """Positive real and negative imaginary parts: in the interleaved order every value
    differs from its predecessor in the sign bit, so all take code 0 and all S bits
    and STREAM reaches the bound; no other chunk exceeds it."""
    A = 1 << kc
    rng = np.random.default_rng(kc)
    worst = rng.uniform(1, 2, A) - 1j * rng.uniform(1, 2, A)
    for S in (13, 22, 26, 29, 40, 64):
        bound = _format_max_image(kc, S)
        assert len(O.encode_chunk(worst, kc, S)) == bound
        for _ in range(5):
            a = (rng.standard_normal(A) + 1j * rng.standard_normal(A)) * 2.0 ** rng.integers(-30, 30, A)
            assert len(O.encode_chunk(a, kc, S)) <= bound


def test_guarded_ladder_picks_the_smallest_level_that_fits():
    """Ladder 2 before an uncontrolled gate: the smallest level whose largest images on
    every chunk fit floor(tau * budget)."""
    n, b, kc, tau = 10, 10, 4, 0.9
    nch = 1 << (n - kc)
    levels = [(1e-5, 29), (1e-4, 26), (1e-3, 22)]
    g = Cc.gate(0, Cc.H)
    for want in range(4):
        S_fit = 64 if want == 0 else levels[want - 1][1]
        # the budget admits exactly level `want` (and every level after it)
        budget = math.ceil(nch * _format_max_image(kc, S_fit) / tau) + 1
        cs = O.CSim(n, b, kc, 1e-3, budget=budget, tau=tau, ladder=2)
        cs.apply([g])
        st = cs.stats()
        assert st["level"] == want
        if want:
            assert st["S_current"] == S_fit and st["eps_switch_gate"] == 0
        else:
            assert st["S_current"] == 64 and st["eps_switch_gate"] == -1
    # nothing fits: the largest bound
    cs = O.CSim(n, b, kc, 1e-3, budget=16, tau=tau, ladder=2)
    cs.apply([g])
    assert cs.stats()["S_current"] == 22


def test_guarded_ladder_keeps_the_state_under_the_threshold():
    """QAOA (CNOTs with controls on chunk bits rewrite half the chunks): whenever the
    largest level fits, every gate ends with E <= floor(tau * budget)."""
    n, kc = 12, 6
    gates, _ = Cc.qaoa_maxcut(n, 2, 3, seed=5)
    nch = 1 << (n - kc)
    budget = math.ceil(nch * _format_max_image(kc, 64) / 0.9) + 1  # lossless fits at first
    thresh = math.floor(0.9 * budget)
    cs = O.CSim(n, n, kc, 1e-3, budget=budget, ladder=2)
    levels = []
    for g in gates:
        cs.apply([g])
        st = cs.stats()
        assert st["encoded_bytes"] <= thresh
        levels.append(st["level"])
    assert levels == sorted(levels)  # the bound never tightens
    assert levels[0] == 0 and levels[-1] > 0


def wide_chunk_circuit():
    """A random circuit on qubits 0-2 and 4-9 (qubit 3 stays |0>) makes every amplitude
    look random; a rotation on qubit 3 with cos = 1e-310 (subnormal; the matrix is
    unitary to the last bit) then puts c * a, a subnormal, beside every amplitude a, so
    each 16-amplitude chunk (qubits 0-3) holds random normal values and subnormals;
    a random circuit on qubits 0-2 after it pairs subnormals with subnormals and
    normals with normals, so every chunk keeps both."""
    rest = [0, 1, 2, 4, 5, 6, 7, 8, 9]

    def remap(gates, qubits):
        out = gates.copy()
        for rec in out:
            rec["target"] = qubits[int(rec["target"])]
            m, v = int(rec["ctrl_mask"]), int(rec["ctrl_vals"])
            rec["ctrl_mask"] = sum(1 << qubits[q] for q in range(len(qubits)) if (m >> q) & 1)
            rec["ctrl_vals"] = sum(1 << qubits[q] for q in range(len(qubits)) if (v >> q) & 1)
        return out

    c = 1e-310
    rot = Cc.to_array([Cc.gate(3, np.array([[c, -1.0], [1.0, c]], dtype=np.complex128))])
    return np.concatenate([remap(Cc.rcs_n(9, 8, seed=41), rest), rot, remap(Cc.rcs_n(3, 6, seed=42), [0, 1, 2])])


def test_guarded_ladder_bounds_chunks_coded_at_full_width():
    """Section 3.7, guarded ladder: a chunk holding a subnormal is coded at 64 bits
    whatever the level (Eq. sigbits cannot truncate it), so its image may be as large
    as RAW.  Whenever the controller reports that the chosen level's worst case fits,
    the gate must end with E <= floor(tau * budget) -- over budgets from where the
    truncated worst case fits but the RAW one does not, to where both fit."""
    n, kc = 10, 4
    gates = wide_chunk_circuit()
    nch = 1 << (n - kc)
    lo = nch * _format_max_image(kc, O.sig_bits(1e-4))
    hi = nch * _format_max_image(kc, 64)
    checked = 0
    for thresh in range(lo, hi + 1024, 512):
        budget = math.ceil(thresh / 0.9)
        cs = O.CSim(n, n, kc, 1e-4, budget=budget, ladder=2)
        t = math.floor(0.9 * budget)
        for g in gates:
            cs.apply([g])
            st = cs.stats()
            if st["guard_fit"]:
                checked += 1
                assert st["encoded_bytes"] <= t, (thresh, st["encoded_bytes"], st["level"])
    assert checked > 0


def subnormal_circuit():
    """A real rotation with cos = 1e-310 (subnormal; cos^2 underflows, so the matrix is
    unitary to the last bit) applied under a control on qubit 8 puts subnormal amplitudes
    into the half of the state with bit 8 set; later gates stay on qubits below 8, so the
    other half never meets them."""
    c = 1e-310
    U = np.array([[c, -1.0], [1.0, c]], dtype=np.complex128)
    g = [Cc.gate(8, Cc.H), Cc.gate(0, U, {8: 1}), Cc.gate(1, Cc.H), Cc.gate(4, Cc.H), Cc.gate(5, Cc.H),
         Cc.gate(2, Cc.SX), Cc.gate(6, Cc.H), Cc.gate(3, Cc.T), Cc.gate(7, Cc.H), Cc.gate(1, Cc.SY)]
    return Cc.to_array(g)


def test_chunks_with_subnormals_are_coded_at_full_width():
    n, kc = 10, 4
    cs = O.CSim(n, n, kc, 1e-4, 1)  # lossy from the first gate
    cs.apply(subnormal_circuit())
    assert cs.stats()["S_current"] == O.sig_bits(1e-4)
    for q in range(cs.nchunks):
        img = cs.image(q)
        if (q >> 5) & 1:  # qubit 9 is never touched: those chunks stay ZERO
            assert img[0] == 0
            continue
        vals = O.decode_chunk(img, kc)
        bits = np.concatenate([vals.real, vals.imag]).view(np.uint64)
        has_sub = bool(np.any(((bits >> 52) & 0x7FF == 0) & ((bits << 12) != 0)))
        if (q >> 4) & 1:  # bit 8 of the amplitude index = bit 4 of the chunk index
            assert has_sub and img[1] == 64
        else:
            assert not has_sub and img[1] == O.sig_bits(1e-4)


def test_error_statistics_section_4_2():
    """All relative errors below the bound; errors normalised by the last kept
    mantissa unit are spread over [0, 1); lag-1 autocorrelation near zero."""
    n, kc = 14, 10
    gates = Cc.rcs(2, 7, 20, seed=6)  # deep enough that the amplitudes look random
    psi = O.sv_init(n)
    O.sv_run(psi, n, gates)
    S = O.sig_bits(1e-4)
    rel_all = []
    for c in range(1 << (n - kc)):
        chunk = psi[c << kc:(c + 1) << kc]
        img = O.encode_chunk(chunk, kc, S)
        dec = O.decode_chunk(img, kc)
        x, t = chunk.view(np.float64), dec.view(np.float64)
        nz = x != 0
        rel = np.abs(x - t)[nz] / np.abs(x)[nz]
        assert np.all(rel < 2.0 ** (12 - S))
        ulp = 2.0 ** (np.floor(np.log2(np.abs(x[nz]))) - (S - 12))
        u = np.abs(x - t)[nz] / ulp
        assert np.all((u >= 0) & (u < 1))
        rel_all.append((x - t)[nz] / x[nz])
    e = np.concatenate(rel_all)
    assert e.size > 30000
    u_mean = e.mean() / 2.0 ** (12 - S)
    assert 0.2 < u_mean < 0.5
    ec = e - e.mean()
    rho1 = float(np.dot(ec[:-1], ec[1:]) / np.dot(ec, ec))
    assert abs(rho1) < 5.0 / math.sqrt(e.size)  # 5 sigma of a zero correlation


def test_measure_rule_and_distribution():
    n = 5
    gates = Cc.rcs(1, 5, 4, seed=1)
    psi = O.sv_init(n)
    O.sv_run(psi, n, gates)
    p = np.abs(psi) ** 2
    cum = np.cumsum(p)
    counts = np.zeros(1 << n)
    for seed in range(4000):
        out, prob = O.sv_measure(psi, n, seed)
        u = (O.splitmix64(seed) >> 11) * 2.0 ** -53
        expect = int(np.searchsorted(cum, u * cum[-1], side="left"))
        if abs(cum[min(expect, len(cum) - 1)] - u * cum[-1]) > 1e-12:
            assert out == expect
        assert prob == pytest.approx(p[out] / cum[-1], rel=1e-12)
        counts[out] += 1
    chi2 = np.sum((counts - 4000 * p) ** 2 / (4000 * p + 1e-300))
    assert chi2 < 80  # 31 degrees of freedom


def test_splitmix64_reference_values():
    # splitmix64 outputs for seeds 0 and 1 (Steele, Lea, Flood 2014; the same
    # constants as Java's SplittableRandom)
    assert O.splitmix64(0) == 0xE220A8397B1DCDAF
    assert O.splitmix64(1) == 0x910A2DEC89025CC1
