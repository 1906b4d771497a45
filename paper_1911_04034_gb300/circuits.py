"""Seeded synthetic circuits: the inputs that the simulator and the CPU oracle both read.

This module holds no part of the simulation method: it only lists gates.  Each gate is
one record of ``GATE_DTYPE``: a target qubit, a control mask and control values (a
gate acts on the amplitude pairs whose index matches the controls, Eq. matrix2), and
the 2x2 unitary as eight doubles ``u00r u00i u01r u01i u10r u10i u11r u11i`` computed
here on the host, so the device never evaluates a trigonometric function.

Amplitude index bit k is qubit k.  The benchmark families follow Section 5.3 of the
paper (Grover, random circuit sampling, QAOA MaxCut, QFT of a random basis state) and
the H-on-every-qubit program of Section 5.2; the paper's own circuit files are not
available, so these generators produce circuits of the same kind and size from a seed.
"""
from __future__ import annotations

import math

import numpy as np

GATE_DTYPE = np.dtype(
    [
        ("target", "<i4"),
        ("kind", "<i4"),
        ("ctrl_mask", "<u8"),
        ("ctrl_vals", "<u8"),
        ("u", "<f8", (8,)),
    ]
)

KIND_GENERAL, KIND_DIAGONAL, KIND_PERMUTATION = 0, 1, 2

S2 = 1.0 / math.sqrt(2.0)
H = np.array([[S2, S2], [S2, -S2]], dtype=np.complex128)
X = np.array([[0, 1], [1, 0]], dtype=np.complex128)
Z = np.array([[1, 0], [0, -1]], dtype=np.complex128)
SX = 0.5 * np.array([[1 + 1j, 1 - 1j], [1 - 1j, 1 + 1j]], dtype=np.complex128)
SY = 0.5 * np.array([[1 + 1j, -1 - 1j], [1 + 1j, 1 + 1j]], dtype=np.complex128)
T = np.array([[1, 0], [0, complex(S2, S2)]], dtype=np.complex128)


def rx(theta: float) -> np.ndarray:
    c, s = math.cos(theta / 2), math.sin(theta / 2)
    return np.array([[c, -1j * s], [-1j * s, c]], dtype=np.complex128)


def ry(theta: float) -> np.ndarray:
    c, s = math.cos(theta / 2), math.sin(theta / 2)
    return np.array([[c, -s], [s, c]], dtype=np.complex128)


def rz(theta: float) -> np.ndarray:
    return np.array(
        [[complex(math.cos(theta / 2), -math.sin(theta / 2)), 0], [0, complex(math.cos(theta / 2), math.sin(theta / 2))]],
        dtype=np.complex128,
    )


def phase(phi: float) -> np.ndarray:
    return np.array([[1, 0], [0, complex(math.cos(phi), math.sin(phi))]], dtype=np.complex128)


def _kind(u: np.ndarray) -> int:
    if u[0, 1] == 0 and u[1, 0] == 0:
        return KIND_DIAGONAL
    if u[0, 0] == 0 and u[1, 1] == 0:
        return KIND_PERMUTATION
    return KIND_GENERAL


def gate(target: int, u: np.ndarray, controls: dict[int, int] | None = None) -> np.void:
    """One gate record.  ``controls`` maps control qubit -> required bit value."""
    rec = np.zeros((), dtype=GATE_DTYPE)
    rec["target"] = int(target)
    mask = vals = 0
    for q, v in (controls or {}).items():
        mask |= 1 << int(q)
        vals |= (int(v) & 1) << int(q)
    rec["ctrl_mask"] = mask
    rec["ctrl_vals"] = vals
    rec["u"] = np.array([u[0, 0].real, u[0, 0].imag, u[0, 1].real, u[0, 1].imag,
                         u[1, 0].real, u[1, 0].imag, u[1, 1].real, u[1, 1].imag], dtype=np.float64)
    rec["kind"] = _kind(u)
    return rec


def to_array(gates: list) -> np.ndarray:
    out = np.zeros(len(gates), dtype=GATE_DTYPE)
    for k, g in enumerate(gates):
        out[k] = g
    return out


def matrix_of(rec) -> np.ndarray:
    u = np.asarray(rec["u"], dtype=np.float64)
    return np.array([[u[0] + 1j * u[1], u[2] + 1j * u[3]], [u[4] + 1j * u[5], u[6] + 1j * u[7]]])


def inverse(gates: np.ndarray) -> np.ndarray:
    """The inverse circuit: the gates in reverse order, each unitary replaced by its
    conjugate transpose (exact in floating point; zero parts stay +0).  Run after
    ``gates`` it returns every state to itself up to rounding: a Loschmidt echo, whose
    overlap with the starting state measures what the compression lost."""
    g = np.asarray(gates, dtype=GATE_DTYPE)
    out = np.array(g[::-1], dtype=GATE_DTYPE, copy=True)
    u = np.array(out["u"], dtype=np.float64, copy=True)
    re = (0, 4, 2, 6)  # u00, u10 -> u01, u01 -> u10, u11
    for k, src in enumerate(re):
        out["u"][:, 2 * k] = u[:, src]
        out["u"][:, 2 * k + 1] = 0.0 - u[:, src + 1]
    return out


# --------------------------------------------------------------------------- #
# Circuit families                                                             #
# --------------------------------------------------------------------------- #


def h_all(n: int) -> np.ndarray:
    """Hadamard on every qubit (the scalability program of Section 5.2)."""
    return to_array([gate(q, H) for q in range(n)])


def grover(n: int, iterations: int, seed: int) -> tuple[np.ndarray, int]:
    """Grover search with one seed-chosen marked item.

    Oracle: one multi-controlled Z whose control values spell the marked item (target
    qubit 0 carries the phase on the marked value of bit 0).  Diffusion: H, X on all
    qubits, a multi-controlled Z on |1...1>, X, H.  4n + 2 gates per iteration after
    the initial Hadamard layer.  Returns (gates, marked).
    """
    rng = np.random.default_rng(seed)
    marked = int(rng.integers(0, 1 << n))
    others = {q: (marked >> q) & 1 for q in range(1, n)}
    oracle_u = np.diag([1.0, -1.0]).astype(np.complex128) if (marked & 1) else np.diag([-1.0, 1.0]).astype(np.complex128)
    ones = {q: 1 for q in range(1, n)}
    gs = [gate(q, H) for q in range(n)]
    for _ in range(iterations):
        gs.append(gate(0, oracle_u, others))
        gs += [gate(q, H) for q in range(n)]
        gs += [gate(q, X) for q in range(n)]
        gs.append(gate(0, Z, ones))
        gs += [gate(q, X) for q in range(n)]
        gs += [gate(q, H) for q in range(n)]
    return to_array(gs), marked


def grid_edges(rows: int, cols: int, n: int, cls: int) -> list[tuple[int, int]]:
    """One of four rotating coupler classes on a rows x cols grid (qubit = row*cols + col):
    0/1 = horizontal couplers starting at even/odd columns, 2/3 = vertical couplers
    starting at even/odd rows.  Couplers touching a qubit index >= n are dropped."""
    out = []
    for r in range(rows):
        for c in range(cols):
            a = r * cols + c
            if cls in (0, 1) and c + 1 < cols and c % 2 == cls:
                b = a + 1
            elif cls in (2, 3) and r + 1 < rows and r % 2 == cls - 2:
                b = a + cols
            else:
                continue
            if a < n and b < n:
                out.append((a, b))
    return out


def rcs(rows: int, cols: int, depth: int, seed: int, n: int | None = None) -> np.ndarray:
    """Random circuit on a rows x cols grid: a Hadamard layer, then ``depth`` layers of
    CZ on the rotating coupler class followed by one random gate from {sqrt(X),
    sqrt(Y), T} on every qubit."""
    n = rows * cols if n is None else n
    rng = np.random.default_rng(seed)
    pool = (SX, SY, T)
    gs = [gate(q, H) for q in range(n)]
    for layer in range(depth):
        for a, b in grid_edges(rows, cols, n, layer % 4):
            gs.append(gate(b, Z, {a: 1}))
        for q in range(n):
            gs.append(gate(q, pool[int(rng.integers(0, 3))]))
    return to_array(gs)


def rcs_n(n: int, depth: int, seed: int) -> np.ndarray:
    """Random circuit with n qubits on the most square grid holding them."""
    cols = int(math.ceil(math.sqrt(n)))
    rows = int(math.ceil(n / cols))
    return rcs(rows, cols, depth, seed, n=n)


def random_regular_graph(n: int, d: int, seed: int) -> list[tuple[int, int]]:
    """Seeded random d-regular simple graph by the pairing model with restarts."""
    if (n * d) % 2 or d >= n:
        raise ValueError("no d-regular graph with these sizes")
    rng = np.random.default_rng(seed)
    for _ in range(10000):
        stubs = np.repeat(np.arange(n), d)
        rng.shuffle(stubs)
        pairs = stubs.reshape(-1, 2)
        edges = set()
        ok = True
        for a, b in pairs:
            a, b = int(min(a, b)), int(max(a, b))
            if a == b or (a, b) in edges:
                ok = False
                break
            edges.add((a, b))
        if ok:
            return sorted(edges)
    raise RuntimeError("pairing model did not converge")


def qaoa_maxcut(n: int, p: int, degree: int, seed: int) -> tuple[np.ndarray, list[tuple[int, int]]]:
    """QAOA for MaxCut on a seeded random regular graph, angles uniform in [0, pi).
    Each cost term exp(-i gamma Z_a Z_b) is CNOT(a->b) RZ(2 gamma) on b, CNOT(a->b);
    the mixer is RX(2 beta) on every qubit."""
    edges = random_regular_graph(n, degree, seed)
    rng = np.random.default_rng(seed + 1)
    gammas = rng.uniform(0.0, math.pi, size=p)
    betas = rng.uniform(0.0, math.pi, size=p)
    gs = [gate(q, H) for q in range(n)]
    for k in range(p):
        for a, b in edges:
            gs.append(gate(b, X, {a: 1}))
            gs.append(gate(b, rz(2 * gammas[k])))
            gs.append(gate(b, X, {a: 1}))
        for q in range(n):
            gs.append(gate(q, rx(2 * betas[k])))
    return to_array(gs), edges


def qft(n: int, seed: int) -> tuple[np.ndarray, int]:
    """Quantum Fourier transform of a random basis state |x> (X gates on the set bits).
    Maps |x> to sum_k exp(2 pi i x k / 2^n) |k> / 2^(n/2).  Returns (gates, x)."""
    rng = np.random.default_rng(seed)
    x = int(rng.integers(0, 1 << n))
    gs = [gate(q, X) for q in range(n) if (x >> q) & 1]
    for j in reversed(range(n)):
        gs.append(gate(j, H))
        for m in reversed(range(j)):
            gs.append(gate(j, phase(math.pi / (1 << (j - m))), {m: 1}))
    for i in range(n // 2):
        a, b = i, n - 1 - i
        gs += [gate(b, X, {a: 1}), gate(a, X, {b: 1}), gate(b, X, {a: 1})]
    return to_array(gs), x


def random_batch(count: int, n_lo: int, n_hi: int, d_lo: int, d_hi: int, seed: int) -> list[tuple[int, np.ndarray]]:
    """``count`` independent random circuits, qubits uniform in [n_lo, n_hi] and depth
    uniform in [d_lo, d_hi], each with the random-circuit gate set."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        n = int(rng.integers(n_lo, n_hi + 1))
        d = int(rng.integers(d_lo, d_hi + 1))
        out.append((n, rcs_n(n, d, seed * 100003 + k)))
    return out


def selector_init(seed: int) -> np.ndarray:
    """Seeded starting parameters of the chunk-mode selector network (16 -> 32 -> 32 ->
    8): He-normal weights and zero biases, float32, in the order W1 b1 W2 b2 W3 b3 with
    row-major weight matrices (1864 numbers).  Random numbers only; the trainer rounds
    them to bfloat16."""
    rng = np.random.default_rng(seed)
    parts = []
    for rows, cols in ((32, 16), (32, 32), (8, 32)):
        parts.append((rng.standard_normal((rows, cols)) * math.sqrt(2.0 / cols)).astype(np.float32).ravel())
        parts.append(np.zeros(rows, dtype=np.float32))
    return np.concatenate(parts)
