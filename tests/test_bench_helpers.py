"""Host logic of bench.py (no GPU): gate classes, the algorithmic FP64 flop count, the
amplitude-update count and the per-class roofline bookkeeping, each against values
worked out by hand."""
import math

import numpy as np
import pytest

import bench
from paper_1911_04034_gb300 import circuits as Cc


def one(g):
    return Cc.to_array([g])


def test_gate_classes():
    assert bench.gate_class(one(Cc.gate(0, Cc.SX))[0]) == "dense"
    assert bench.gate_class(one(Cc.gate(0, Cc.SY))[0]) == "dense"  # (1 + i) / 2 times a real matrix
    assert bench.gate_class(one(Cc.gate(0, Cc.H))[0]) == "real"
    assert bench.gate_class(one(Cc.gate(0, Cc.T))[0]) == "diagonal"
    assert bench.gate_class(one(Cc.gate(1, Cc.Z, {0: 1}))[0]) == "diagonal"
    assert bench.gate_class(one(Cc.gate(0, Cc.X))[0]) == "permutation"
    other = np.array([[1.0, 0.0], [0.6, 0.8]], dtype=np.complex128)  # one zero entry
    assert bench.gate_class(one(Cc.gate(0, other))[0]) == "other"


def test_fp64_flops_by_hand():
    n, kc = 10, 4
    pairs = (1 << n) // 2
    # sqrt(X): every output part is a chain of four nonzero terms -> 1 product + 3 FMAs = 7
    # flops, four parts per pair = 28
    assert bench.fp64_flops(one(Cc.gate(3, Cc.SX)), n, kc) == 28 * pairs
    # T = diag(1, e^{i pi/4}): row 0 is two chains of one coefficient 1 (no flop); row 1's
    # real part c * br - s * bi (1 product + 1 FMA = 3 flops), its imaginary part the same
    assert bench.fp64_flops(one(Cc.gate(3, Cc.T)), n, kc) == 6 * pairs
    # H: four chains of two real terms whose first coefficient is 1/sqrt(2): 3 flops each
    assert bench.fp64_flops(one(Cc.gate(3, Cc.H)), n, kc) == 12 * pairs
    # a control inside the chunk halves the pairs, one on a chunk bit halves the amplitudes
    assert bench.fp64_flops(one(Cc.gate(3, Cc.SX, {1: 1})), n, kc) == 28 * pairs / 2
    assert bench.fp64_flops(one(Cc.gate(3, Cc.SX, {7: 0})), n, kc) == 28 * pairs / 2
    # X copies: no arithmetic
    assert bench.fp64_flops(one(Cc.gate(3, Cc.X)), n, kc) == 0


def test_amp_updates_counts_touched_chunks():
    n, kc = 12, 5
    assert bench.amp_updates(one(Cc.gate(2, Cc.H)), n, kc) == 1 << n
    assert bench.amp_updates(one(Cc.gate(2, Cc.H, {7: 1})), n, kc) == 1 << (n - 1)  # chunk bit: half the chunks
    assert bench.amp_updates(one(Cc.gate(2, Cc.H, {1: 1})), n, kc) == 1 << n  # in-chunk control: every chunk
    assert bench.amp_updates(one(Cc.gate(9, Cc.Z, {7: 1, 8: 0})), n, kc) == 1 << (n - 2)


def test_per_class_bookkeeping():
    n, kc = 10, 4
    gates = Cc.to_array([Cc.gate(3, Cc.SX), Cc.gate(4, Cc.T), Cc.gate(5, Cc.SX)])
    tl = {"ms": np.array([2.0, 1.0, 4.0]), "bytes_read": np.array([100.0, 50.0, 300.0]),
          "bytes_written": np.array([100.0, 50.0, 300.0])}
    out = bench.per_class(gates, tl, n, kc, hbm=1000.0)
    d = out["dense"]
    assert d["launches"] == 2 and d["kernel_ms_per_launch"] == pytest.approx(3.0)
    assert d["image_bytes_per_launch"] == pytest.approx(400.0)
    assert d["hbm_gbs"] == pytest.approx(800.0 / 6e-3 / 1e9)
    assert d["hbm_frac"] == pytest.approx(d["hbm_gbs"] / 1000.0)
    assert d["amp_updates_per_s"] == pytest.approx(2 * (1 << n) / 6e-3)
    assert d["fp64_tflops"] == pytest.approx(2 * 28 * (1 << (n - 1)) / 6e-3 / 1e12)
    assert out["diagonal"]["launches"] == 1 and "permutation" not in out


def test_layers_split_the_random_circuit():
    rows, cols = bench.ROWS, bench.COLS
    n = rows * cols
    g = Cc.rcs(rows, cols, 5, seed=1)
    layers = bench.layers_of(g, n, 5)
    assert len(layers) == 6 and len(layers[0]) == n
    assert sum(len(x) for x in layers) == len(g)
    assert all(len(x) == n + len(Cc.grid_edges(rows, cols, n, k % 4)) for k, x in enumerate(layers[1:]))
