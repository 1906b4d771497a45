#!/usr/bin/env python
"""Benchmark: compressed-state amplitude updates/s on the 30-qubit random circuit.

Workload (the configuration the metric is quoted on): random circuit sampling on a
5 x 6 grid (30 qubits), a Hadamard layer then layers of CZ on a rotating coupler
class plus one random gate from {sqrt(X), sqrt(Y), T} per qubit; complex128 state in
blocks of 2^20 amplitudes (chunks of 2^10), lossless first and lossy at pointwise
relative bound 1e-4 once the state passes 90 % of the budget (raw/4).  Synthetic,
seeded circuits; the compressed state (several GB) is larger than L2, so no flush.

One step = one circuit layer (about 42 gates) on the evolving compressed state: every
gate runs the whole path (classify, decode, apply, controller, truncate, XOR-code,
mode select, page commit, stats).  Warm-up steps are the first layers after the
Hadamard layer; timed steps follow.  `value` is device-timed (CUDA events on the
simulator's stream); `e2e` times the same calls from the host, including the
per-step read-back of the statistics.  Fidelity is measured against the uncompressed
complex128 state vector run on the same GPU (same gates).

--impl reference times the CPU oracle (tests' reference implementation) on a
bounded sample of the same workload on the host cores.
With torchrun (N > 1) every rank runs an independent replica (the method does not
shard across GPUs here); value = all ranks' updates / slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1911_04034_gb300 import circuits as Cc  # noqa: E402

METRIC = "compressed-state amplitude updates/s"
UNIT = "amp-updates/s"
ROWS, COLS, BLOCK_LOG2, CHUNK_LOG2, SEED = 5, 6, 20, 10, 2024  # defaults; --rows/--cols override

# DRAM traffic of a gate's launches from the last ncu capture, with the hash of the kernel
# sources it applies to.  A 30-qubit launch is too large to capture, so the capture ran the
# 26-qubit 2 x 13 grid in its steady state (k_gate_fast launches 801-804, every item on the
# streaming kernel): dram__bytes_read.sum + dram__bytes_write.sum = 832 MB per launch
# against 860.5 MB of image bytes per gate, a ratio of 0.968 (reads 447 MB: the input
# images plus directory entries; writes 384 MB, the rest of the output images still dirty
# in L2 when the launch ends); traffic scales with the image bytes, so a 30-qubit gate's
# traffic is that ratio times its image bytes.
NCU_TRAFFIC = {"ratio_to_image_bytes": 0.968, "source_sha": "4880ea788b2bc48a"}


def kernel_sha() -> str:
    h = hashlib.sha256()
    for f in ("paper_1911_04034_gb300/csrc/fast.cu", "paper_1911_04034_gb300/csrc/kernels.cu",
              "paper_1911_04034_gb300/csrc/gate_common.cuh", "paper_1911_04034_gb300/csrc/device.cuh"):
        h.update(open(os.path.join(ROOT, f), "rb").read())
    return h.hexdigest()[:16]


def layers_of(gates: np.ndarray, n: int, depth: int) -> list[np.ndarray]:
    """Splits an rcs() gate list into [Hadamard layer, layer 1, ..., layer depth]."""
    out = [gates[:n]]
    pos = n
    for layer in range(depth):
        m = len(Cc.grid_edges(ROWS, COLS, n, layer % 4)) + n
        out.append(gates[pos:pos + m])
        pos += m
    assert pos == len(gates)
    return out


def amp_updates(gates: np.ndarray, n: int, kc: int) -> int:
    """Amplitudes in the chunks each gate touches (controls on chunk-index bits
    remove chunks), summed over the gates."""
    tot = 0
    for g in gates:
        hi = int(g["ctrl_mask"]) >> kc
        tot += (1 << n) >> bin(hi).count("1")
    return tot


def fp64_flops(gates: np.ndarray, n: int, kc: int) -> float:
    """Algorithmic FP64 flops of the gate arithmetic: per amplitude pair, each output
    component is a chain over its nonzero coefficients (the first a product, unless it
    is +-1 and needs no arithmetic, each later one a fused multiply-add = 2 flops);
    pairs = amplitudes in touched chunks / 2, thinned by controls inside a chunk."""
    tot = 0.0
    for g in gates:
        u = [float(x) for x in g["u"]]
        rows = ((u[0], -u[1], u[2], -u[3]), (u[0], u[1], u[2], u[3]), (u[4], -u[5], u[6], -u[7]), (u[4], u[5], u[6], u[7]))
        per_pair = 0
        for r in rows:
            kept = [c for c in r if c != 0.0]
            if kept:
                per_pair += (0 if kept[0] in (1.0, -1.0) else 1) + 2 * (len(kept) - 1)
        mask = int(g["ctrl_mask"])
        amps = (1 << n) >> bin(mask >> kc).count("1")
        tot += per_pair * (amps / 2) / (1 << bin(mask & ((1 << kc) - 1)).count("1"))
    return tot


def gate_class(g) -> str:
    """dense: all four entries of the 2x2 matrix nonzero, some complex (sqrt(X));
    real: all four nonzero and real (sqrt(Y), H); diagonal: zero off-diagonal (T, CZ,
    phases); permutation: zero diagonal (X, CNOT); other: one zero entry."""
    u = [float(x) for x in g["u"]]
    z = [u[2 * k] == 0.0 and u[2 * k + 1] == 0.0 for k in range(4)]
    if not any(z):
        return "real" if all(u[2 * k + 1] == 0.0 for k in range(4)) else "dense"
    if z[1] and z[2]:
        return "diagonal"
    if z[0] and z[3]:
        return "permutation"
    return "other"


def per_class(gates: np.ndarray, tl: dict, n: int, kc: int, hbm: float | None) -> dict:
    """Kernel time, image bytes and the two roofline fractions per gate class, from the
    per-launch CUDA-event times and traffic counters of the timed gates."""
    out = {}
    cls = [gate_class(g) for g in gates]
    assert len(cls) == len(tl["ms"])
    for c in ("dense", "real", "diagonal", "permutation", "other"):
        idx = [i for i, x in enumerate(cls) if x == c]
        if not idx:
            continue
        ms = float(np.sum(tl["ms"][idx]))
        by = float(np.sum(tl["bytes_read"][idx]) + np.sum(tl["bytes_written"][idx]))
        fl = fp64_flops(gates[idx], n, kc)
        ach = by / (ms * 1e-3) / 1e9
        out[c] = {"launches": len(idx), "kernel_ms_per_launch": ms / len(idx),
                  "image_bytes_per_launch": by / len(idx), "hbm_gbs": ach,
                  "hbm_frac": ach / hbm if hbm else None,
                  "fp64_tflops": fl / (ms * 1e-3) / 1e12, "fp64_frac": fl / (ms * 1e-3) / 1e12 / FP64_PEAK_TFLOPS,
                  "amp_updates_per_s": amp_updates(gates[idx], n, kc) / (ms * 1e-3)}
    return out


# GB300 FP64 (vector pipe): the nominal rate of the part; a DFMA-throughput loop on this
# pool's GB300 (eight independent chains per thread, 1216 CTAs of 256 threads) measured
# 6.27e11 fused multiply-adds per second = 1.255 TFLOP/s.
FP64_PEAK_TFLOPS = 1.25
FP64_PEAK_SOURCE = "nominal GB300 FP64 (vector) rate; a DFMA-throughput loop measured 1.255 TFLOP/s"


def peaks() -> dict:
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


class Clocks:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self) -> dict:
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        rows = [r.split(",") for r in open(self.f.name).read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except (ValueError, IndexError):
                continue
            for k, nm in enumerate(names):
                if len(r) > 5 + k and r[5 + k].lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def reduce_over_ranks(ms: float, updates: float, dist, device: str) -> tuple[float, float]:
    """Replicas: the job's time is the slowest rank's, its work the sum of all ranks'."""
    import torch

    t = torch.tensor([ms, float(updates)], dtype=torch.float64, device=device)
    tmax = t.clone()
    dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(tmax[0]), float(t[1])


def replica_seed(rank: int) -> int:
    """Each replica simulates its own random circuit of the same family and size."""
    return SEED + rank


CFG2_DEPTH = 20  # the random-circuit configuration's depth: fidelity and the bound sweep are taken there


def depth20_run(qcsim, torch, gates_d20: np.ndarray, n: int, eps: float, kc_req: int, sv_data_ptr: int | None,
                no_fast: bool) -> dict:
    """The depth-20 random circuit alone at bound eps (device-timed from |0...0>, the
    lossless start included): rate, compression and fidelity against the uncompressed
    state vector's device buffer."""
    raw = 16 << n
    stream = torch.cuda.Stream()
    sim = qcsim.Sim(n, BLOCK_LOG2, eps, chunk_log2=kc_req, budget=raw // 4, pool_bytes=raw + raw // 8 + (64 << 20),
                    stream=stream)
    if no_fast:
        sim.set_option("fast_path", 0)
    kc = sim.chunk_log2
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    sim.apply_circuit(gates_d20)
    ev1.record(stream)
    ev1.synchronize()
    ms = ev0.elapsed_time(ev1)
    st = sim.stats()
    out = {"amp_updates_per_s": amp_updates(gates_d20, n, kc) / (ms * 1e-3), "seconds": ms * 1e-3,
           "compression_ratio": st["ratio"], "min_compression_ratio": st["min_ratio"],
           "fidelity_lb_sum": st["fidelity_lb_sum"], "eps_switch_gate": st["eps_switch_gate"]}
    if sv_data_ptr is not None:
        F = qcsim.C.c_double()
        qcsim._check(qcsim.lib().sim_fidelity(sim._h, qcsim.C.c_void_p(sv_data_ptr), 1, qcsim.C.byref(F), None, None),
                     "sim_fidelity")
        out["fidelity"] = float(F.value)
    sim.close()
    return out


def run_gpu(args) -> dict | None:
    import torch

    from paper_1911_04034_gb300 import qcsim

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    n = ROWS * COLS
    # the depth-20 circuit, then further layers of the same family for the timed steps
    depth = CFG2_DEPTH + args.warmup + 2 * args.steps
    gates = Cc.rcs(ROWS, COLS, depth, seed=replica_seed(rank))
    layers = layers_of(gates, n, depth)
    d20 = np.concatenate(layers[: 1 + CFG2_DEPTH])
    raw = 16 << n
    stream = torch.cuda.Stream()
    pool = raw + raw // 8 + (64 << 20)  # page rounding + per-CTA page caches
    sim = qcsim.Sim(n, BLOCK_LOG2, args.eps, chunk_log2=args.kc, budget=raw // 4, pool_bytes=pool,
                    stream=stream)
    if args.no_fast:
        sim.set_option("fast_path", 0)
    kc = sim.chunk_log2

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()

    # the depth-20 circuit (untimed here) and its fidelity against the uncompressed
    # complex128 state vector on the same GPU (same gates)
    sim.apply_circuit(d20)
    fid = sv_rate = None
    sweep = {}
    sv = None
    if not args.no_sv:
        sv = qcsim.StateVector(n)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sv.apply_circuit(d20)
        torch.cuda.synchronize()
        sv_rate = len(d20) * float(1 << n) / (time.perf_counter() - t0)
        F = qcsim.C.c_double()
        qcsim._check(qcsim.lib().sim_fidelity(sim._h, qcsim.C.c_void_p(sv.data_ptr()), 1, qcsim.C.byref(F), None, None),
                     "sim_fidelity")
        fid = float(F.value)
    st_d20 = sim.stats()
    # warm-up: W further layers
    for L in layers[1 + CFG2_DEPTH: 1 + CFG2_DEPTH + args.warmup]:
        sim.apply_circuit(L)
    st0 = sim.stats()
    # timed region (device time, CUDA events on the simulator's stream)
    t_first = 1 + CFG2_DEPTH + args.warmup
    timed = layers[t_first: t_first + args.steps]
    clocks = Clocks(local)
    sim.set_timing(2 if args.phases else 1)
    barrier()
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for L in timed:
        sim.apply_circuit(L)
    ev1.record(stream)
    ev1.synchronize()
    barrier()
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    tl = sim.timing_launches()
    tm = sim.timing()
    sim.set_timing(False)
    st1 = sim.stats()
    updates = st1["amp_updates"] - st0["amp_updates"]
    assert updates == amp_updates(np.concatenate(timed), n, kc)
    # end to end through the public API: host gate records in, statistics read back
    e2e_layers = layers[t_first + args.steps: t_first + 2 * args.steps]
    barrier()
    t0 = time.perf_counter()
    h2d = d2h = 0
    for L in e2e_layers:
        sim.apply_circuit(L)
        _ = sim.stats()
        h2d += L.nbytes
        d2h += qcsim.C.sizeof(qcsim.Stats)
    barrier()
    e2e_s = time.perf_counter() - t0
    e2e_updates = amp_updates(np.concatenate(e2e_layers), n, kc)
    st2 = sim.stats()
    sim.close()
    # the bound sweep of the configuration: the depth-20 circuit at 1e-5 and 1e-3 (and
    # 1e-4 above), each from |0...0> with its fidelity against the same state vector
    if not args.no_sweep:
        for e in (1e-5, 1e-3):
            sweep[f"{e:g}"] = depth20_run(qcsim, torch, d20, n, e, args.kc, sv.data_ptr() if sv is not None else None,
                                          args.no_fast)
    if sv is not None:
        sv.close()
    ms_max, upd_total = ms, updates
    if dist is not None:
        ms_max, upd_total = reduce_over_ranks(ms, updates, dist, "cuda")
        dist.destroy_process_group()
    if rank != 0:
        return None
    sweep["0.0001"] = {"fidelity": fid, "compression_ratio": st_d20["ratio"], "min_compression_ratio": st_d20["min_ratio"],
                       "fidelity_lb_sum": st_d20["fidelity_lb_sum"], "eps_switch_gate": st_d20["eps_switch_gate"],
                       "note": "the timed simulator itself at depth 20"}
    pk = peaks()
    hbm = pk.get("hbm_gbs")
    kernel_ms_avg = tm["gate_kernel_ms"] / max(1, tm["launches"])
    bytes_per_launch = (tm["bytes_read"] + tm["bytes_written"]) / max(1, tm["launches"])
    achieved = bytes_per_launch / (kernel_ms_avg * 1e-3) / 1e9 if kernel_ms_avg > 0 else 0.0
    traffic = (NCU_TRAFFIC["ratio_to_image_bytes"] * bytes_per_launch
               if NCU_TRAFFIC["source_sha"] == kernel_sha() else None)
    flops = fp64_flops(np.concatenate(timed), n, kc)
    out = {
        "metric": METRIC,
        "value": upd_total / (ms_max * 1e-3),
        "unit": UNIT,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_max / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic",
        "config": {
            "workload": f"random circuit {ROWS}x{COLS} grid, {n} qubits: the depth-{CFG2_DEPTH} circuit, then "
                        f"{args.warmup} warm-up layers and layers {t_first}-{t_first + args.steps - 1} timed; "
                        f"eps {args.eps}; blocks 2^{BLOCK_LOG2}, chunks 2^{kc}",
            "n_qubits": n, "block_log2": BLOCK_LOG2, "chunk_log2": kc, "eps": args.eps,
            "budget_bytes": raw // 4, "pool_bytes": pool, "gates_timed": int(sum(len(x) for x in timed)),
            "l2": "no flush: compressed state larger than L2",
            "parallelism": "replicas" if world > 1 else "1 gpu",
        },
        "compression_ratio": st1["ratio"],
        "min_compression_ratio": st2["min_ratio"],
        "fidelity": fid,
        "fidelity_depth": CFG2_DEPTH,
        "fidelity_lb_sum": st_d20["fidelity_lb_sum"],
        "eps_switch_gate": st_d20["eps_switch_gate"],
        "eps_sweep_depth20": sweep,
        "encoded_gb": st1["encoded_bytes"] / 1e9,
        "chunks_by_mode": st1["chunks_by_mode"][:7],
        "fast_items_timed": st1["fast_items"] - st0["fast_items"],
        "fast_deferred_timed": st1["fast_deferred"] - st0["fast_deferred"],
        "uncompressed_value": sv_rate,
        "roofline": {
            "bound": "hbm",
            "achieved": achieved,
            "peak": hbm,
            "unit": "GB/s",
            "frac": (achieved / hbm) if hbm else None,
            "traffic": traffic,
            "kernel": "k_gate_fast + k_gate (one gate's launches)",
            "kernel_ms_avg": kernel_ms_avg,
            "algorithmic_bytes_per_launch": bytes_per_launch,
            "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured)" if hbm else None,
        },
        "roofline_fp64": {
            "bound": "alu",
            "achieved": flops / (tm["gate_kernel_ms"] * 1e-3) / 1e12,
            "peak": FP64_PEAK_TFLOPS,
            "unit": "TFLOP/s",
            "frac": flops / (tm["gate_kernel_ms"] * 1e-3) / 1e12 / FP64_PEAK_TFLOPS,
            "kernel": "k_gate_fast + k_gate",
            "peak_source": FP64_PEAK_SOURCE,
            "note": "the fused kernels' arithmetic ceiling: dense gates cost 28 flops per amplitude pair",
        },
        "roofline_by_class": per_class(np.concatenate(timed), tl, n, kc, hbm),
        "gpu_launches": st1["kernel_launches"] - st0["kernel_launches"],
        "phase_share": ({k: round(v / max(1, sum(st1["phase_cycles"])), 4) for k, v in
                         zip(("stage", "decode", "apply", "encode", "commit", "const"), st1["phase_cycles"])}
                        if args.phases else None),
        "clocks": clk,
        "e2e": {"value": e2e_updates / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d // max(1, len(e2e_layers)),
                "d2h_bytes_per_step": d2h // max(1, len(e2e_layers))},
    }
    if not args.no_batch:
        # the batched workload beside the headline: one replayed step after a capture
        bt = run_batch(args, steps=1, warmup=2)
        out["batch_workload"] = {k: bt[k] for k in ("value", "unit", "ms_per_step", "plain_per_gate_value",
                                                    "speedup_vs_plain", "graph_replays", "min_fidelity_lb_sum",
                                                    "mean_compression_ratio")}
        out["batch_workload"]["workload"] = bt["config"]["workload"]
        out["batch_workload"]["autotuned"] = bt["autotune"]["best"]
        out["batch_workload"]["autotune_points"] = bt["autotune"]["points_measured"]
    return out


def run_batch(args, steps: int | None = None, warmup: int | None = None) -> dict:
    """256 independent random circuits (qubits uniform in 14..24, depth in 12..24, the
    random-circuit gate set, eps 1e-4).  The autotuner picks block size (2^10..2^16),
    tile (chunk) size and codec schedule (bound ladder, mode set) on a 20-qubit probe;
    then each step runs the whole batch from |0...0> in one persistent launch per gate
    step: the first warm-up step captures the CUDA graph, every later step replays it
    after sim_reset.  Against it: the same circuits on the same handles one after
    another through the per-gate path.  Wall-clock time of the calls (both synchronise
    at the end); the resets between steps are not timed."""
    import torch

    from paper_1911_04034_gb300 import qcsim

    steps = args.steps if steps is None else steps
    warmup = args.warmup if warmup is None else warmup
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    batch = Cc.random_batch(args.batch, 14, 24, 12, 24, seed=SEED)
    probe = Cc.rcs_n(20, 6, seed=SEED)
    t0 = time.perf_counter()
    best, tried = qcsim.autotune(20, args.eps, probe)
    tune_s = time.perf_counter() - t0
    kc, b, ladder, modes = best["chunk_log2"], best["block_log2"], best["ladder"], best["modes"]
    sims = []
    for n, _ in batch:
        s_ = qcsim.Sim(n, b, args.eps, chunk_log2=kc, budget=(16 << n) // 4, ladder=ladder,
                       pool_bytes=(16 << n) + (16 << n) // 8 + (8 << 20))
        s_.set_modes(modes)
        sims.append(s_)
    circuits = [g for _, g in batch]
    per_pass = sum(amp_updates(g, n, min(kc, n)) for n, g in batch)

    def reset_all():
        for s_ in sims:
            s_.reset()
        torch.cuda.synchronize()

    def timed(fn, k):
        tot = 0.0
        for _ in range(k):
            reset_all()
            t = time.perf_counter()
            fn()
            torch.cuda.synchronize()
            tot += time.perf_counter() - t
        return tot

    def batched():
        qcsim.batch_apply(sims, circuits, use_graph=True)

    def plain():
        for s_, g in zip(sims, circuits):
            s_.apply_circuit(g)

    capture_s = timed(batched, 1)  # the first call captures and instantiates the graph
    timed(batched, warmup - 1)
    t_batch = timed(batched, steps)
    replays = sims[0].stats()["graph_replays"]
    ratio = [s_.stats()["ratio"] for s_ in sims]
    lb = min(s_.stats()["fidelity_lb_sum"] for s_ in sims)
    upd = sum(s_.stats()["amp_updates"] for s_ in sims)
    timed(plain, 1)
    t_plain = timed(plain, steps)
    for s_ in sims:
        s_.close()
    assert upd == per_pass, (upd, per_pass)
    return {"metric": METRIC, "value": per_pass * steps / t_batch, "unit": UNIT, "n_gpus": 1, "steps": steps,
            "warmup": warmup, "ms_per_step": t_batch / steps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"batch of {args.batch} random circuits, 14-24 qubits, depth 12-24, eps {args.eps}, "
                                   f"one launch per gate step, CUDA graph kept and replayed after sim_reset; "
                                   f"blocks 2^{b}, chunks 2^{kc}, ladder {ladder}, modes {modes:#x} (autotuned)",
                       "l2": "no flush: the batch's compressed states exceed L2"},
            "autotune": {"best": best, "points_measured": len(tried), "seconds": tune_s, "points": tried},
            "plain_per_gate_value": per_pass * steps / t_plain, "speedup_vs_plain": t_plain / t_batch,
            "seconds_batched_per_step": t_batch / steps, "seconds_plain_per_step": t_plain / steps,
            "seconds_first_call_with_capture": capture_s, "graph_replays": replays,
            "min_fidelity_lb_sum": lb, "mean_compression_ratio": float(np.mean(ratio))}


def run_qaoa34(args) -> dict:
    """QAOA p = 2 MaxCut on a seeded random 3-regular graph (51 edges), 34 qubits: the
    raw state (256 GiB) does not fit, so the compressed state has to stay inside a
    180 GB page pool.  Bound 1e-4 reached through the guarded ladder (before each gate
    the smallest level 1e-5 / 1e-4 whose worst case fits 0.9 x 180 GB).  Timed: every
    gate after the Hadamard layer and `warmup` further gates, on the device."""
    import torch

    from paper_1911_04034_gb300 import qcsim

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    n, kc = 34, args.kc
    # every byte the handle holds within 180 GB: the directory (one entry per chunk), the
    # free-page stack and freed list (4 bytes per page each) and small bookkeeping come
    # out of the 180 GB first, the page arena gets the rest
    limit = 180 * 10**9
    dir_bytes = (1 << (n - kc)) * (((16 + 4 * ((16 + (16 << kc) + 511) // 512)) + 15) // 16 * 16)
    pool = int((limit - dir_bytes - (256 << 20)) / (1 + 8 / 512)) // 512 * 512
    gates, edges = Cc.qaoa_maxcut(n, 2, 3, seed=SEED)
    stream = torch.cuda.Stream()
    sim = qcsim.Sim(n, 20, args.eps, chunk_log2=kc, budget=pool, ladder=2, pool_bytes=pool, stream=stream)
    assert sim.stats()["device_bytes"] <= limit, sim.stats()["device_bytes"]
    w = n + args.warmup
    sim.apply_circuit(gates[:w])
    st0 = sim.stats()
    timed = gates[w:]
    clocks = Clocks(int(os.environ.get("LOCAL_RANK", "0")))
    sim.set_timing(1)
    torch.cuda.synchronize()
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    sim.apply_circuit(timed)
    ev1.record(stream)
    ev1.synchronize()
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    tm = sim.timing()
    st = sim.stats()
    updates = st["amp_updates"] - st0["amp_updates"]
    kernel_ms = tm["gate_kernel_ms"] / max(1, tm["launches"])
    bpl = (tm["bytes_read"] + tm["bytes_written"]) / max(1, tm["launches"])
    pk = peaks().get("hbm_gbs")
    echo = None
    if args.echo:
        # Loschmidt echo (untimed): the inverse circuit run compressed after the forward one;
        # |<0...0|state>| >= 1 - sum(delta) over both halves (the fidelity bound)
        sim.apply_circuit(Cc.inverse(gates))
        a0 = complex(sim.amplitudes(0, 1)[0])
        st2 = sim.stats()
        echo = {"amp0_abs": abs(a0), "bound": st2["fidelity_lb_sum"], "gates": 2 * len(gates),
                "max_encoded_gb": st2["max_encoded_bytes"] / 1e9, "eps_final": st2["eps_current"]}
    return {"metric": METRIC, "value": updates / (ms * 1e-3), "unit": UNIT, "n_gpus": 1, "steps": len(timed),
            "warmup": args.warmup, "ms_per_step": ms / len(timed), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"QAOA p=2 MaxCut, random 3-regular graph ({len(edges)} edges), {n} qubits, "
                                   f"eps {args.eps} via the guarded ladder, all device memory of the simulator within "
                                   f"180 GB (page arena {pool / 1e9:.1f} GB); gates {w}-{len(gates) - 1} timed",
                       "n_qubits": n, "chunk_log2": kc, "block_log2": 20, "gates": len(gates), "pool_bytes": pool,
                       "raw_bytes": 16 << n},
            "max_encoded_gb": st["max_encoded_bytes"] / 1e9, "peak_pages_gb": st["peak_pages_bytes"] / 1e9,
            "device_gb": st["device_bytes"] / 1e9, "compression_ratio": st["ratio"], "min_compression_ratio": st["min_ratio"],
            "eps_final": st["eps_current"], "eps_switch_gate": st["eps_switch_gate"],
            "fidelity_lb_sum": st["fidelity_lb_sum"], "fidelity_lb_prod": st["fidelity_lb_prod"],
            "roofline": {"bound": "hbm", "achieved": bpl / (kernel_ms * 1e-3) / 1e9 if kernel_ms else None, "peak": pk,
                         "unit": "GB/s", "frac": (bpl / (kernel_ms * 1e-3) / 1e9 / pk) if (pk and kernel_ms) else None,
                         "traffic": None, "kernel": "k_gate", "kernel_ms_avg": kernel_ms},
            "gpu_launches": 2 * tm["launches"], "clocks": clk, "echo": echo}


def train_selector(qcsim, eps: float, seed: int):
    """Selector network trained on the GPU from exhaustive-trial traces of a 20-qubit
    random circuit and a 20-qubit QAOA circuit (the families of the 30- and 34-qubit
    workloads); returns (bfloat16 parameters, trace rows, last loss)."""
    rows = []
    for g in (Cc.rcs(4, 5, 8, seed=seed), Cc.qaoa_maxcut(20, 2, 3, seed=seed)[0]):
        s = qcsim.Sim(20, 20, eps, chunk_log2=10, budget=(16 << 20) // 4, pool_bytes=2 * (16 << 20) + (64 << 20))
        s.set_selector(1)
        s.trace(1 << 20)
        s.apply_circuit(g)
        rows.append(s.trace_read())
        s.close()
    tr = np.concatenate(rows)
    p0 = Cc.selector_init(seed)
    _, wb, loss = qcsim.mlp_train(tr[:, :16], tr[:, 16].astype(np.int32), tr[:, 17:18], p0, epochs=40, batch=256,
                                  lr=3e-3, seed=seed)
    return wb, int(tr.shape[0]), loss


def run_grover(args) -> dict:
    """Grover search, 8 iterations, 32 qubits (64 GiB raw; the 36-qubit state does not
    fit one GB300 with this codec at 1e-4), blocks of 2^20, lossless then 1e-4 at raw/4:
    the chunk-mode selectors side by side -- Solution C only, the exhaustive trial of
    every mode, and the trained network granting the SPLIT / PALETTE trials.  Per
    selector: time per iteration (CUDA events), peak compressed bytes, trials run, and
    the marked item's probability against sin^2((2k+1) theta)."""
    import math

    import torch

    from paper_1911_04034_gb300 import qcsim

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    n, iters = args.grover_n, args.grover_iters
    gates, marked = Cc.grover(n, iters, seed=SEED)
    per_iter = 4 * n + 2
    raw = 16 << n
    runs = [r for r in (("C only", 0), ("exhaustive", 1), ("network", 2)) if str(r[1]) in args.selectors.split(",")]
    wb, nrows, loss, train_s = None, 0, None, 0.0
    if any(sel == 2 for _, sel in runs):
        t0 = time.perf_counter()
        wb, nrows, loss = train_selector(qcsim, args.eps, SEED)
        train_s = time.perf_counter() - t0
    theta = math.asin(2.0 ** (-n / 2))
    out = {}
    for name, sel in runs:
        stream = torch.cuda.Stream()
        pool = int(args.pool_gb * 1e9) if args.pool_gb else raw + raw // 8
        budget = pool if args.ladder == 2 else raw // 4
        s = qcsim.Sim(n, 20, args.eps, chunk_log2=args.kc, budget=budget, ladder=args.ladder, pool_bytes=pool,
                      stream=stream)
        if sel == 2:
            s.set_selector(2, wb)
        else:
            s.set_selector(sel)
        if args.cache:
            s.set_block_cache(True)
        s.apply_circuit(gates[:n])
        st0 = s.stats()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(iters + 1)]
        ev[0].record(stream)
        for k in range(iters):
            s.apply_circuit(gates[n + k * per_iter: n + (k + 1) * per_iter])
            ev[k + 1].record(stream)
        ev[-1].synchronize()
        ms = [ev[k].elapsed_time(ev[k + 1]) for k in range(iters)]
        st = s.stats()
        a = s.amplitudes(marked, 1)[0]
        out[name] = {"ms_per_iteration": ms, "amp_updates_per_s": (st["amp_updates"] - st0["amp_updates"]) / (sum(ms) * 1e-3),
                     "max_encoded_gb": st["max_encoded_bytes"] / 1e9, "min_compression_ratio": st["min_ratio"],
                     "split_trials": st["split_trials"], "palette_trials": st["palette_trials"],
                     "eps_switch_gate": st["eps_switch_gate"],
                     "p_marked": abs(a) ** 2, "p_closed_form": math.sin((2 * iters + 1) * theta) ** 2,
                     "fidelity_lb_sum": st["fidelity_lb_sum"], "cache_lookups": st["cache_lookups"],
                     "cache_hits": st["cache_hits"], "peak_pages_gb": st["peak_pages_bytes"] / 1e9,
                     "device_gb": st["device_bytes"] / 1e9, "eps_final": st["eps_current"]}
        s.close()
    head = out[runs[-1][0]]
    ratios = {}
    if len(out) == 3:
        ratios = {"network_vs_c_only_peak_bytes": out["network"]["max_encoded_gb"] / out["C only"]["max_encoded_gb"],
                  "network_vs_exhaustive_peak_bytes": out["network"]["max_encoded_gb"] / out["exhaustive"]["max_encoded_gb"],
                  "network_vs_exhaustive_trials": (out["network"]["split_trials"] + out["network"]["palette_trials"])
                  / max(1, out["exhaustive"]["split_trials"] + out["exhaustive"]["palette_trials"])}
    return {"metric": METRIC, "value": head["amp_updates_per_s"], "unit": UNIT, "n_gpus": 1, "steps": iters,
            "warmup": 0, "ms_per_step": sum(head["ms_per_iteration"]) / iters, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"Grover search {n} qubits, {iters} iterations ({per_iter} gates each), eps {args.eps}, "
                                   + (f"guarded ladder in a {args.pool_gb:g} GB pool" if args.ladder == 2 else "budget raw/4")
                                   + f", chunks 2^{args.kc}; selectors compared"
                                   + ("; block cache on" if args.cache else ""),
                       "n_qubits": n, "marked": marked, "block_cache": bool(args.cache)},
            "selector": {"train_rows": nrows, "train_loss": loss, "train_seconds": train_s},
            "selectors": out, **ratios}


def _oracle_sample(job: tuple) -> tuple[int, float, int]:
    """One oracle run on the host: the random-circuit family on a 4 x 5 grid (20 qubits),
    the same bound and budget rule, whole layers timed after a warm-up until budget_s.
    Returns (amplitude updates, seconds, timed layers)."""
    eps, seed, warm_layers, timed_layers, budget_s = job
    import oracle as O

    n, rows, cols = 20, 4, 5
    depth = warm_layers + timed_layers
    gates = Cc.rcs(rows, cols, depth, seed=seed)
    out = [gates[:n]]
    pos = n
    for layer in range(depth):
        m = len(Cc.grid_edges(rows, cols, n, layer % 4)) + n
        out.append(gates[pos:pos + m])
        pos += m
    cs = O.CSim(n, n - 10, CHUNK_LOG2, eps, (16 << n) // 4)  # 2^10 blocks, as at 30 qubits
    for L in out[: 1 + warm_layers]:
        cs.apply(L)
    t0 = time.perf_counter()
    upd = k = 0
    for L in out[1 + warm_layers:]:
        cs.apply(L)
        upd += amp_updates(L, n, min(CHUNK_LOG2, n))
        k += 1
        if time.perf_counter() - t0 > budget_s:
            break
    return upd, time.perf_counter() - t0, k


def _oracle_cfg2_gate(job: tuple) -> tuple[int, float]:
    """The oracle on the random-circuit configuration's own 30-qubit circuit: its first
    gate on |0...0>, a whole-state pass like every later gate.  Returns (amplitude
    updates, seconds)."""
    eps, seed, rows, cols = job
    import oracle as O

    n = rows * cols
    gates = Cc.rcs(rows, cols, 1, seed=seed)
    cs = O.CSim(n, BLOCK_LOG2, CHUNK_LOG2, eps, (16 << n) // 4)
    t0 = time.perf_counter()
    cs.apply(gates[:1])
    dt = time.perf_counter() - t0
    upd = amp_updates(gates[:1], n, CHUNK_LOG2)
    cs.close()
    return upd, dt


def cpu_sample(eps: float, warm_layers: int = 3, timed_layers: int = 2, budget_s: float = 20.0) -> dict:
    """The oracle on the host cores.  The baseline proper is the configuration's own
    circuit: one process per core at once (started with spawn), each applying the first
    gate of the 30-qubit circuit (a whole-state pass, about 45 s of one core); value =
    all processes' updates / the slowest one's time.  The first 50 gates of that circuit
    would take about 50 times one gate's time on each core.  Beside it, the 20-qubit
    sample of the same family (whole layers after a warm-up, one circuit seed per core)."""
    import multiprocessing as mp

    cores = host_cores()
    with mp.get_context("spawn").Pool(cores) as pool:
        res = pool.map(_oracle_cfg2_gate, [(eps, SEED, ROWS, COLS)] * cores)
    upd = sum(r[0] for r in res)
    wall = max(r[1] for r in res)
    u1, s1, _ = _oracle_sample((eps, SEED, warm_layers, timed_layers, budget_s))
    with mp.get_context("spawn").Pool(cores) as pool:
        res20 = pool.map(_oracle_sample, [(eps, SEED + c, warm_layers, timed_layers, budget_s) for c in range(cores)])
    n = ROWS * COLS
    return {"value": upd / wall, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"CPU oracle on the {ROWS}x{COLS} random circuit ({n} qubits), eps {eps}: its first gate (a "
                      f"whole-state pass of 2^{n} amplitudes) applied by {cores} single-threaded processes at once; "
                      f"the first 50 gates extrapolate to 50 x {wall:.1f} s per core",
            "seconds": wall, "single_core_value": res[0][0] / min(r[1] for r in res),
            "stand_in_20q": {"value": sum(r[0] for r in res20) / max(r[1] for r in res20), "cores": cores,
                             "single_core_value": u1 / s1,
                             "sample": f"CPU oracle, random circuit 4x5 grid (20 qubits), eps {eps}, budget raw/4, "
                                       f"{timed_layers} layers after the Hadamard layer + {warm_layers} warm-up layers, "
                                       f"one circuit seed per process"}}


def host_cores() -> int:
    """Cores this process may run on."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def run_reference(args) -> dict | None:
    """The oracle as it stands on the host cores: one single-threaded process per core,
    each on its own seeded 20-qubit sample of the random-circuit workload; `steps` timed
    layers after the Hadamard layer and `warmup` layers; all updates over the slowest
    process's time."""
    import multiprocessing as mp

    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return None
    cores = host_cores()
    job = lambda c: (args.eps, SEED + c, args.warmup, args.steps, float("inf"))
    with mp.get_context("spawn").Pool(cores) as pool:
        res = pool.map(_oracle_sample, [job(c) for c in range(cores)])
    upd = sum(r[0] for r in res)
    s = max(r[1] for r in res)
    v = upd / s
    sample = (f"CPU oracle, random circuit 4x5 grid (20 qubits), eps {args.eps}, {args.steps} timed layers after the "
              f"Hadamard layer + {args.warmup} warm-up layers, {cores} single-threaded processes at once "
              f"(one circuit seed each)")
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": int(os.environ.get("WORLD_SIZE", "1")),
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": s * 1e3 / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": sample, "n_qubits": 20, "eps": args.eps},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=8)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--eps", type=float, default=1e-4)
    ap.add_argument("--no-sv", action="store_true", help="skip the uncompressed comparator and fidelity")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--phases", action="store_true", help="also count SM cycles per phase of the fused kernel")
    ap.add_argument("--workload", default="rcs30", choices=["rcs30", "batch", "qaoa34", "grover"],
                    help="rcs30: the 30-qubit random circuit (default); batch: 256 circuits of 14-24 qubits; "
                         "qaoa34: 34-qubit QAOA in a 180 GB pool; grover: chunk-mode selectors on Grover search")
    ap.add_argument("--grover-n", type=int, default=32)
    ap.add_argument("--grover-iters", type=int, default=8)
    ap.add_argument("--pool-gb", type=float, default=0.0, help="grover: page pool in GB (default raw x 9/8)")
    ap.add_argument("--ladder", type=int, default=0, help="grover: controller ladder (2 = guarded, budget = pool)")
    ap.add_argument("--selectors", default="0,1,2", help="grover: which selectors to run (0 C only, 1 exhaustive, 2 network)")
    ap.add_argument("--cache", action="store_true", help="grover: switch the compressed block cache on")
    ap.add_argument("--echo", action="store_true",
                    help="qaoa34: after the timed run, run the inverse circuit (untimed) and report |<0|state>|")
    ap.add_argument("--batch", type=int, default=256)
    ap.add_argument("--rows", type=int, default=5, help="grid rows (profiling cases use smaller grids)")
    ap.add_argument("--cols", type=int, default=6)
    ap.add_argument("--kc", type=int, default=CHUNK_LOG2, help="chunk_log2 (amplitudes per coded chunk = 2^kc)")
    ap.add_argument("--no-fast", action="store_true", help="every work item through the general gate kernel")
    ap.add_argument("--no-sweep", action="store_true", help="skip the depth-20 runs at 1e-5 and 1e-3")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched workload summary in the default run")
    args = ap.parse_args()
    global ROWS, COLS, BLOCK_LOG2
    ROWS, COLS = args.rows, args.cols
    BLOCK_LOG2 = min(20, ROWS * COLS - 10)
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.workload == "batch" and args.impl == "gpu":
        print(json.dumps(run_batch(args)), flush=True)
        return
    if args.workload == "qaoa34" and args.impl == "gpu":
        print(json.dumps(run_qaoa34(args)), flush=True)
        return
    if args.workload == "grover" and args.impl == "gpu":
        print(json.dumps(run_grover(args)), flush=True)
        return
    if args.impl == "reference":
        out = run_reference(args)
        if out is not None:
            print(json.dumps(out), flush=True)
        return
    out = run_gpu(args)
    if out is None:
        return
    if not args.no_cpu_baseline and out["n_gpus"] == 1:
        out["cpu_baseline"] = cpu_sample(args.eps)
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
