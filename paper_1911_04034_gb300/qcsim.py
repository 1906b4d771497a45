"""ctypes binding of libqcsim (include/qcsim.h): argument marshalling only.

Every step of the simulation runs in the library's CUDA kernels.  There is no CPU
fallback: if libqcsim.so cannot be loaded this module raises.  Device buffers may be
torch CUDA tensors (their data_ptr() is passed through); host buffers are numpy
arrays.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

OK, ERR_INVALID, ERR_OOM, ERR_CUDA, ERR_CORRUPT, ERR_TIMEOUT, ERR_STATE = 0, -1, -2, -3, -4, -5, -6
STATUS_NAMES = {0: "SIM_OK", -1: "SIM_ERR_INVALID", -2: "SIM_ERR_OOM", -3: "SIM_ERR_CUDA", -4: "SIM_ERR_CORRUPT",
                -5: "SIM_ERR_TIMEOUT", -6: "SIM_ERR_STATE"}

# sim_gate: int32 target, int32 kind, uint64 ctrl_mask, uint64 ctrl_vals, double u[8]
SIM_GATE = np.dtype([("target", "<i4"), ("kind", "<i4"), ("ctrl_mask", "<u8"), ("ctrl_vals", "<u8"),
                     ("u", "<f8", (8,))])
assert SIM_GATE.itemsize == 88


class SimError(RuntimeError):
    def __init__(self, code: int, call: str, msg: str):
        super().__init__(f"{call}: {STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


class Stats(C.Structure):
    _fields_ = [
        ("gates", C.c_uint64), ("encoded_bytes", C.c_uint64), ("max_encoded_bytes", C.c_uint64),
        ("raw_bytes", C.c_uint64), ("inflight_bytes", C.c_uint64), ("chunks_by_mode", C.c_uint64 * 8),
        ("pool_bytes", C.c_uint64), ("pages_in_use_bytes", C.c_uint64), ("peak_pages_bytes", C.c_uint64),
        ("device_bytes", C.c_uint64), ("amp_updates", C.c_uint64),
        ("ratio", C.c_double), ("min_ratio", C.c_double), ("eps_current", C.c_double),
        ("fidelity_lb_sum", C.c_double), ("fidelity_lb_prod", C.c_double), ("eps_switch_gate", C.c_int64),
        ("sig_bits_current", C.c_int32), ("level", C.c_int32), ("chunk_log2", C.c_int32), ("block_log2", C.c_int32),
        ("phase_cycles", C.c_uint64 * 6),
        ("split_trials", C.c_uint64),
        ("cache_lookups", C.c_uint64), ("cache_hits", C.c_uint64),
        ("fast_items", C.c_uint64), ("fast_deferred", C.c_uint64), ("kernel_launches", C.c_uint64),
        ("palette_trials", C.c_uint64), ("graph_replays", C.c_uint64), ("ladder", C.c_int32),
        ("modes", C.c_uint32), ("wide_images", C.c_uint64),
    ]

    def as_dict(self) -> dict:
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["chunks_by_mode"] = list(self.chunks_by_mode)
        d["phase_cycles"] = list(self.phase_cycles)
        return d


class TunePoint(C.Structure):
    _fields_ = [("block_log2", C.c_int32), ("chunk_log2", C.c_int32), ("ladder", C.c_int32), ("modes", C.c_uint32),
                ("rate", C.c_double), ("ratio", C.c_double), ("fidelity_lb_sum", C.c_double)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def lib():
    """Loads libqcsim.so (building it first if the sources are newer)."""
    global _lib
    if _lib is None:
        path = _build.build()
        if not os.path.exists(path):
            raise RuntimeError("libqcsim.so is missing; the CUDA library must be built (nvcc, sm_103a)")
        L = C.CDLL(path)
        vp, u64, i32, dbl, sz = C.c_void_p, C.c_uint64, C.c_int, C.c_double, C.c_size_t
        pp = C.POINTER(C.c_void_p)
        sig = {
            "sim_create": [i32, i32, dbl, pp],
            "sim_create_ex": [i32, i32, i32, dbl, u64, dbl, i32, u64, pp],
            "sim_destroy": [vp],
            "sim_checkpoint_size": [vp, C.POINTER(C.c_uint64)],
            "sim_set_block_cache": [vp, i32],
            "sim_set_budget": [vp, u64],
            "sim_set_option": [vp, C.c_char_p, C.c_int64],
            "sim_batch_run": [i32, vp, vp, vp, dbl, vp],
            "sim_checkpoint_save": [vp, vp, u64, i32],
            "sim_checkpoint_load": [vp, vp, u64, i32],
            "sim_set_stream": [vp, vp],
            "sim_apply_gate": [vp, vp],
            "sim_apply_circuit": [vp, vp, sz],
            "sim_sync": [vp],
            "sim_amplitudes": [vp, u64, u64, vp, i32],
            "sim_measure": [vp, u64, C.POINTER(C.c_uint64), C.POINTER(C.c_double)],
            "sim_fidelity": [vp, vp, i32, C.POINTER(C.c_double), vp, vp],
            "sim_stats": [vp, C.POINTER(Stats)],
            "sim_chunk_image": [vp, u64, vp, sz, C.POINTER(C.c_size_t)],
            "sim_layout": [vp, C.POINTER(C.c_uint64), C.POINTER(C.c_int), C.POINTER(C.c_int)],
            "sim_codec_encode": [vp, u64, i32, dbl, i32, vp, u64, vp, i32],
            "sim_codec_decode": [vp, u64, vp, u64, i32, vp, i32],
            "sim_codec_encode_ex": [vp, u64, i32, dbl, i32, C.c_uint32, vp, u64, vp, i32],
            "sim_set_modes": [vp, C.c_uint32],
            "sim_codec_encode_noalloc": [vp, u64, i32, dbl, i32, vp, u64, vp],
            "sim_batch_apply": [vp, i32, vp, vp, i32],
            "sim_autotune_chunk": [i32, i32, dbl, vp, sz, vp, i32, C.POINTER(C.c_int), vp],
            "sim_autotune": [i32, dbl, vp, sz, vp, i32, vp, i32, vp, i32, vp, i32, C.POINTER(TunePoint), vp, sz,
                             C.POINTER(C.c_size_t)],
            "sim_reset": [vp],
            "sim_set_timing": [vp, i32],
            "sim_set_selector": [vp, i32, vp],
            "sim_trace": [vp, u64],
            "sim_trace_read": [vp, vp, u64, C.POINTER(C.c_uint64)],
            "sim_mlp_train": [vp, vp, vp, u64, i32, i32, C.c_float, u64, vp, vp, C.POINTER(C.c_float)],
            "sim_mlp_grad": [vp, vp, vp, vp, u64, vp, C.POINTER(C.c_float)],
            "sim_timing": [vp, C.POINTER(C.c_double), C.POINTER(C.c_uint64), C.POINTER(C.c_uint64),
                           C.POINTER(C.c_uint64)],
            "sim_timing_launches": [vp, u64, vp, vp, vp, C.POINTER(C.c_uint64)],
            "sim_sv_create": [i32, pp],
            "sim_sv_destroy": [vp],
            "sim_sv_set_stream": [vp, vp],
            "sim_sv_apply_circuit": [vp, vp, sz],
            "sim_sv_amplitudes": [vp, u64, u64, vp, i32],
            "sim_sv_data": [vp, C.POINTER(C.c_void_p)],
        }
        for name, args in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = C.c_int
        L.sim_last_error.restype = C.c_char_p
        L.sim_last_error.argtypes = []
        _lib = L
    return _lib


def _check(rc: int, call: str) -> None:
    if rc != OK:
        raise SimError(rc, call, lib().sim_last_error().decode(errors="replace"))


def gates_array(gates) -> np.ndarray:
    """Copies gate records (fields target, kind, ctrl_mask, ctrl_vals, u) into the
    sim_gate layout."""
    src = np.atleast_1d(np.asarray(gates))
    out = np.zeros(src.shape[0], dtype=SIM_GATE)
    for f in SIM_GATE.names:
        out[f] = src[f]
    return out


def _ptr(x) -> int:
    """Address of a numpy array or a torch tensor."""
    if hasattr(x, "data_ptr"):
        return int(x.data_ptr())
    return int(x.ctypes.data)


def _is_device(x) -> bool:
    return bool(getattr(x, "is_cuda", False))


class Sim:
    """A compressed n-qubit state on the GPU (sim_t)."""

    def __init__(self, n_qubits: int, block_log2: int, err_bound: float, chunk_log2: int | None = None,
                 budget: int | None = None, tau: float = 0.9, ladder: int = 0, pool_bytes: int = 0, stream=None):
        h = C.c_void_p()
        if chunk_log2 is None and budget is None and tau == 0.9 and ladder == 0 and not pool_bytes:
            _check(lib().sim_create(n_qubits, block_log2, float(err_bound), C.byref(h)), "sim_create")
        else:
            kc = min(10, block_log2) if chunk_log2 is None else chunk_log2
            if budget is None:
                budget = (16 << n_qubits) + 16 * (1 << max(0, n_qubits - kc)) + 4096
            _check(lib().sim_create_ex(n_qubits, block_log2, kc, float(err_bound), int(budget), float(tau),
                                       int(ladder), int(pool_bytes), C.byref(h)), "sim_create_ex")
        self._h = h
        self.n = n_qubits
        nc, kc_, b_ = C.c_uint64(), C.c_int(), C.c_int()
        _check(lib().sim_layout(self._h, C.byref(nc), C.byref(kc_), C.byref(b_)), "sim_layout")
        self.n_chunks, self.chunk_log2, self.block_log2 = int(nc.value), int(kc_.value), int(b_.value)
        if stream is not None:
            self.set_stream(stream)

    def close(self) -> None:
        if self._h:
            _check(lib().sim_destroy(self._h), "sim_destroy")
            self._h = None

    def reset(self) -> None:
        """Back to |0...0>, the lossless stage and zero statistics; settings kept."""
        _check(lib().sim_reset(self._h), "sim_reset")

    def __del__(self):
        try:
            if getattr(self, "_h", None):
                lib().sim_destroy(self._h)
                self._h = None
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_stream(self, stream) -> None:
        handle = getattr(stream, "cuda_stream", stream)
        _check(lib().sim_set_stream(self._h, C.c_void_p(int(handle))), "sim_set_stream")

    def apply_gate(self, gate) -> None:
        g = gates_array(gate)
        _check(lib().sim_apply_gate(self._h, C.c_void_p(_ptr(g))), "sim_apply_gate")

    def apply_circuit(self, gates) -> None:
        g = gates_array(gates)
        _check(lib().sim_apply_circuit(self._h, C.c_void_p(_ptr(g)), g.shape[0]), "sim_apply_circuit")

    def set_modes(self, modes: int) -> None:
        """0x1F: Solution C modes (default); bit 5 adds SPLIT (Solution D), bit 6 PALETTE."""
        _check(lib().sim_set_modes(self._h, int(modes)), "sim_set_modes")

    def set_selector(self, selector: int, bf16_params=None) -> None:
        """0 the mode set (default Solution C), 1 every mode with the SPLIT and PALETTE
        trials on every chunk (exhaustive), 2 Solution C plus the trials the selector
        network grants each chunk before the gate (bf16_params: 1864 uint16)."""
        p = None
        if bf16_params is not None:
            p = np.ascontiguousarray(bf16_params, dtype=np.uint16)
            assert p.size == 1864
        _check(lib().sim_set_selector(self._h, int(selector), C.c_void_p(_ptr(p)) if p is not None else None),
               "sim_set_selector")

    def set_budget(self, nbytes: int) -> None:
        """The controller's budget from the next gate on (see sim_set_budget)."""
        _check(lib().sim_set_budget(self._h, int(nbytes)), "sim_set_budget")

    def set_option(self, key: str, value: int) -> None:
        """A named setting (see sim_set_option)."""
        _check(lib().sim_set_option(self._h, key.encode(), int(value)), "sim_set_option")

    def set_block_cache(self, on: bool = True) -> None:
        """Section 3.4 compressed block cache for later gates (see sim_set_block_cache)."""
        _check(lib().sim_set_block_cache(self._h, int(bool(on))), "sim_set_block_cache")

    def checkpoint(self, out=None):
        """The compressed state as a checkpoint (Section 3.5): a numpy uint8 array, or
        written into `out` (a torch CUDA uint8 tensor large enough) and returned."""
        n = C.c_uint64()
        _check(lib().sim_checkpoint_size(self._h, C.byref(n)), "sim_checkpoint_size")
        if out is None:
            out = np.zeros(n.value, dtype=np.uint8)
        _check(lib().sim_checkpoint_save(self._h, C.c_void_p(_ptr(out)), int(n.value), int(_is_device(out))),
               "sim_checkpoint_save")
        return out

    def restore(self, ck) -> None:
        """Replaces the state with a checkpoint (numpy uint8 array / bytes, or a torch
        CUDA uint8 tensor)."""
        if isinstance(ck, (bytes, bytearray)):
            ck = np.frombuffer(bytes(ck), dtype=np.uint8).copy()
        size = ck.numel() if _is_device(ck) else ck.size
        _check(lib().sim_checkpoint_load(self._h, C.c_void_p(_ptr(ck)), int(size), int(_is_device(ck))),
               "sim_checkpoint_load")

    def trace(self, capacity: int) -> None:
        _check(lib().sim_trace(self._h, int(capacity)), "sim_trace")

    def trace_read(self, cap: int = 1 << 20) -> np.ndarray:
        """Records as an array of shape (n, 20)."""
        out = np.zeros((cap, 20), dtype=np.float32)
        n = C.c_uint64()
        _check(lib().sim_trace_read(self._h, C.c_void_p(_ptr(out)), cap, C.byref(n)), "sim_trace_read")
        return out[: n.value]

    def sync(self) -> None:
        _check(lib().sim_sync(self._h), "sim_sync")

    def amplitudes(self, first: int = 0, count: int | None = None, out=None):
        """Decoded amplitudes as complex128 (numpy), or into `out` (numpy complex128 or
        a torch CUDA tensor of 2*count float64)."""
        if count is None:
            count = (1 << self.n) - first
        if out is None:
            out = np.zeros(count, dtype=np.complex128)
        _check(lib().sim_amplitudes(self._h, first, count, C.c_void_p(_ptr(out)), int(_is_device(out))),
               "sim_amplitudes")
        return out

    def measure(self, seed: int) -> tuple[int, float]:
        o, p = C.c_uint64(), C.c_double()
        _check(lib().sim_measure(self._h, C.c_uint64(seed), C.byref(o), C.byref(p)), "sim_measure")
        return int(o.value), float(p.value)

    def fidelity(self, ref) -> dict:
        """F = |<ref|psi>| against a full reference state (numpy complex128, or a torch
        CUDA tensor)."""
        if not _is_device(ref):
            ref = np.ascontiguousarray(ref, dtype=np.complex128)
        F = C.c_double()
        ri = np.zeros(2)
        nn = np.zeros(1)
        _check(lib().sim_fidelity(self._h, C.c_void_p(_ptr(ref)), int(_is_device(ref)), C.byref(F),
                                  C.c_void_p(_ptr(ri)), C.c_void_p(_ptr(nn))), "sim_fidelity")
        return {"F": float(F.value), "overlap": complex(ri[0], ri[1]), "norm2": float(nn[0])}

    def stats(self) -> dict:
        st = Stats()
        _check(lib().sim_stats(self._h, C.byref(st)), "sim_stats")
        return st.as_dict()

    def set_timing(self, on) -> None:
        """0 off, 1 gate-kernel events, 2 events and per-phase SM cycles."""
        _check(lib().sim_set_timing(self._h, int(on)), "sim_set_timing")

    def timing(self) -> dict:
        """Gate-kernel time (CUDA events), launches and image bytes read/written since
        the last call (or since timing was switched on)."""
        ms, n, rd, wr = C.c_double(), C.c_uint64(), C.c_uint64(), C.c_uint64()
        _check(lib().sim_timing(self._h, C.byref(ms), C.byref(n), C.byref(rd), C.byref(wr)), "sim_timing")
        return {"gate_kernel_ms": float(ms.value), "launches": int(n.value), "bytes_read": int(rd.value),
                "bytes_written": int(wr.value)}

    def timing_launches(self) -> dict:
        """Per gate-kernel launch since timing was switched on or last read by timing():
        CUDA-event ms and image bytes read / written (call before timing())."""
        n = C.c_uint64()
        _check(lib().sim_timing_launches(self._h, 0, None, None, None, C.byref(n)), "sim_timing_launches")
        k = int(n.value)
        ms = np.zeros(k, dtype=np.float32)
        rd = np.zeros(k, dtype=np.uint64)
        wr = np.zeros(k, dtype=np.uint64)
        if k:
            _check(lib().sim_timing_launches(self._h, k, C.c_void_p(_ptr(ms)), C.c_void_p(_ptr(rd)),
                                             C.c_void_p(_ptr(wr)), C.byref(n)), "sim_timing_launches")
        return {"ms": ms, "bytes_read": rd, "bytes_written": wr}

    def chunk_image(self, c: int) -> bytes:
        cap = 16 + (16 << self.chunk_log2) + 64
        buf = np.zeros(cap, dtype=np.uint8)
        ln = C.c_size_t()
        _check(lib().sim_chunk_image(self._h, c, C.c_void_p(_ptr(buf)), cap, C.byref(ln)), "sim_chunk_image")
        return buf[: ln.value].tobytes()


def batch_apply(sims: list, circuits: list, use_graph: bool = True) -> None:
    """Runs circuits[k] on sims[k] for all k in shared launches (sim_batch_apply)."""
    arrs = [gates_array(c) for c in circuits]
    n = len(sims)
    handles = (C.c_void_p * n)(*[s._h.value for s in sims])
    ptrs = (C.c_void_p * n)(*[_ptr(a) if a.size else 0 for a in arrs])
    counts = (C.c_size_t * n)(*[a.shape[0] for a in arrs])
    _check(lib().sim_batch_apply(C.cast(handles, C.c_void_p), n, C.cast(ptrs, C.c_void_p), C.cast(counts, C.c_void_p),
                                 int(bool(use_graph))), "sim_batch_apply")


def batch_run(circuits: list, n_qubits: list, err_bound: float) -> list[dict]:
    """Runs independent circuits through the batched path (see sim_batch_run); returns
    each circuit's statistics."""
    arrs = [gates_array(g) for g in circuits]
    k = len(arrs)
    ptrs = (C.c_void_p * k)(*[_ptr(a) for a in arrs])
    ns = (C.c_size_t * k)(*[a.shape[0] for a in arrs])
    qs = (C.c_int * k)(*[int(n) for n in n_qubits])
    out = (Stats * k)()
    _check(lib().sim_batch_run(k, C.cast(qs, C.c_void_p), C.cast(ptrs, C.c_void_p), C.cast(ns, C.c_void_p),
                               float(err_bound), C.cast(out, C.c_void_p)), "sim_batch_run")
    return [out[i].as_dict() for i in range(k)]


def autotune_chunk(n_qubits: int, block_log2: int, err_bound: float, probe, candidates=(8, 9, 10, 11)):
    """Returns (best chunk_log2, {candidate: amplitude updates/s of kernel time})."""
    g = gates_array(probe)
    cand = (C.c_int * len(candidates))(*candidates)
    rates = np.zeros(len(candidates))
    best = C.c_int()
    _check(lib().sim_autotune_chunk(n_qubits, block_log2, float(err_bound), C.c_void_p(_ptr(g)), g.shape[0],
                                    C.cast(cand, C.c_void_p), len(candidates), C.byref(best), C.c_void_p(_ptr(rates))),
           "sim_autotune_chunk")
    return int(best.value), dict(zip(candidates, rates.tolist()))


def autotune(n_qubits: int, err_bound: float, probe, block_log2s=(16, 10, 11, 12, 13, 14, 15), chunk_log2s=(10, 9, 8),
             ladders=(0, 1, 2), mode_sets=(0x1F, 0x5F)):
    """Coordinate-descent autotuner over block size, tile (chunk) size and codec
    schedule (sim_autotune); returns (best point, every measured point) as dicts."""
    g = gates_array(probe)
    bs = (C.c_int32 * len(block_log2s))(*block_log2s)
    cs = (C.c_int32 * len(chunk_log2s))(*chunk_log2s)
    ls = (C.c_int32 * len(ladders))(*ladders)
    ms = (C.c_uint32 * len(mode_sets))(*mode_sets)
    best = TunePoint()
    cap = len(block_log2s) * len(chunk_log2s) * len(ladders) * len(mode_sets)
    tried = (TunePoint * cap)()
    n = C.c_size_t()
    _check(lib().sim_autotune(int(n_qubits), float(err_bound), C.c_void_p(_ptr(g)), g.shape[0], C.cast(bs, C.c_void_p),
                              len(block_log2s), C.cast(cs, C.c_void_p), len(chunk_log2s), C.cast(ls, C.c_void_p),
                              len(ladders), C.cast(ms, C.c_void_p), len(mode_sets), C.byref(best),
                              C.cast(tried, C.c_void_p), cap, C.byref(n)), "sim_autotune")
    return best.as_dict(), [tried[i].as_dict() for i in range(min(n.value, cap))]


def mlp_grad(params, x, mode, sizes):
    """(loss, gradient) of the selector loss at bfloat16(params), computed on the GPU."""
    p = np.ascontiguousarray(params, dtype=np.float32)
    xx = np.ascontiguousarray(x, dtype=np.float32)
    m = np.ascontiguousarray(mode, dtype=np.int32)
    sz = np.ascontiguousarray(sizes, dtype=np.float32)
    g = np.zeros(1864, dtype=np.float32)
    loss = C.c_float()
    _check(lib().sim_mlp_grad(C.c_void_p(_ptr(p)), C.c_void_p(_ptr(xx)), C.c_void_p(_ptr(m)), C.c_void_p(_ptr(sz)),
                              m.size, C.c_void_p(_ptr(g)), C.byref(loss)), "sim_mlp_grad")
    return float(loss.value), g


def mlp_train(x, mode, sizes, params, epochs: int = 20, batch: int = 256, lr: float = 3e-3, seed: int = 1):
    """Trains the selector on the GPU; returns (float32 params, bfloat16 params as
    uint16, last epoch's loss)."""
    p = np.ascontiguousarray(params, dtype=np.float32).copy()
    xx = np.ascontiguousarray(x, dtype=np.float32)
    m = np.ascontiguousarray(mode, dtype=np.int32)
    sz = np.ascontiguousarray(sizes, dtype=np.float32)
    wb = np.zeros(1864, dtype=np.uint16)
    loss = C.c_float()
    _check(lib().sim_mlp_train(C.c_void_p(_ptr(xx)), C.c_void_p(_ptr(m)), C.c_void_p(_ptr(sz)), m.size, int(epochs),
                               int(batch), C.c_float(lr), C.c_uint64(seed), C.c_void_p(_ptr(p)), C.c_void_p(_ptr(wb)),
                               C.byref(loss)), "sim_mlp_train")
    return p, wb, float(loss.value)


def codec_stride(chunk_log2: int) -> int:
    need = 16 + (16 << chunk_log2) + (1 << chunk_log2) // 2 + 32
    return (need + 15) // 16 * 16


def codec_encode(values, chunk_log2: int, eps: float, force_mode: int = -1, modes: int = 0x1F):
    """Encodes chunks with the device encoder.  values: numpy complex128 of
    n_chunks * 2^chunk_log2 amplitudes (host) or a torch CUDA float64 tensor.
    Returns (images as a list of bytes, lengths) for host input; for device input
    returns (image buffer tensor, lengths tensor, stride)."""
    stride = codec_stride(chunk_log2)
    if _is_device(values):
        import torch

        n = values.numel() // (2 << chunk_log2)
        out = torch.zeros(n * stride, dtype=torch.uint8, device=values.device)
        lens = torch.zeros(n, dtype=torch.int32, device=values.device)
        _check(lib().sim_codec_encode_ex(C.c_void_p(_ptr(values)), n, chunk_log2, float(eps), force_mode, modes,
                                         C.c_void_p(_ptr(out)), stride, C.c_void_p(_ptr(lens)), 1), "sim_codec_encode")
        return out, lens, stride
    x = np.ascontiguousarray(values, dtype=np.complex128)
    n = x.size >> chunk_log2
    assert n << chunk_log2 == x.size
    out = np.zeros(n * stride, dtype=np.uint8)
    lens = np.zeros(n, dtype=np.uint32)
    _check(lib().sim_codec_encode_ex(C.c_void_p(_ptr(x)), n, chunk_log2, float(eps), force_mode, modes,
                                     C.c_void_p(_ptr(out)), stride, C.c_void_p(_ptr(lens)), 0), "sim_codec_encode")
    return [out[k * stride: k * stride + int(lens[k])].tobytes() for k in range(n)], lens


def codec_encode_noalloc(values, chunk_log2: int, eps: float, force_mode: int = -1):
    """Like codec_encode for host arrays, through sim_codec_encode_noalloc: the
    library stages the call in its fixed device array instead of allocating."""
    stride = codec_stride(chunk_log2)
    x = np.ascontiguousarray(values, dtype=np.complex128)
    n = x.size >> chunk_log2
    assert n << chunk_log2 == x.size
    out = np.zeros(max(1, n) * stride, dtype=np.uint8)
    lens = np.zeros(max(1, n), dtype=np.uint32)
    _check(lib().sim_codec_encode_noalloc(C.c_void_p(_ptr(x)), n, chunk_log2, float(eps), force_mode,
                                          C.c_void_p(_ptr(out)), stride, C.c_void_p(_ptr(lens))),
           "sim_codec_encode_noalloc")
    return [out[k * stride: k * stride + int(lens[k])].tobytes() for k in range(n)], lens[:n]


def codec_decode(images: list[bytes], chunk_log2: int) -> np.ndarray:
    """Decodes host images with the device decoder; returns complex128 amplitudes."""
    n = len(images)
    stride = max([codec_stride(chunk_log2)] + [(len(b) + 15) // 16 * 16 for b in images])
    buf = np.zeros(max(1, n) * stride, dtype=np.uint8)
    lens = np.zeros(max(1, n), dtype=np.uint32)
    for k, b in enumerate(images):
        buf[k * stride: k * stride + len(b)] = np.frombuffer(b, dtype=np.uint8)
        lens[k] = len(b)
    out = np.zeros(n << chunk_log2, dtype=np.complex128)
    _check(lib().sim_codec_decode(C.c_void_p(_ptr(buf)), stride, C.c_void_p(_ptr(lens)), n, chunk_log2,
                                  C.c_void_p(_ptr(out)), 0), "sim_codec_decode")
    return out


class StateVector:
    """Uncompressed complex128 state vector on the GPU (sim_sv_t)."""

    def __init__(self, n_qubits: int, stream=None):
        h = C.c_void_p()
        _check(lib().sim_sv_create(n_qubits, C.byref(h)), "sim_sv_create")
        self._h = h
        self.n = n_qubits
        if stream is not None:
            handle = getattr(stream, "cuda_stream", stream)
            _check(lib().sim_sv_set_stream(self._h, C.c_void_p(int(handle))), "sim_sv_set_stream")

    def close(self):
        if self._h:
            _check(lib().sim_sv_destroy(self._h), "sim_sv_destroy")
            self._h = None

    def __del__(self):
        try:
            if getattr(self, "_h", None):
                lib().sim_sv_destroy(self._h)
                self._h = None
        except Exception:
            pass

    def apply_circuit(self, gates) -> None:
        g = gates_array(gates)
        _check(lib().sim_sv_apply_circuit(self._h, C.c_void_p(_ptr(g)), g.shape[0]), "sim_sv_apply_circuit")

    def amplitudes(self, first: int = 0, count: int | None = None, out=None):
        if count is None:
            count = (1 << self.n) - first
        if out is None:
            out = np.zeros(count, dtype=np.complex128)
        _check(lib().sim_sv_amplitudes(self._h, first, count, C.c_void_p(_ptr(out)), int(_is_device(out))),
               "sim_sv_amplitudes")
        return out

    def data_ptr(self) -> int:
        p = C.c_void_p()
        _check(lib().sim_sv_data(self._h, C.byref(p)), "sim_sv_data")
        return int(p.value)
