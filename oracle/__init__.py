"""CPU oracle for compressed full-state circuit simulation -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / reference leg
of ``bench.py`` may import this package.  The simulator library never calls it, and it
shares no code with the simulator: ``qc_oracle.c`` is a plain sequential fp64
restatement of the paper (truncation and XOR coding of Section 4.2, gate application
of Eq. matrix1/matrix2, the error-bound controller of Section 3.7, fidelity of
Section 3.8), compiled with ``-ffp-contract=off`` and called here through ctypes.

Every oracle function is pinned by ``tests/test_oracle_*.py`` against facts that do not
come from the oracle itself: the constants and worked example of Eq. sigbits, hand
derived byte streams, closed forms (Grover, QFT), brute-force unitaries for n <= 6 and
invariants (norm, error bound, fidelity bound).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qc_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

OK, ERR_INVALID, ERR_OOM, ERR_CORRUPT, ERR_STATE = 0, -1, -2, -4, -6
MODE_ZERO, MODE_CONST, MODE_PERIOD, MODE_STREAM, MODE_RAW, MODE_SPLIT = 0, 1, 2, 3, 4, 5
MODE_NAMES = ("ZERO", "CONST", "PERIOD", "STREAM", "RAW", "SPLIT")
DEFAULT_MODES = 0x1F  # Solution C; SPLIT (Solution D) and PALETTE only when asked for
ALL_MODES = 0x7F      # ZERO, CONST, PERIOD, STREAM, RAW, SPLIT, PALETTE


class OracleError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"oracle {what} failed with code {code}")
        self.code = code


class _Gate(C.Structure):
    _fields_ = [
        ("target", C.c_int32),
        ("kind", C.c_int32),
        ("ctrl_mask", C.c_uint64),
        ("ctrl_vals", C.c_uint64),
        ("u", C.c_double * 8),
    ]


class _Stats(C.Structure):
    _fields_ = [
        ("gates", C.c_uint64),
        ("encoded_bytes", C.c_uint64),
        ("max_encoded_bytes", C.c_uint64),
        ("raw_bytes", C.c_uint64),
        ("inflight_bytes", C.c_uint64),
        ("chunks_by_mode", C.c_uint64 * 8),
        ("min_ratio", C.c_double),
        ("eps_current", C.c_double),
        ("fid_lb_sum", C.c_double),
        ("fid_lb_prod", C.c_double),
        ("eps_switch_gate", C.c_int64),
        ("S_current", C.c_int32),
        ("level", C.c_int32),
        ("guard_fit", C.c_int32),
        ("pad", C.c_int32),
        ("wide_images", C.c_uint64),
    ]


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (plain C11, no contraction of a*b+c)."""
    with _lock:
        if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
            return _LIB_PATH
        os.makedirs(_OUT_DIR, exist_ok=True)
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
        return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB_PATH)
        u64p, dp, u8p = C.POINTER(C.c_uint64), C.POINTER(C.c_double), C.POINTER(C.c_uint8)
        sig = {
            "orc_set_mutant": (None, [C.c_int]),
            "orc_exp_of": (C.c_int, [C.c_double]),
            "orc_sig_bits": (C.c_int, [C.c_double]),
            "orc_truncate": (C.c_uint64, [C.c_uint64, C.c_int]),
            "orc_chunk_sig_bits": (C.c_int, [u64p, C.c_size_t, C.c_int]),
            "orc_mode_sizes": (C.c_int, [u64p, C.c_int, C.c_int, u64p]),
            "orc_encode_chunk": (C.c_long, [u64p, C.c_int, C.c_int, C.c_int, u8p, C.c_size_t]),
            "orc_encode_chunk_mask": (C.c_long, [u64p, C.c_int, C.c_int, C.c_int, C.c_uint, u8p, C.c_size_t]),
            "orc_csim_set_modes": (C.c_int, [C.c_void_p, C.c_uint]),
            "orc_csim_set_mlp": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_float)]),
            "orc_mlp_forward": (None, [C.POINTER(C.c_float), C.POINTER(C.c_float), C.POINTER(C.c_float)]),
            "orc_mlp_trials": (C.c_int, [C.POINTER(C.c_float), C.POINTER(C.c_float)]),
            "orc_mlp_features": (None, [u8p, C.c_size_t, C.c_int, C.POINTER(_Gate), C.c_int, C.POINTER(C.c_float)]),
            "orc_decode_chunk": (C.c_int, [u8p, C.c_size_t, C.c_int, u64p]),
            "orc_gate_check": (C.c_int, [C.POINTER(_Gate), C.c_int]),
            "orc_sv_init": (None, [dp, C.c_int]),
            "orc_sv_apply": (C.c_int, [dp, C.c_int, C.POINTER(_Gate)]),
            "orc_sv_run": (C.c_int, [dp, C.c_int, C.POINTER(_Gate), C.c_size_t]),
            "orc_sv_norm2": (C.c_double, [dp, C.c_int]),
            "orc_sv_inner": (None, [dp, dp, C.c_int, dp]),
            "orc_splitmix64": (C.c_uint64, [C.c_uint64]),
            "orc_sv_measure": (C.c_int, [dp, C.c_int, C.c_uint64, u64p, dp]),
            "orc_csim_create": (C.c_void_p, [C.c_int, C.c_int, C.c_int, C.c_double, C.c_uint64, C.c_double, C.c_int]),
            "orc_csim_destroy": (None, [C.c_void_p]),
            "orc_csim_apply": (C.c_int, [C.c_void_p, C.POINTER(_Gate)]),
            "orc_csim_run": (C.c_int, [C.c_void_p, C.POINTER(_Gate), C.c_size_t]),
            "orc_csim_amplitudes": (C.c_int, [C.c_void_p, dp]),
            "orc_csim_image": (C.c_int, [C.c_void_p, C.c_uint64, u8p, C.c_size_t, u64p]),
            "orc_csim_set_image": (C.c_int, [C.c_void_p, C.c_uint64, u8p, C.c_size_t]),
            "orc_csim_stats": (None, [C.c_void_p, C.POINTER(_Stats)]),
            "orc_csim_nchunks": (C.c_uint64, [C.c_void_p]),
            "orc_csim_chunk_log2": (C.c_int, [C.c_void_p]),
            "orc_csim_block_log2": (C.c_int, [C.c_void_p]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(C.POINTER(ctype))


def _gates(gates) -> C.Array:
    """Copies gate records (any structured array with the fields target, kind,
    ctrl_mask, ctrl_vals, u) into the oracle's own C layout."""
    gates = np.atleast_1d(gates)
    arr = (_Gate * len(gates))()
    for k, g in enumerate(gates):
        arr[k].target = int(g["target"])
        arr[k].kind = int(g["kind"])
        arr[k].ctrl_mask = int(g["ctrl_mask"])
        arr[k].ctrl_vals = int(g["ctrl_vals"])
        for j in range(8):
            arr[k].u[j] = float(g["u"][j])
    return arr


def set_mutant(m: int) -> None:
    lib().orc_set_mutant(int(m))


# ---------------------------------------------------------------- codec ----- #

def exp_of(eps: float) -> int:
    return int(lib().orc_exp_of(float(eps)))


def sig_bits(eps: float) -> int:
    return int(lib().orc_sig_bits(float(eps)))


def truncate(bits: int, S: int) -> int:
    return int(lib().orc_truncate(C.c_uint64(int(bits) & (2**64 - 1)), int(S)))


def truncate_double(x: float, S: int) -> float:
    b = np.array([x], dtype=np.float64).view(np.uint64)[0]
    return float(np.array([truncate(int(b), S)], dtype=np.uint64).view(np.float64)[0])


def _as_bits(values) -> np.ndarray:
    v = np.ascontiguousarray(values)
    if v.dtype == np.complex128:
        v = v.view(np.float64)
    if v.dtype == np.float64:
        v = v.view(np.uint64)
    return np.ascontiguousarray(v, dtype=np.uint64)


def encode_chunk(values, kc: int, S: int, force_mode: int = -1, modes: int = DEFAULT_MODES) -> bytes:
    """values: 2^kc complex128 amplitudes (or 2^(kc+1) float64 / uint64 patterns)."""
    x = _as_bits(values)
    assert x.size == 2 << kc, (x.size, kc)
    cap = 16 + 9 * x.size + x.size // 4 + 2048 + 64  # forced STREAM or PALETTE can exceed RAW
    out = np.zeros(cap, dtype=np.uint8)
    L = lib().orc_encode_chunk_mask(_ptr(x, C.c_uint64), kc, S, force_mode, modes, _ptr(out, C.c_uint8), cap)
    if L < 0:
        raise OracleError(int(L), "encode_chunk")
    return out[:L].tobytes()


def decode_chunk(img: bytes, kc: int) -> np.ndarray:
    """Returns 2^kc complex128 amplitudes."""
    buf = np.frombuffer(bytes(img), dtype=np.uint8).copy()
    out = np.zeros(2 << kc, dtype=np.uint64)
    rc = lib().orc_decode_chunk(_ptr(buf, C.c_uint8), buf.size, kc, _ptr(out, C.c_uint64))
    if rc:
        raise OracleError(rc, "decode_chunk")
    return out.view(np.complex128)


def mode_sizes(values, kc: int, S: int) -> list[int]:
    x = _as_bits(values)
    sizes = np.zeros(8, dtype=np.uint64)
    rc = lib().orc_mode_sizes(_ptr(x, C.c_uint64), kc, S, _ptr(sizes, C.c_uint64))
    if rc:
        raise OracleError(rc, "mode_sizes")
    return [int(s) for s in sizes[:7]]


# ---------------------------------------------------------- state vector --- #

def sv_init(n: int) -> np.ndarray:
    psi = np.zeros(1 << n, dtype=np.complex128)
    lib().orc_sv_init(_ptr(psi.view(np.float64), C.c_double), n)
    return psi


def sv_run(psi: np.ndarray, n: int, gates) -> np.ndarray:
    """Applies the gates in place to a complex128 state vector."""
    g = _gates(gates)
    rc = lib().orc_sv_run(_ptr(psi.view(np.float64), C.c_double), n, g, len(g))
    if rc:
        raise OracleError(rc, "sv_run")
    return psi


def gate_check(gate_rec, n: int) -> int:
    g = _gates(gate_rec)
    return int(lib().orc_gate_check(g, n))


def sv_norm2(psi: np.ndarray, n: int) -> float:
    return float(lib().orc_sv_norm2(_ptr(psi.view(np.float64), C.c_double), n))


def sv_inner(x: np.ndarray, y: np.ndarray, n: int) -> complex:
    out = np.zeros(2, dtype=np.float64)
    lib().orc_sv_inner(_ptr(x.view(np.float64), C.c_double), _ptr(y.view(np.float64), C.c_double), n,
                       _ptr(out, C.c_double))
    return complex(out[0], out[1])


def fidelity(ideal: np.ndarray, sim: np.ndarray, n: int) -> float:
    """F = |<psi_ideal|psi_sim>| (Section 3.8, Eq. idealsim)."""
    return abs(sv_inner(ideal, sim, n))


def mlp_forward_c(params_flat, x) -> np.ndarray:
    """The C oracle's selector inference on one feature row."""
    v = np.ascontiguousarray(params_flat, dtype=np.float32)
    xx = np.ascontiguousarray(x, dtype=np.float32)
    out = np.zeros(8, dtype=np.float32)
    lib().orc_mlp_forward(_ptr(v, C.c_float), _ptr(xx, C.c_float), _ptr(out, C.c_float))
    return out


def mlp_trials_c(params_flat, x) -> int:
    """The C oracle's selector decision on one feature row: bit 0 the SPLIT trial,
    bit 1 the PALETTE trial."""
    v = np.ascontiguousarray(params_flat, dtype=np.float32)
    xx = np.ascontiguousarray(x, dtype=np.float32)
    return int(lib().orc_mlp_trials(_ptr(v, C.c_float), _ptr(xx, C.c_float)))


def mlp_features_c(img: bytes, kc: int, gate_rec, S_gate: int) -> np.ndarray:
    """The C oracle's selector inputs for a chunk whose current image is img, about to
    be rewritten by the gate (no decoded value is needed)."""
    buf = np.frombuffer(bytes(img), dtype=np.uint8).copy()
    out = np.zeros(16, dtype=np.float32)
    lib().orc_mlp_features(_ptr(buf, C.c_uint8), buf.size, kc, _gates(gate_rec), S_gate, _ptr(out, C.c_float))
    return out


def splitmix64(x: int) -> int:
    return int(lib().orc_splitmix64(C.c_uint64(int(x) & (2**64 - 1))))


def sv_measure(psi: np.ndarray, n: int, seed: int) -> tuple[int, float]:
    out = C.c_uint64(0)
    prob = C.c_double(0)
    lib().orc_sv_measure(_ptr(psi.view(np.float64), C.c_double), n, C.c_uint64(seed), C.byref(out), C.byref(prob))
    return int(out.value), float(prob.value)


# ---------------------------------------------------- compressed simulator --- #

LADDER_JUMP, LADDER_PAPER = 0, 1


class CSim:
    """The oracle's compressed simulator: chunk images, decode -> apply -> encode per
    work item, and the error-bound controller run before every gate."""

    def __init__(self, n: int, block_log2: int, chunk_log2: int, eps_max: float, budget: int, tau: float = 0.9,
                 ladder: int = LADDER_JUMP, modes: int = DEFAULT_MODES):
        self._h = lib().orc_csim_create(n, block_log2, chunk_log2, float(eps_max), int(budget), float(tau),
                                        int(ladder))
        if not self._h:
            raise OracleError(ERR_INVALID, "csim_create")
        self.n = n
        self.kc = int(lib().orc_csim_chunk_log2(self._h))
        self.b = int(lib().orc_csim_block_log2(self._h))
        if modes != DEFAULT_MODES:
            rc = lib().orc_csim_set_modes(self._h, modes)
            if rc:
                raise OracleError(rc, "csim_set_modes")
        self.nchunks = int(lib().orc_csim_nchunks(self._h))

    def close(self):
        if self._h:
            lib().orc_csim_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def apply(self, gates) -> None:
        g = _gates(gates)
        rc = lib().orc_csim_run(self._h, g, len(g))
        if rc:
            raise OracleError(rc, "csim_run")

    def amplitudes(self) -> np.ndarray:
        out = np.zeros(1 << self.n, dtype=np.complex128)
        rc = lib().orc_csim_amplitudes(self._h, _ptr(out.view(np.float64), C.c_double))
        if rc:
            raise OracleError(rc, "csim_amplitudes")
        return out

    def set_mlp(self, params_flat) -> None:
        """Solution D is tried for a chunk only where the selector network says so;
        params_flat: the network's 1864 parameters (bfloat16 values) in W1 b1 W2 b2 W3 b3 order."""
        v = np.ascontiguousarray(params_flat, dtype=np.float32)
        assert v.size == 1864
        lib().orc_csim_set_mlp(self._h, 1, _ptr(v, C.c_float))

    def image(self, c: int) -> bytes:
        cap = 16 + 16 * (1 << self.kc)
        buf = np.zeros(cap, dtype=np.uint8)
        ln = C.c_uint64(0)
        rc = lib().orc_csim_image(self._h, c, _ptr(buf, C.c_uint8), cap, C.byref(ln))
        if rc:
            raise OracleError(rc, "csim_image")
        return buf[: ln.value].tobytes()

    def set_image(self, c: int, img: bytes) -> None:
        buf = np.frombuffer(bytes(img), dtype=np.uint8).copy()
        rc = lib().orc_csim_set_image(self._h, c, _ptr(buf, C.c_uint8), buf.size)
        if rc:
            raise OracleError(rc, "csim_set_image")

    def stats(self) -> dict:
        st = _Stats()
        lib().orc_csim_stats(self._h, C.byref(st))
        d = {name: getattr(st, name) for name, _ in _Stats._fields_}
        d["chunks_by_mode"] = list(st.chunks_by_mode)
        return d
