"""The C-ABI library loads and exports every function include/qcsim.h declares (no GPU
needed: nothing is called)."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "qcsim.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(?:sim_status|const char\*)\s+(sim_\w+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("sim_create", "sim_apply_gate", "sim_amplitudes", "sim_measure", "sim_stats", "sim_destroy",
                 "sim_fidelity", "sim_codec_encode", "sim_codec_decode"):
        assert must in names


@pytest.mark.skipif(shutil.which("nvcc") is None, reason="nvcc not available to build the library")
def test_library_exports_every_declared_symbol():
    from paper_1911_04034_gb300 import build

    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_gate_struct_layout_matches_header():
    from paper_1911_04034_gb300 import qcsim

    assert qcsim.SIM_GATE.itemsize == 88
    assert [qcsim.SIM_GATE.fields[f][1] for f in ("target", "kind", "ctrl_mask", "ctrl_vals", "u")] == [0, 4, 8, 16, 24]


@pytest.mark.skipif(shutil.which("nvcc") is None, reason="nvcc not available to build the library")
def test_codec_entry_points_reject_sizes_that_would_wrap():
    """Sizes whose byte counts overflow 64 bits are refused before any device call (so
    this runs without a GPU): 2^62 chunks of 2^10 amplitudes."""
    import numpy as np

    from paper_1911_04034_gb300 import build, qcsim

    lib = ctypes.CDLL(build.build())
    lib.sim_codec_encode_noalloc.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int, ctypes.c_double,
                                             ctypes.c_int, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p]
    lib.sim_codec_encode_ex.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                        ctypes.c_uint32, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_int]
    lib.sim_codec_decode.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int,
                                     ctypes.c_void_p, ctypes.c_int]
    buf = np.zeros(64, dtype=np.uint8)
    p = ctypes.c_void_p(buf.ctypes.data)
    stride = qcsim.codec_stride(10)
    for big in (1 << 62, (1 << 64) - 1):
        assert lib.sim_codec_encode_noalloc(p, big, 10, 1e-4, -1, p, stride, p) == qcsim.ERR_INVALID
        assert lib.sim_codec_encode_ex(p, big, 10, 1e-4, -1, 0x1F, p, stride, p, 0) == qcsim.ERR_INVALID
        assert lib.sim_codec_decode(p, stride, p, big, 10, p, 0) == qcsim.ERR_INVALID
    assert lib.sim_codec_encode_noalloc(p, 1, 10, 1e-4, -1, p, (1 << 64) - 16, p) == qcsim.ERR_INVALID


@pytest.mark.skipif(shutil.which("nvcc") is None, reason="nvcc not available to build the library")
def test_entry_points_reject_bad_arguments_before_any_device_call():
    """NULL handles and out-of-range settings are refused on the host (so this runs
    without a GPU): sim_reset, sim_batch_apply, sim_set_selector and sim_autotune's lists
    (a chunk size above 11, a ladder above 2, a mode set without Solution C's modes, an
    empty list, a gate on a missing qubit)."""
    import numpy as np

    from paper_1911_04034_gb300 import build, circuits, qcsim

    lib = ctypes.CDLL(build.build())
    vp = ctypes.c_void_p
    lib.sim_reset.argtypes = [vp]
    lib.sim_batch_apply.argtypes = [vp, ctypes.c_int, vp, vp, ctypes.c_int]
    lib.sim_set_selector.argtypes = [vp, ctypes.c_int, vp]
    lib.sim_autotune.argtypes = [ctypes.c_int, ctypes.c_double, vp, ctypes.c_size_t, vp, ctypes.c_int, vp, ctypes.c_int,
                                 vp, ctypes.c_int, vp, ctypes.c_int, vp, vp, ctypes.c_size_t, vp]
    assert lib.sim_reset(None) == qcsim.ERR_INVALID
    assert lib.sim_batch_apply(None, 1, None, None, 1) == qcsim.ERR_INVALID
    assert lib.sim_set_selector(None, 2, None) == qcsim.ERR_INVALID
    g = qcsim.gates_array(circuits.rcs_n(10, 2, seed=1))
    best = qcsim.TunePoint()

    def tune(bs, cs, ls, ms, gates=g, n=10):
        arr = lambda t, v: (t * max(1, len(v)))(*v)
        return lib.sim_autotune(n, 1e-4, vp(gates.ctypes.data), gates.shape[0],
                                ctypes.cast(arr(ctypes.c_int32, bs), vp), len(bs),
                                ctypes.cast(arr(ctypes.c_int32, cs), vp), len(cs),
                                ctypes.cast(arr(ctypes.c_int32, ls), vp), len(ls),
                                ctypes.cast(arr(ctypes.c_uint32, ms), vp), len(ms), ctypes.byref(best), None, 0, None)

    assert tune([10], [12], [0], [0x1F]) == qcsim.ERR_INVALID
    assert tune([10], [8], [3], [0x1F]) == qcsim.ERR_INVALID
    assert tune([10], [8], [0], [0x0F]) == qcsim.ERR_INVALID
    assert tune([10], [8], [0], [0x80 | 0x1F]) == qcsim.ERR_INVALID
    assert tune([], [8], [0], [0x1F]) == qcsim.ERR_INVALID
    bad = g.copy()
    bad[0]["target"] = 10
    assert tune([10], [8], [0], [0x1F], gates=bad) == qcsim.ERR_INVALID
