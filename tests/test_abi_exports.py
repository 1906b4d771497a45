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
