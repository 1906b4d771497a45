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
