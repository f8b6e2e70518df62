"""CPU checks of the C-ABI library: it loads and exports every symbol that
include/dmrgc.h declares (no compute call is made without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "dmrgc.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(dmrgc_[a-z_0-9]+)\s*\(", txt)))


def test_header_declares_the_boundary():
    names = _declared()
    for want in ("dmrgc_create", "dmrgc_apply_layer", "dmrgc_sweep", "dmrgc_fidelity",
                 "dmrgc_amplitude", "dmrgc_sample", "dmrgc_destroy", "dmrgc_last_error"):
        assert want in names


def test_library_exports_every_declared_symbol():
    from paper_2207_05612_gb300 import binding
    lib = binding.lib()
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_struct_layouts_match_header():
    from paper_2207_05612_gb300 import binding
    assert ctypes.sizeof(binding.Gate) == 8 + 32 * 8
    assert ctypes.sizeof(binding.Stats) == 11 * 8
    o = binding.dmrgc_default_options()      # host-only entry point
    assert o.precision == binding.DMRGC_FP64 and o.max_jacobi_sweeps == 40


def test_pack_gates_roundtrip():
    import numpy as np
    from paper_2207_05612_gb300 import binding
    from synthetic import circuits as sc
    u = sc.fsim(0.3, 0.2)
    arr = binding.pack_gates([(3, 5, u), (1, -1, sc.sqrt_pauli("Y"))])
    m = np.array(arr[0].mat[:])
    assert np.allclose(m[0::2] + 1j * m[1::2], u.reshape(-1))
    assert arr[1].q1 == -1
