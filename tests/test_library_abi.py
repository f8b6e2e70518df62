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
    assert ctypes.sizeof(binding.Stats) == 16 * 8
    assert binding.MLP_PARAMS == 21377
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


def test_batch_item_layout_and_host_validation():
    """dmrgc_batch_run validates every item on the host before any CUDA call."""
    from paper_2207_05612_gb300 import binding
    from synthetic import circuits as sc
    assert ctypes.sizeof(binding.BatchItem) == 80
    lib = binding.lib()
    wall = ctypes.c_double(-1.0)
    opt = binding.dmrgc_default_options()
    assert lib.dmrgc_batch_run(None, 0, 1, ctypes.byref(opt), None, ctypes.byref(wall)) == 0
    assert wall.value == 0.0
    circ = sc.random_circuit(2, 3, 2, seed=0)
    items, keep = binding.pack_batch([(2, 3, 4, circ.layers, 2), (2, 3, 4, circ.layers, 2)])
    bad = [
        ("n_workers", lambda it: None, 0),
        ("chi", lambda it: setattr(it, "chi", 0), 1),
        ("grid", lambda it: setattr(it, "grid_view", binding.Grid(3, 2, 0)), 1),
        ("order", lambda it: setattr(it, "grid_view", binding.Grid(2, 3, 3)), 1),
        ("sweeps", lambda it: setattr(it, "n_sweeps", -1), 1),
        ("gates", lambda it: setattr(it, "gates", None), 1),
    ]
    for name, mutate, workers in bad:
        items, keep = binding.pack_batch([(2, 3, 4, circ.layers, 2), (2, 3, 4, circ.layers, 2)])
        mutate(items[1])
        st = lib.dmrgc_batch_run(items, 2, workers, ctypes.byref(opt), None, ctypes.byref(wall))
        assert st == binding.DMRGC_EINVAL, name
        assert items[0].status == -1        # nothing ran, outputs untouched
    opt.precision = 7
    items, keep = binding.pack_batch([(2, 3, 4, circ.layers, 2)])
    assert lib.dmrgc_batch_run(items, 1, 1, ctypes.byref(opt), None, ctypes.byref(wall)) == binding.DMRGC_EINVAL
    opt.precision = 0
    opt.svd_mode = 2   # the learned mode without a rank model
    assert lib.dmrgc_batch_run(items, 1, 1, ctypes.byref(opt), None, ctypes.byref(wall)) == binding.DMRGC_EINVAL


def test_grouped_create_validates_on_the_host():
    """dmrgc_create_grouped rejects group sizes that do not tile the qubits, or
    a grid order it does not know, before any CUDA call."""
    import numpy as np
    from paper_2207_05612_gb300 import binding
    lib = binding.lib()
    opt = binding.dmrgc_default_options()
    h = ctypes.c_void_p()
    for rows, cols, order, sizes in ((3, 4, 0, [3, 3, 3]), (3, 4, 0, [12, 0]), (3, 4, 0, [21, -9]),
                                     (3, 4, 3, [6, 6]), (3, 4, 0, [])):
        gs = np.ascontiguousarray(sizes or [1], dtype=np.int32)
        g = binding.Grid(rows, cols, order)
        st = lib.dmrgc_create_grouped(rows * cols, ctypes.byref(g), gs.ctypes.data, len(sizes), 8,
                                      ctypes.byref(opt), ctypes.byref(h))
        assert st == binding.DMRGC_EINVAL, (order, sizes)
        assert not h.value


@pytest.mark.parametrize("lang,std", [("c", "-std=c99"), ("c++", "-std=c++17")])
def test_header_is_plain_c(lang, std):
    """include/dmrgc.h compiles on its own as strict C99 and as C++ (plain
    types and pointers only, nothing from CUDA or torch); the source is fed on
    stdin, so nothing is written."""
    import shutil
    import subprocess
    cc = shutil.which("gcc" if lang == "c" else "g++")
    if cc is None:
        pytest.skip("no host compiler")
    src = ('#include "dmrgc.h"\n'
           "int main(void) { dmrgc_options o; dmrgc_status s = dmrgc_default_options(&o);"
           " return (int)s + o.precision; }\n")
    r = subprocess.run([cc, "-x", lang, std, "-Wall", "-Wextra", "-pedantic", "-Werror", "-fsyntax-only",
                        "-I", os.path.join(ROOT, "include"), "-"], input=src, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_entry_points_reject_a_null_context():
    """The public calls return DMRGC_EINVAL for a NULL context before any CUDA
    call (their NVTX ranges open and close without a profiler attached)."""
    from paper_2207_05612_gb300 import binding
    lib = binding.lib()
    einval = binding.DMRGC_EINVAL
    assert lib.dmrgc_apply_layer(None, None, 0) == einval
    assert lib.dmrgc_sweep(None, 1, None) == einval
    assert lib.dmrgc_sweep_updates(None, 1, None) == einval
    assert lib.dmrgc_amplitude(None, None, 0, None) == einval
    assert lib.dmrgc_sample(None, 0, 0, None) == einval
    assert lib.dmrgc_metropolis(None, 1, 1, 0, None, None) == einval
    assert lib.dmrgc_overlap(None, None, None) == einval
    assert lib.dmrgc_fidelity(None, None, None) == einval
    assert lib.dmrgc_last_error(None) == b"null context"
    lib.dmrgc_destroy(None)
