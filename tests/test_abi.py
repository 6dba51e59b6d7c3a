"""The C-ABI library loads and exports every entry point include/adress.h declares
(no GPU needed: only symbol lookup), and the binding's signature table matches it."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    txt = open(os.path.join(ROOT, "include", "adress.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(adress_[a-z_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    from paper_1806_10841_gb300 import build

    build.build()
    return ctypes.CDLL(build.LIB)


def test_header_declares_the_core_calls():
    names = declared_functions()
    for core in ("adress_init", "adress_build_lists", "adress_compute_forces", "adress_step"):
        assert core in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_covers_every_declared_symbol():
    from paper_1806_10841_gb300 import adress

    assert sorted(adress.EXPORTS) == declared_functions()


def test_status_strings_without_gpu(lib):
    lib.adress_status_string.restype = ctypes.c_char_p
    assert lib.adress_status_string(0) == b"ok"
    assert b"overflow" in lib.adress_status_string(3)


def test_init_rejects_bad_config_without_touching_the_gpu(lib):
    from paper_1806_10841_gb300 import adress

    L = adress.load_library()
    cfg = adress.adress_config(n_mols=1, atoms_per_mol=4)
    h = ctypes.c_void_p()
    assert L.adress_init(ctypes.byref(cfg), None, ctypes.byref(h)) == 1
    assert b"n_mols" in L.adress_last_error(None)
    assert not h.value


def test_batch_init_rejects_replicas_that_differ_in_shared_parameters(lib):
    """Replicas of a batch may differ in size, box, slab and replica id only; validation
    happens on the host before any device call."""
    from paper_1806_10841_gb300 import adress, inputs

    L = adress.load_library()
    keep = []
    a = inputs.tetra_system(216, (25.8, 12.9, 6.45), 5.0, 2.5, tf_bins=20)
    b = inputs.tetra_system(300, (30.0, 15.0, 15.0), 3.0, 1.0, tf_bins=20)
    bad = inputs.tetra_system(300, (30.0, 15.0, 15.0), 3.0, 1.0, tf_bins=20, gamma=1.0)
    h = ctypes.c_void_p()
    cfgs = (adress.adress_config * 2)(adress._config(a, keep, 0, 0, "fp32"), adress._config(bad, keep, 1, 0, "fp32"))
    assert L.adress_init_batch(cfgs, 2, None, ctypes.byref(h)) == 1
    assert b"replica 1" in L.adress_last_error(None) and b"thermostat" in L.adress_last_error(None)
    assert not h.value
    c = inputs.tetra_system(300, (30.0, 15.0, 15.0), 3.0, 1.0, tf_bins=21)
    cfgs = (adress.adress_config * 2)(adress._config(a, keep, 0, 0, "fp32"), adress._config(c, keep, 1, 0, "fp32"))
    assert L.adress_init_batch(cfgs, 2, None, ctypes.byref(h)) == 1
    assert b"thermodynamic-force grid" in L.adress_last_error(None)
    cfgs = (adress.adress_config * 2)(adress._config(a, keep, 0, 0, "fp32"), adress._config(b, keep, 1, 0, "fp32"))
    assert L.adress_init_batch(cfgs, 0, None, ctypes.byref(h)) == 1
    small = inputs.tetra_system(8, (4.0, 4.0, 4.0), 1.0, 1.0, tf_bins=20)
    cfgs = (adress.adress_config * 2)(adress._config(a, keep, 0, 0, "fp32"), adress._config(small, keep, 1, 0, "fp32"))
    assert L.adress_init_batch(cfgs, 2, None, ctypes.byref(h)) == 1 and not h.value
    assert b"replica 1: box edge shorter" in L.adress_last_error(None)


def test_oracle_and_cuda_path_share_no_code():
    """Neither side imports or includes the other (only the input generator is shared)."""
    pkg = os.path.join(ROOT, "paper_1806_10841_gb300")
    for dirpath, _, files in os.walk(pkg):
        for fn in files:
            if fn.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, fn)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, fn
                assert "adress_oracle" not in txt, fn
    for fn in os.listdir(os.path.join(ROOT, "oracle")):
        if fn.endswith((".py", ".c", ".h")):
            txt = open(os.path.join(ROOT, "oracle", fn)).read()
            assert "paper_1806_10841_gb300" not in txt, fn
            assert "adress.h" not in txt, fn


def test_init_rejects_bad_coupling_scheme_without_touching_the_gpu(lib):
    """Energy interpolation's switches are validated on the host: the scheme number, a
    free-energy correction without scheme 1 or with a single node, and replicas of a batch
    that disagree on the scheme."""
    import numpy as np

    from paper_1806_10841_gb300 import adress, inputs

    L = adress.load_library()
    keep = []
    h = ctypes.c_void_p()
    s = inputs.tetra_system(216, (25.8, 12.9, 6.45), 5.0, 2.5, tf_bins=20)
    for scheme, fec, msg in ((2, None, b"scheme must be"), (0, np.zeros(5), b"needs scheme 1"),
                             (1, np.zeros(1), b"fec_n must be"), (1, np.array([0.0, np.nan]), b"finite")):
        s.scheme, s.fec = scheme, fec
        cfg = adress._config(s, keep, 0, 0, "fp32")
        assert L.adress_init(ctypes.byref(cfg), None, ctypes.byref(h)) == 1
        assert msg in L.adress_last_error(None), msg
        assert not h.value
    a = inputs.tetra_system(216, (25.8, 12.9, 6.45), 5.0, 2.5, tf_bins=20)
    b = inputs.tetra_system(300, (30.0, 15.0, 15.0), 3.0, 1.0, tf_bins=20)
    b.scheme = 1
    cfgs = (adress.adress_config * 2)(adress._config(a, keep, 0, 0, "fp32"), adress._config(b, keep, 1, 0, "fp32"))
    assert L.adress_init_batch(cfgs, 2, None, ctypes.byref(h)) == 1
    assert b"coupling scheme" in L.adress_last_error(None)


def test_init_rejects_bad_multiple_time_stepping(lib):
    from paper_1806_10841_gb300 import adress, inputs

    L = adress.load_library()
    keep = []
    h = ctypes.c_void_p()
    s = inputs.tetra_system(216, (25.8, 12.9, 6.45), 5.0, 2.5, tf_bins=20)
    for n in (-1, 65):
        s.respa_n = n
        cfg = adress._config(s, keep, 0, 0, "fp32")
        assert L.adress_init(ctypes.byref(cfg), None, ctypes.byref(h)) == 1
        assert b"respa_n" in L.adress_last_error(None)
    a = inputs.tetra_system(216, (25.8, 12.9, 6.45), 5.0, 2.5, tf_bins=20)
    b = inputs.tetra_system(300, (30.0, 15.0, 15.0), 3.0, 1.0, tf_bins=20)
    b.respa_n = 2
    cfgs = (adress.adress_config * 2)(adress._config(a, keep, 0, 0, "fp32"), adress._config(b, keep, 1, 0, "fp32"))
    assert L.adress_init_batch(cfgs, 2, None, ctypes.byref(h)) == 1
    assert b"multiple time stepping" in L.adress_last_error(None)


def test_binding_fails_loudly_without_the_library():
    """No fallback: without the built CUDA library the binding raises (fresh interpreter)."""
    import subprocess
    import sys

    code = ("import sys; sys.path.insert(0, %r)\n"
            "from paper_1806_10841_gb300 import adress\n"
            "try:\n"
            "    adress.load_library('/nonexistent/libadress_gb300.so')\n"
            "except RuntimeError as e:\n"
            "    print('raised:', e)\n" % ROOT)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and "raised:" in r.stdout and "missing" in r.stdout, r.stdout + r.stderr
