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
