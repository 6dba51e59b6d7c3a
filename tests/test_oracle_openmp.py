"""The all-core (OpenMP) build of the oracle, used only to time the CPU baseline, computes
the same definition as the plain serial build: forces, energies and trajectories agree to
rounding (sums in another order), the per-atom loops exactly."""
import math
import os

import numpy as np
import pytest

import oracle
from paper_1806_10841_gb300 import inputs


@pytest.fixture(scope="module")
def omp_path():
    return oracle.build(extra_flags=("-fopenmp",))


@pytest.mark.parametrize("scheme", [0, 1])
def test_openmp_build_forces_equal_serial(omp_path, scheme):
    s = inputs.tetra_system(1000, (34.20, 17.10, 17.10), 5.0, 2.5, seed=3)
    s.scheme = scheme
    x, _ = inputs.tetra_state(s)
    f1, e1 = oracle.Oracle(s).forces(x)
    f2, e2 = oracle.Oracle(s, lib_path=omp_path).forces(x)
    assert math.sqrt(((f1 - f2) ** 2).sum() / (f1 ** 2).sum()) < 1e-13
    for k in e1:
        assert e2[k] == pytest.approx(e1[k], rel=1e-12, abs=1e-12)


def test_openmp_build_trajectory_and_com_equal_serial(omp_path):
    s = inputs.tetra_system(1000, (34.20, 17.10, 17.10), 5.0, 2.5, seed=4)
    x, v = inputs.tetra_state(s)
    a, b = oracle.Oracle(s), oracle.Oracle(s, lib_path=omp_path)
    assert all(np.array_equal(p, q) for p, q in zip(a.com_lambda(x), b.com_lambda(x)))
    f0, _ = a.forces(x)
    xa, va, _ = a.run(x, v, f0, 0, 5)
    xb, vb, _ = b.run(x, v, f0, 0, 5)
    L = np.array(s.box)
    dx = xa - xb
    dx -= L * np.rint(dx / L)
    assert np.abs(dx).max() < 1e-12 and np.abs(va - vb).max() < 1e-10


def test_openmp_build_uses_several_threads(omp_path):
    import ctypes as C

    lib = C.CDLL(omp_path)
    # the build links the OpenMP runtime; the thread count follows the host (OMP_NUM_THREADS)
    n = C.CDLL(None).omp_get_max_threads() if hasattr(C.CDLL(None), "omp_get_max_threads") else \
        lib.omp_get_max_threads()
    assert n >= 1
    if (os.cpu_count() or 1) > 1 and "OMP_NUM_THREADS" not in os.environ:
        assert n > 1
