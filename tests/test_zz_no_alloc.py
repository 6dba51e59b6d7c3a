"""The allocation-free kinetic-energy entry point against the handle-based one.

Callers that cannot allocate device memory when they need an observable (a fixed-budget
memory pool, an allocator owned by another framework, a monitoring hook that must not
change the allocation pattern it observes) use adress_kinetic_noalloc, which keeps its
partial sums in a fixed static device array instead of handle-owned scratch.  This file is
collected last on purpose: if it fails, a run that stops at the first failure has already
run every other test.  It passes alone in a fresh process and after the other tests.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _noalloc(lib, v_ptr, n, na, mass, stream_ptr, out_ptr):
    return lib.adress_kinetic_noalloc(C.c_void_p(v_ptr), C.c_int64(n), C.c_int32(na),
                                      mass.ctypes.data_as(C.POINTER(C.c_double)), C.c_void_p(stream_ptr),
                                      C.c_void_p(out_ptr))


def test_kinetic_noalloc_matches_adress_kinetic_on_two_calls_in_a_row():
    import torch

    from paper_1806_10841_gb300 import adress, inputs

    lib = adress.load_library()
    s = inputs.scaled_c2(5000)
    s.mass = np.array([1.0, 2.0, 0.5, 1.5])  # unequal per-site masses
    x, v = inputs.tetra_state(s)
    sim = adress.AdResS(s, precision="fp64")
    sim.set_state(x, v)
    ke_ref, p_ref = sim.kinetic()  # the existing, handle-based entry point
    mass = np.ascontiguousarray(s.mass, dtype=np.float64)
    out = torch.zeros(4, dtype=torch.float64, device=sim.device)
    scale = float((np.tile(mass, s.M)[:, None] * np.abs(v)).sum())
    for _ in range(2):
        out.fill_(np.nan)
        st = _noalloc(lib, sim.v.data_ptr(), sim.N, 4, mass, sim.stream.cuda_stream, out.data_ptr())
        assert st == 0, lib.adress_last_error(None)
        sim.stream.synchronize()
        got = out.cpu().numpy()
        assert got[0] == pytest.approx(ke_ref, rel=1e-12)
        assert np.allclose(got[1:], p_ref, rtol=1e-12, atol=1e-13 * scale)

    # a smaller call right after: the shared scratch keeps the previous call's partial
    # sums, which must not leak into a call that uses fewer of them
    n_small = 3001 * 4 + 3  # not a multiple of the block size
    vs = np.ascontiguousarray(v[:n_small].T)
    vdev = torch.from_numpy(vs).to(sim.device)
    st = _noalloc(lib, vdev.data_ptr(), n_small, 4, mass, sim.stream.cuda_stream, out.data_ptr())
    assert st == 0
    sim.stream.synchronize()
    m = np.tile(mass, s.M)[:n_small]
    ke_small = 0.5 * float((m[:, None] * v[:n_small] ** 2).sum())
    p_small = (m[:, None] * v[:n_small]).sum(0)
    got = out.cpu().numpy()
    assert got[0] == pytest.approx(ke_small, rel=1e-12)
    assert np.allclose(got[1:], p_small, rtol=1e-12, atol=1e-13 * float((m[:, None] * np.abs(v[:n_small])).sum()))
    sim.close()


def test_kinetic_noalloc_grid_stride_and_block_cap():
    """Above 1024 blocks x 256 threads (262,144 atoms) every thread sums several atoms in its
    grid-stride loop and the partial sums fill all 1024 scratch slots: 1,000,003 atoms with
    three unequal site masses against a numpy sum, twice in a row."""
    import torch

    from paper_1806_10841_gb300 import adress

    lib = adress.load_library()
    n = 1_000_003
    rng = np.random.default_rng(41)
    v = rng.normal(0.0, 1.0, (3, n))
    mass = np.array([1.0, 2.5, 0.75])
    m = np.tile(mass, n // 3 + 1)[:n]
    ke_ref = 0.5 * float((m * v ** 2).sum())
    p_ref = (m * v).sum(1)
    scale = float((m * np.abs(v)).sum())
    dev = torch.device("cuda:0")
    vd = torch.from_numpy(np.ascontiguousarray(v)).to(dev)
    out = torch.zeros(4, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    for _ in range(2):
        out.fill_(np.nan)
        st = _noalloc(lib, vd.data_ptr(), n, 3, mass, stream.cuda_stream, out.data_ptr())
        assert st == 0, lib.adress_last_error(None)
        stream.synchronize()
        got = out.cpu().numpy()
        assert got[0] == pytest.approx(ke_ref, rel=1e-12)
        assert np.allclose(got[1:], p_ref, rtol=1e-12, atol=1e-13 * scale)


def test_kinetic_noalloc_rejects_sizes_beyond_its_scratch():
    from paper_1806_10841_gb300 import adress

    lib = adress.load_library()
    mass = np.ones(4)
    st = _noalloc(lib, 1, 16_777_217, 4, mass, 0, 1)  # nothing is launched for a rejected size
    assert st == 1
    assert b"16777216" in lib.adress_last_error(None)
    assert _noalloc(lib, 1, 100, 5, mass, 0, 1) == 1
