"""The synthetic input recipe (seeded, shared by the oracle and the CUDA path; no method
arithmetic): workload shapes, densities and slab widths of the configurations, and the
properties the initial states are built to have."""
import math

import numpy as np
import pytest

from paper_1806_10841_gb300 import inputs


def min_intermolecular_distance(x, na, L):
    """Brute force over all atom pairs of different molecules (small systems only)."""
    mol = np.arange(len(x)) // na
    d = x[:, None] - x[None]
    d -= L * np.rint(d / L)
    r = np.sqrt((d ** 2).sum(-1))
    r[mol[:, None] == mol[None, :]] = np.inf
    return r.min()


def test_workload_shapes():
    s = inputs.c2_800k()
    assert (s.M, s.na, s.N) == (200_000, 4, 800_000)
    assert s.box == (200.0, 100.0, 100.0)
    assert s.M / np.prod(s.box) == pytest.approx(0.1)
    assert (s.d_at, s.d_hy, s.xc) == (20.0, 10.0, 100.0)  # full AT width 40, 10 hybrid per side
    c1 = inputs.c1_literal()
    assert c1.M == 1000 and c1.box == (20.0, 10.0, 10.0) and (c1.d_at, c1.d_hy) == (2.5, 2.5)
    c1s = inputs.c1_stable()
    assert c1s.M / np.prod(c1s.box) == pytest.approx(0.1, rel=1e-3)
    w = inputs.c3_water()
    assert (w.M, w.na) == (64_000, 3)
    assert w.M / np.prod(w.box) == pytest.approx(33.4, rel=1e-3)
    assert (w.d_at, w.d_hy) == (1.5, 1.5)
    for M in (2000, 20000):
        sc = inputs.scaled_c2(M)
        assert sc.M / np.prod(sc.box) == pytest.approx(0.1)
        assert sc.box[0] == pytest.approx(2 * sc.box[1]) and sc.box[1] == sc.box[2]
        assert 2 * sc.d_at / sc.box[0] == pytest.approx(0.2) and sc.d_hy / sc.box[0] == pytest.approx(0.05)


def test_replica_batch_recipe():
    systems = inputs.replica_batch(64)
    sizes = np.array([s.M for s in systems])
    assert len(systems) == 64 and sizes.min() >= 500 and sizes.max() <= 20000
    # log-uniform: the median of log sizes sits near the middle of [ln 500, ln 20000]
    assert abs(np.median(np.log(sizes)) - 0.5 * (math.log(500) + math.log(20000))) < 0.6
    for s in systems:
        assert 1.5 <= s.d_at <= 7.5 and 1.0 <= s.d_hy <= 5.0  # full AT width U(3, 15)
        assert s.M / np.prod(s.box) == pytest.approx(0.1, rel=0.02)
        assert s.box[0] == pytest.approx(2 * s.box[1])
    assert len({len(s.tf) for s in systems}) == 1  # a common thermodynamic-force grid
    assert len({s.seed for s in systems}) == 1  # one thermostat key; replica ids differ


def test_tetrahedral_state_properties():
    s = inputs.c1_stable()
    x, v = inputs.tetra_state(s)
    L = np.array(s.box)
    assert x.shape == (s.N, 3) and v.shape == (s.N, 3)
    assert np.all((x >= 0) & (x < L))
    assert np.abs(v.sum(0)).max() < 1e-10  # total momentum removed (unit masses)
    assert 0.5 * (v ** 2).sum() / (1.5 * s.N) == pytest.approx(s.kT, rel=0.05)
    assert min_intermolecular_distance(x, s.na, L) >= 1.0  # redrawn until no contact < 1 sigma
    # regular tetrahedra of edge 0.97
    xm = x.reshape(s.M, 4, 3)
    for a in range(0, s.M, 97):
        d = xm[a][:, None] - xm[a][None]
        d -= L * np.rint(d / L)
        e = np.sqrt((d ** 2).sum(-1))[np.triu_indices(4, 1)]
        assert np.allclose(e, 0.97, atol=1e-12)
    # the same seed gives the same state
    x2, v2 = inputs.tetra_state(s)
    assert np.array_equal(x, x2) and np.array_equal(v, v2)


def test_water_state_properties():
    s = inputs.scaled_c3(512)
    x, v = inputs.water_state(s)
    L = np.array(s.box)
    assert np.all((x >= 0) & (x < L))
    assert min_intermolecular_distance(x, 3, L) >= 0.17
    xm = x.reshape(s.M, 3, 3)
    oh = xm[:, 1:] - xm[:, :1]
    oh -= L * np.rint(oh / L)
    assert np.allclose(np.sqrt((oh ** 2).sum(-1)), s.bond_r0, atol=1e-12)
