"""Pins of the oracle's force-matched CG table (oracle.force_matched_table): the per-bin mean
of the atomistic pair force projected on the COM axis, interpolated between bin centres,
shifted to vanish at the cutoff, integrated to a potential."""
import math

import numpy as np
import pytest

import oracle
from paper_1806_10841_gb300 import inputs


def lj(r, eps=1.0, sig=1.75):
    """Lennard-Jones force F = -dV/dr, its two derivatives and V."""
    sr6 = (sig / r) ** 6
    V = 4 * eps * (sr6 * sr6 - sr6)
    F = 24 * eps * (2 * sr6 * sr6 - sr6) / r
    F1 = -24 * eps * (26 * sr6 * sr6 - 7 * sr6) / r ** 2
    F2 = 24 * eps * (26 * 14 * sr6 * sr6 - 7 * 8 * sr6) / r ** 3
    return F, F1, F2, V


def test_samples_at_bin_centres_give_the_interpolant_of_the_force():
    """Targets equal to an analytic force at the bin centres: every bin mean is that value,
    so the table is the linear interpolant of F through the centres, shifted by F(rc), within
    the interpolation bound h^2/8 max|F''| of the analytic shifted force; V the shifted
    potential V(r) - V(rc) - (rc - r) F(rc) within the trapezoid and interpolation bounds.
    (Bin edges taken for centres would be off by h/2 |F'|, far beyond the bound.)"""
    h, dr, rc = 0.02, 0.001, 2.3
    cg_n = int(round(rc / dr))
    j = np.arange(int(math.ceil(1.6 / h)), int(math.ceil(rc / h)))
    c = (j + 0.5) * h
    d = np.repeat(c, 3)
    t = np.repeat(lj(c)[0], 3)
    F, V = oracle.force_matched_table(d, t, h, 1, dr, cg_n, rc)
    r = np.arange(cg_n + 1) * dr
    inside = (r >= c[0]) & (r <= c[-1])
    Fa, _, F2, Va = lj(np.maximum(r, 1e-3))
    Frc, _, _, Vrc = lj(rc)
    # the interpolant of the samples at rc is the last centre's value (rc beyond it)
    f_rc = lj(c[-1])[0]
    bound = h * h / 8 * np.abs(lj(np.linspace(c[0], c[-1], 20001))[2]).max()
    assert np.abs(F[inside] - (Fa[inside] - f_rc)).max() <= bound * 1.0001
    assert F[-1] == 0.0
    # below the first centre: the first mean, shifted
    below = r < c[0]
    assert np.allclose(F[below], lj(c[0])[0] - f_rc, rtol=0, atol=1e-12)
    # V(r) = int_r^rc F: the centres are table nodes, so the trapezoid rule is exact on the
    # piecewise-linear table and V differs from the analytic integral of the shifted force by
    # at most the interpolation bound times the length
    k0 = int(np.nonzero(inside)[0][0])
    k1 = int(np.nonzero(inside)[0][-1])
    Va_shift = (Va[k0] - Va[k1]) - (r[k1] - r[k0]) * f_rc
    assert V[k0] - V[k1] == pytest.approx(Va_shift, abs=(r[k1] - r[k0]) * bound * 1.0001 + 1e-12)
    assert V[-1] == 0.0


def test_point_particle_fluid_reproduces_the_pair_force():
    """One atom per molecule: the atomistic interaction (WCA) is central between the centres
    of mass, so every sample's projected force is the WCA force at its distance and the
    table reproduces it within the bin width times its slope."""
    s = inputs.tetra_system(400, (20.0, 10.0, 10.0), 1e3, 1.0, seed=10)
    s.na, s.mass, s.bonds = 1, np.ones(1), np.zeros((0, 2), np.int32)
    rng = np.random.default_rng(12)
    x = rng.uniform(0, 1, (s.M, 3)) * np.array(s.box)
    feat, t, _ = oracle.Oracle(s).collect_pairs(x, 1.12)
    d = feat[:, 0]
    # targets are the WCA force magnitude (positive = repulsive)
    sr6 = (1.0 / d) ** 6
    assert np.allclose(t, 24 * (2 * sr6 * sr6 - sr6) / d, rtol=1e-12)
    h, dr, rc = 0.01, 0.001, 2.3
    F, _ = oracle.force_matched_table(d, t, h, 1, dr, int(round(rc / dr)), rc)
    r = np.arange(len(F)) * dr
    pop = np.unique(np.floor(d / h).astype(int))
    # at the centre of a populated bin whose neighbours are populated too, the table is the
    # bin mean: within h/2 max|F'| over the bin of the WCA force there
    for j in pop[1:-1]:
        if j - 1 not in pop or j + 1 not in pop:
            continue
        k = int(round((j + 0.5) * h / dr))
        rr = k * dr
        sr6 = (1.0 / rr) ** 6
        Fw = 24 * (2 * sr6 * sr6 - sr6) / rr
        dF = 24 * (26 * sr6 * sr6 - 7 * sr6) / (rr - h) ** 2
        assert abs(F[k] - Fw) <= 0.5 * h * dF + 1e-9, (j, F[k], Fw)


def test_table_invariances():
    rng = np.random.default_rng(3)
    d = rng.uniform(0.9, 2.3, 20000)
    t = 3.0 - 1.5 * d + rng.normal(0, 0.5, d.size)
    h, dr, rc = 0.05, 0.001, 2.3
    n = int(round(rc / dr))
    F, V = oracle.force_matched_table(d, t, h, 5, dr, n, rc)
    p = rng.permutation(d.size)
    F2, V2 = oracle.force_matched_table(d[p], t[p], h, 5, dr, n, rc)
    assert np.allclose(F, F2, rtol=0, atol=1e-12) and np.allclose(V, V2, rtol=0, atol=1e-12)
    # a constant force is removed by the shift; a linear one stays linear
    Fc, Vc = oracle.force_matched_table(d, np.full(d.size, 2.5), h, 5, dr, n, rc)
    assert np.abs(Fc).max() < 1e-12 and np.abs(Vc).max() < 1e-12
    Fl, _ = oracle.force_matched_table(d, 3.0 - 1.5 * d, h, 1, dr, n, rc)
    r = np.arange(n + 1) * dr
    mid = (r > 1.0) & (r < 2.2)
    # bin means of a linear function over uniform samples are the line at the mean d of the
    # bin's samples, within h/2 of the centre: slope error below 1.5 (h/2) / h per unit r
    assert np.allclose(np.diff(Fl[mid]) / dr, -1.5, atol=0.2)
    with pytest.raises(ValueError):
        oracle.force_matched_table(d, t, h, 10 ** 9, dr, n, rc)
