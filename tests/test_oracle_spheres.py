"""Pins of the oracle's self-adjusting geometry (AT region = union of spheres around
resolution centres; Sec. "Self-adjusting adaptive resolution simulations").

Checked against: the squared-cosine closed form of the distance to a single centre across a
periodic face, lambda of a union equal to the largest single-centre lambda (numpy),
the thermodynamic force along the direction from the nearest centre (difference of two
force evaluations against numpy), and a density proportional to the shell volumes giving
no thermodynamic-force update.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1806_10841_gb300 import inputs


def point_system(n, box, d_at, d_hy, centers, **kw):
    s = inputs.tetra_system(n, box, 2 * d_at, d_hy, **kw)
    s.na, s.mass, s.bonds = 1, np.ones(1), np.zeros((0, 2), np.int32)
    s.centers = None if centers is None else np.asarray(centers, dtype=np.float64)
    return s


def w_closed(d, d_at, d_hy):
    if d < d_at:
        return 1.0
    if d >= d_at + d_hy:
        return 0.0
    return math.cos(0.5 * math.pi * (d - d_at) / d_hy) ** 2


def test_lambda_of_one_centre_across_the_periodic_face():
    L = (20.0, 16.0, 12.0)
    c = np.array([[0.5, 15.8, 6.0]])  # close to two faces
    s = point_system(200, L, 3.0, 2.0, c)
    rng = np.random.default_rng(1)
    x = rng.uniform(0, 1, (200, 3)) * np.array(L)
    R, d, w = oracle.Oracle(s).com_lambda(x)
    dd = x - c[0]
    dd -= np.array(L) * np.rint(dd / np.array(L))
    dist = np.sqrt((dd ** 2).sum(1))
    assert np.allclose(d, dist, rtol=1e-14, atol=1e-14)
    assert np.allclose(w, [w_closed(v, 3.0, 2.0) for v in dist], rtol=1e-13, atol=1e-15)
    assert (w == 1).any() and ((w > 0) & (w < 1)).any() and (w == 0).any()


def test_lambda_of_a_union_is_the_largest_single_centre_lambda():
    L = (30.0, 30.0, 30.0)
    rng = np.random.default_rng(2)
    c = rng.uniform(0, 30, (5, 3))
    s = point_system(500, L, 2.5, 3.0, c)
    x = rng.uniform(0, 30, (500, 3))
    _, d, w = oracle.Oracle(s).com_lambda(x)
    per = []
    for k in range(len(c)):
        dd = x - c[k]
        dd -= np.array(L) * np.rint(dd / np.array(L))
        per.append(np.sqrt((dd ** 2).sum(1)))
    per = np.array(per)
    assert np.allclose(d, per.min(0), rtol=1e-14)
    wmax = np.array([max(w_closed(per[k, a], 2.5, 3.0) for k in range(len(c))) for a in range(500)])
    assert np.allclose(w, wmax, rtol=1e-13, atol=1e-15)


def test_thermodynamic_force_points_away_from_the_nearest_centre():
    L = (40.0, 40.0, 40.0)
    c = np.array([[10.0, 10.0, 10.0], [30.0, 30.0, 30.0]])
    s = inputs.tetra_system(512, L, 6.0, 4.0, tf_bins=20)
    s.centers = c
    x, _ = inputs.tetra_state(s)
    o = oracle.Oracle(s)
    f0, _ = o.forces(x)
    tf = np.full(len(s.tf), 0.7)
    o.set_tf(tf)
    f1, _ = o.forces(x)
    R, d, _ = o.com_lambda(x)
    df = (f1 - f0).reshape(s.M, 4, 3)
    hy = (d >= s.d_at) & (d < s.d_at + s.d_hy)
    assert hy.any() and (~hy).any()
    for a in range(s.M):
        if not hy[a]:
            assert np.abs(df[a]).max() == 0.0
            continue
        dd = R[a] - c
        dd -= np.array(L) * np.rint(dd / np.array(L))
        k = int(np.argmin((dd ** 2).sum(1)))
        u = dd[k] / np.linalg.norm(dd[k])
        assert np.allclose(df[a], 0.25 * 0.7 * u[None, :], rtol=1e-12, atol=1e-14)


def test_density_proportional_to_shell_volumes_needs_no_update():
    s = point_system(10, (50.0, 50.0, 50.0), 4.0, 3.0, [[10.0, 10.0, 10.0], [35.0, 35.0, 35.0]],
                     tf_bins=20)
    o = oracle.Oracle(s)
    k = np.arange(len(s.tf))
    counts = 7 * ((k + 1) ** 3 - k ** 3)
    tf0 = 0.1 * np.sin(k)
    # flat up to the rounding of the shell volumes (a wrong normalisation moves it by ~1e-2)
    assert np.allclose(o.tf_update(tf0, counts, nsamples=3, alpha=5.0), tf0, rtol=0, atol=1e-13)
    # a slab-normalised profile would not be flat
    s2 = point_system(10, (50.0, 50.0, 50.0), 4.0, 3.0, None, tf_bins=20)
    assert not np.allclose(oracle.Oracle(s2).tf_update(tf0, counts, nsamples=3, alpha=5.0), tf0, rtol=0, atol=1e-6)
