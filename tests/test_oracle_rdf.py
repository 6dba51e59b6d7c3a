"""Pins of the oracle's COM pair-distance histogram (radial distribution function).

Checked against: numpy pair distances of centres of mass computed here from the atoms,
exact neighbour-shell counts of a simple cubic lattice, and g(r) = 1 for an ideal gas
(which also pins the normalisation the binding applies).
"""
import numpy as np
import pytest

import oracle
from paper_1806_10841_gb300 import inputs
from paper_1806_10841_gb300.adress import AdResS


def point_system(n, box):
    s = inputs.tetra_system(n, box, 0.0, 0.0)
    s.na, s.mass, s.bonds = 1, np.ones(1), np.zeros((0, 2), np.int32)
    return s


def test_rdf_counts_equal_numpy_pair_distances_of_molecule_centres():
    s = inputs.tetra_system(300, (20.0, 12.0, 12.5), 4.0, 2.0, seed=8)
    x, _ = inputs.tetra_state(s)
    L = np.array(s.box)
    xm = x.reshape(s.M, 4, 3)
    rel = xm - xm[:, :1]
    rel -= L * np.rint(rel / L)
    R = np.mod(xm[:, 0] + rel.mean(1), L)  # unit masses
    iu = np.triu_indices(s.M, 1)
    d = R[iu[0]] - R[iu[1]]
    d -= L * np.rint(d / L)
    r = np.sqrt((d ** 2).sum(1))
    nb, dr = 250, 0.02
    ref, _ = np.histogram(r, bins=nb, range=(0.0, nb * dr))
    got = oracle.Oracle(s).rdf_counts(x, nb, dr)
    assert np.array_equal(got, ref)
    assert got.sum() == int((r < nb * dr).sum())


def test_rdf_of_a_simple_cubic_lattice_counts_its_neighbour_shells():
    n, a = 8, 1.5
    s = point_system(n ** 3, (n * a,) * 3)
    g = np.stack(np.meshgrid(*[np.arange(n)] * 3, indexing="ij"), -1).reshape(-1, 3)
    x = (g + 0.25) * a
    dr = 0.01
    c = oracle.Oracle(s).rdf_counts(x, 500, dr)
    M = n ** 3
    # shells at a (6 neighbours), a sqrt2 (12), a sqrt3 (8), 2a (6): pairs = M * z / 2
    for dist, z in ((a, 6), (a * 2 ** 0.5, 12), (a * 3 ** 0.5, 8), (2 * a, 6)):
        k = int(np.floor(dist / dr + 1e-9))
        assert c[k - 1:k + 2].sum() == M * z // 2, dist
    assert c[: int(a / dr) - 1].sum() == 0


def test_ideal_gas_rdf_is_one():
    rng = np.random.default_rng(4)
    M, Lb = 3000, 24.0
    s = point_system(M, (Lb, Lb, Lb))
    x = rng.uniform(0, Lb, (M, 3))
    nb, dr = 50, 0.2
    c = oracle.Oracle(s).rdf_counts(x, nb, dr)
    g = AdResS.rdf_normalise(c, M, Lb ** 3, dr)
    # bins from r = 2 on hold >= ~1000 pairs each: 10% per bin, 2% on the mean
    assert np.all(np.abs(g[10:] - 1.0) < 0.12)
    assert abs(g[10:].mean() - 1.0) < 0.02
