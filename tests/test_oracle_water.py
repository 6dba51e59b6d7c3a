"""Pins of the oracle's water-like model (flexible three-site molecules, Lennard-Jones on O,
reaction-field Coulomb, harmonic bonds and angle).

Checked against: the reaction-field and Lennard-Jones closed forms for an isolated pair,
an independent numpy implementation of the all-atomistic model (lambda = 1), F = -grad E
by central differences at fixed lambda (which also pins the angle and bond terms), zero
bonded force at the equilibrium geometry, and Newton's third law in a hybrid system.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1806_10841_gb300 import inputs


def small_water(M=64, at=1.2, hy=0.6, seed=3, distort=0.0):
    Ly = (M / 33.4 / 2.0) ** (1.0 / 3.0)
    # boxes at least twice the list cutoff in every direction: use a cube for small M
    L = max(2.7, Ly)
    s = inputs.water_system(M, (2 * L, L, L), at, hy, seed=seed)
    x, v = inputs.water_state(s)
    if distort:
        x = x + np.random.default_rng(seed).normal(0, distort, x.shape)
    return s, x, v


def two_point_charges(q1, q2, r, eps_o=0.0):
    """Two one-site molecules at distance r along x (all atomistic)."""
    s = inputs.water_system(2, (6.0, 6.0, 6.0), 1e3, 1.0)
    s.na, s.mass, s.bonds, s.angles = 1, np.ones(1), np.zeros((0, 2), np.int32), None
    s.charge = np.array([q1])
    s.lj_eps, s.lj_sig = np.array([eps_o]), np.array([0.3166])
    x = np.array([[3.0, 3.0, 3.0], [3.0 + r, 3.0, 3.0]])
    return s, x


def test_reaction_field_pair_closed_form():
    rc, erf, f = 0.9, 80.0, inputs.COULOMB_F
    krf = (erf - 1) / ((2 * erf + 1) * rc ** 3)
    crf = 1 / rc + krf * rc ** 2
    for r in (0.25, 0.5, 0.89):
        s, x = two_point_charges(0.4238, 0.4238, r)
        # both sites carry the same charge (one site type)
        fo, e = oracle.Oracle(s).forces(x)
        qq = f * 0.4238 ** 2
        assert e["E_at"] == pytest.approx(qq * (1 / r + krf * r * r - crf), rel=1e-12)
        assert fo[1, 0] == pytest.approx(qq * (1 / r ** 2 - 2 * krf * r), rel=1e-12)
        assert fo[0, 0] == pytest.approx(-fo[1, 0], rel=1e-14)
    s, x = two_point_charges(0.4238, 0.4238, 0.95)
    fo, e = oracle.Oracle(s).forces(x)
    assert e["E_at"] == 0.0 and not fo.any()


def test_lennard_jones_pair_is_shifted_to_zero_at_the_cutoff():
    eps, sg, rc = 0.65, 0.3166, 0.9
    for r in (0.3, 0.35, 0.6):
        s, x = two_point_charges(0.0, 0.0, r, eps_o=eps)
        fo, e = oracle.Oracle(s).forces(x)
        V = lambda y: 4 * eps * ((sg / y) ** 12 - (sg / y) ** 6)
        assert e["E_at"] == pytest.approx(V(r) - V(rc), rel=1e-12)
        F = 24 * eps * (2 * (sg / r) ** 12 - (sg / r) ** 6) / r
        assert fo[1, 0] == pytest.approx(F, rel=1e-12)


def _plain_water(s, x):
    """Independent all-atomistic water forces and energy: every intermolecular atom pair within
    rc (LJ O-O shifted, reaction field), harmonic O-H bonds, harmonic H-O-H angle."""
    L = np.array(s.box)
    N = s.N
    mol = np.arange(N) // 3
    site = np.arange(N) % 3
    r = x[:, None, :] - x[None, :, :]
    r -= L * np.rint(r / L)
    r2 = (r ** 2).sum(-1)
    inter = (mol[:, None] != mol[None, :]) & (r2 < s.rc_at ** 2)
    rr = np.sqrt(np.where(inter, r2, 1.0))
    q = s.charge[site]
    qq = s.coulomb_f * q[:, None] * q[None, :]
    krf = (s.eps_rf - 1) / ((2 * s.eps_rf + 1) * s.rc_at ** 3)
    crf = 1 / s.rc_at + krf * s.rc_at ** 2
    oo = (site[:, None] == 0) & (site[None, :] == 0)
    eps, sg = s.lj_eps[0], s.lj_sig[0]
    sr6 = (sg / rr) ** 6
    sc6 = (sg / s.rc_at) ** 6
    fr = np.where(inter, qq * (1 / rr ** 3 - 2 * krf), 0.0)
    fr += np.where(inter & oo, 24 * eps * (2 * sr6 ** 2 - sr6) / rr ** 2, 0.0)
    E = 0.5 * np.where(inter, qq * (1 / rr + krf * rr ** 2 - crf), 0.0).sum()
    E += 0.5 * np.where(inter & oo, 4 * eps * (sr6 ** 2 - sr6) - 4 * eps * (sc6 ** 2 - sc6), 0.0).sum()
    f = (fr[:, :, None] * r).sum(1)
    for a in range(s.M):
        o, h1, h2 = 3 * a, 3 * a + 1, 3 * a + 2
        for h in (h1, h2):
            d = x[h] - x[o]
            d -= L * np.rint(d / L)
            dl = np.linalg.norm(d)
            g = -s.bond_k * (dl - s.bond_r0) / dl
            f[h] += g * d
            f[o] -= g * d
            E += 0.5 * s.bond_k * (dl - s.bond_r0) ** 2
        u = x[h1] - x[o]
        w = x[h2] - x[o]
        u -= L * np.rint(u / L)
        w -= L * np.rint(w / L)
        nu, nw = np.linalg.norm(u), np.linalg.norm(w)
        c = u @ w / (nu * nw)
        th = math.acos(c)
        E += 0.5 * s.angle_k * (th - s.angle_theta0) ** 2
        dV = s.angle_k * (th - s.angle_theta0)
        # dtheta/du = -(w/(|u||w|) - c u/|u|^2) / sin(theta)
        du = -(w / (nu * nw) - c * u / nu ** 2) / math.sin(th)
        dw = -(u / (nu * nw) - c * w / nw ** 2) / math.sin(th)
        f[h1] -= dV * du
        f[h2] -= dV * dw
        f[o] += dV * (du + dw)
    return f, E


@pytest.mark.parametrize("seed", [1, 2])
def test_all_atomistic_water_equals_plain_code(seed):
    s, x, _ = small_water(M=48, at=1e3, hy=1.0, seed=seed, distort=0.004)
    o = oracle.Oracle(s)
    _, _, w = o.com_lambda(x)
    assert np.all(w == 1.0)
    f, e = o.forces(x)
    ref, E = _plain_water(s, x)
    assert e["E_cg"] == 0.0
    assert np.allclose(f, ref, rtol=1e-10, atol=1e-10 * np.abs(ref).max())
    assert e["E_at"] + e["E_bond"] == pytest.approx(E, rel=1e-10)


@pytest.mark.parametrize("seed", [3, 4])
def test_water_forces_are_gradient_at_fixed_lambda(seed):
    s, x, _ = small_water(M=24, seed=seed, distort=0.005)
    F, V = inputs.lj_cg_table(0.65, 0.3166, s.rc_cg, 1e-6, r_min=0.2)
    s.cg_F, s.cg_V, s.cg_dr = F, V, 1e-6
    rng = np.random.default_rng(seed)
    wfix = rng.uniform(0, 1, s.M)
    wfix[:3] = [0.0, 1.0, 1.0]
    o = oracle.Oracle(s)
    f, _ = o.forces(x, w_override=wfix)

    def energy(xx):
        _, e = o.forces(xx, w_override=wfix)
        return e["E_at"] + e["E_cg"] + e["E_bond"]

    h = 1e-7
    for i in rng.choice(s.N, 12, replace=False):
        for d in range(3):
            xp, xm = x.copy(), x.copy()
            xp[i, d] += h
            xm[i, d] -= h
            g = -(energy(xp) - energy(xm)) / (2 * h)
            assert f[i, d] == pytest.approx(g, rel=1e-4, abs=1e-4 * (1 + np.abs(f).max() * 1e-3)), (i, d)


def test_equilibrium_geometry_has_no_bonded_force():
    s = inputs.water_system(1, (6.0, 6.0, 6.0), 1e3, 1.0)
    x = inputs.water_sites() + 3.0
    f, e = oracle.Oracle(s).forces(x)
    assert e["E_bond"] == pytest.approx(0.0, abs=1e-20)
    assert np.abs(f).max() < 1e-9


def test_newton_third_law_in_hybrid_water():
    s, x, _ = small_water(M=64, at=1.0, hy=0.8, seed=5, distort=0.003)
    o = oracle.Oracle(s)
    _, _, w = o.com_lambda(x)
    assert 0 < (w == 1).sum() < s.M and ((w > 0) & (w < 1)).any()
    f, _ = o.forces(x)
    assert np.abs(f.sum(0)).max() <= 1e-10 * np.abs(f).sum()
