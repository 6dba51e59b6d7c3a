"""Pins of the oracle's multiple time stepping (Sec. "Multiple time stepping in adaptive
resolution simulations": impulse r-RESPA, CG forces as the slow part).

The force at time level t is F_fast + w(t) F_slow with w = n at every n-th level and 0 in
between.  Checked against: a system whose CG table and thermodynamic force are zeroed (the
fast force of force interpolation), F_fast = -grad (E_at + E_bond) and F_slow =
-grad (E_cg - sum_a DF(l_a)) by central differences with lambda following the centres of
mass (energy interpolation, where the split is a split of the Hamiltonian), bitwise
identity with plain velocity Verlet when the slow part vanishes (all-atom box), and energy
conservation of the multiple-time-step integrator to second order in the outer step.
"""
import copy

import numpy as np
import pytest

import oracle
from paper_1806_10841_gb300 import inputs

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def hybrid(scheme, n=3, M=24, box=(7.0, 5.0, 5.0), at=1.6, hy=1.8, seed=3, dr=1e-5, **kw):
    F, V = inputs.lj_cg_table(dr=dr)
    s = inputs.tetra_system(M, box, at, hy, seed=seed, **kw)
    s.cg_F, s.cg_V, s.cg_dr = F, V, dr
    s.scheme, s.respa_n = scheme, n
    x, v = inputs.tetra_state(s)
    return s, x, v


def free_energy(g, lam):
    n = len(g)
    u = np.asarray(lam) * (n - 1)
    k = np.minimum(np.floor(u).astype(int), n - 2)
    t = u - k
    cum = np.concatenate([[0.0], np.cumsum(0.5 * (g[:-1] + g[1:]))]) / (n - 1)
    gk = g[k] + (g[k + 1] - g[k]) * t
    return cum[k] + 0.5 * (g[k] + gk) * t / (n - 1)


@pytest.mark.parametrize("scheme", [0, 1])
def test_slow_weight_follows_the_time_level(scheme):
    s, x, _ = hybrid(scheme, n=3)
    s.tf = np.linspace(0.5, -0.5, len(s.tf))
    o = oracle.Oracle(s)
    f_full, e_full = o.forces(x)
    f0, e0 = o.forces(x, step=0)  # outer level: weight 3
    f1, e1 = o.forces(x, step=1)  # inner level: weight 0
    f4, _ = o.forces(x, step=4)
    assert np.array_equal(f1, f4)
    assert np.allclose(f0 - f1, 3 * (f_full - f1), rtol=1e-12, atol=1e-12 * np.abs(f_full).max())
    for k in ("E_at", "E_cg", "E_bond"):  # energies are not weighted
        assert e0[k] == e_full[k] == e1[k]


def test_fast_force_of_force_interpolation_is_the_atomistic_and_bonded_part():
    s, x, _ = hybrid(0, n=2)
    s.tf = np.linspace(1.0, -1.0, len(s.tf))
    f1, _ = oracle.Oracle(s).forces(x, step=1)
    s2 = copy.copy(s)
    s2.cg_F, s2.cg_V, s2.tf, s2.respa_n = np.zeros_like(s.cg_F), np.zeros_like(s.cg_V), np.zeros_like(s.tf), 1
    f_ref, _ = oracle.Oracle(s2).forces(x)
    assert np.array_equal(f1, f_ref)


def _fd(o, x, f, idx, pot, h=1e-6, rel=2e-4):
    fmax = np.abs(f).max()
    for i in idx:
        for d in range(3):
            xp, xm = x.copy(), x.copy()
            xp[i, d] += h
            xm[i, d] -= h
            g = -(pot(xp) - pot(xm)) / (2 * h)
            assert f[i, d] == pytest.approx(g, rel=rel, abs=rel * (1 + fmax * 1e-3)), (i, d)


@pytest.mark.parametrize("seed", [5, 6])
def test_energy_interpolation_splits_the_hamiltonian(seed):
    """H = [sum l V_AT + V_bond] + [sum (1 - l) V_CG - sum DF(l)]: the inner-level force is the
    gradient of the first bracket (with its own share of the drift force), the outer-level
    force adds n times the gradient of the second."""
    n = 4
    # a fine CG table: F is interpolated linearly, and so is V, whose slope then differs from
    # -F by O(dr |F'|); at 1e-6 that stays below the difference quotient's tolerance
    s, x, _ = hybrid(1, n=n, seed=seed, dr=1e-6)
    s.mass = np.array([1.0, 2.0, 0.5, 1.5])
    s.fec = np.random.default_rng(seed).uniform(-20, 20, 7)
    o = oracle.Oracle(s)
    _, _, w = o.com_lambda(x)
    hyb = np.flatnonzero((w > 0.02) & (w < 0.98))
    assert len(hyb) >= 3
    rng = np.random.default_rng(seed)
    idx = np.concatenate([4 * hyb[:4] + rng.integers(0, 4, min(4, len(hyb))), rng.choice(s.N, 3, replace=False)])
    f_in, _ = o.forces(x, step=1)
    f_out, _ = o.forces(x, step=4)

    def fast(xx):
        _, e = o.forces(xx, step=1)
        return e["E_at"] + e["E_bond"]

    def slow(xx):
        _, e = o.forces(xx, step=1)
        _, _, ww = o.com_lambda(xx)
        return e["E_cg"] - free_energy(s.fec, ww).sum()

    _fd(o, x, f_in, idx, fast)
    _fd(o, x, (f_out - f_in) / n, idx, slow)


def test_all_atomistic_box_is_plain_velocity_verlet():
    s, x, v = hybrid(0, n=3, M=27, box=(6.8, 6.8, 6.8), at=1e3, hy=1.0, seed=9)
    o = oracle.Oracle(s)
    f, _ = o.forces(x, step=0)
    xr, vr, _ = o.run(x, v, f, 0, 20)
    s1 = copy.copy(s)
    s1.respa_n = 1
    o1 = oracle.Oracle(s1)
    f1, _ = o1.forces(x)
    xp, vp, _ = o1.run(x, v, f1, 0, 20)
    assert np.array_equal(xr, xp) and np.array_equal(vr, vp)


def _nve_error(n, dt_outer, T=2.4, chunks=24):
    s, x, v = hybrid(1, n=n, M=64, box=(12.9, 7.0, 7.0), at=2.0, hy=2.0, seed=13, gamma=0.0, dt=dt_outer / n)
    o = oracle.Oracle(s)
    f, _ = o.forces(x, step=0)

    def total(xx, vv):
        _, e = o.forces(xx)
        return 0.5 * (vv ** 2).sum() + e["E_at"] + e["E_cg"] + e["E_bond"]

    E0 = total(x, v)
    Es = []
    per = int(round(T / dt_outer)) // chunks * n  # inner steps per chunk, whole outer steps
    step = 0
    for _ in range(chunks):
        x, v, f = o.run(x, v, f, step, per)
        step += per
        Es.append(total(x, v))
    return np.abs(np.array(Es) - E0).max() / s.N


def test_multiple_time_stepping_conserves_the_hamiltonian_to_second_order():
    """Energy interpolation, no thermostat: impulse r-RESPA with n = 3 inner steps keeps H with
    an error shrinking like the outer step squared."""
    a1 = _nve_error(3, 0.003)
    a2 = _nve_error(3, 0.0015)
    assert a2 < 2e-3
    assert 3.0 < a1 / a2 < 5.0
