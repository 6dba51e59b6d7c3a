"""Pins of the oracle's energy-interpolation scheme (H-AdResS, Eq. Hmix).

The scheme has a Hamiltonian, H = K + sum_a [l_a V_AT_a + (1 - l_a) V_CG_a] + V_bond, with
V_AT_a and V_CG_a half of molecule a's pair energies.  Checked against: that potential
written out in numpy for one-site molecules (the per-molecule sums, independent of the
oracle's pair weighting), F = -grad H by central differences with lambda following the
centres of mass (which pins the drift force, its sign, its COM mass-fraction spread and its
direction in the slab and in the sphere geometry), F = -grad E at fixed lambda with pair
weight (l_a + l_b)/2, energy conservation of velocity Verlet to second order in a hybrid
system without thermostat, the reductions at lambda = 1 and lambda = 0 where the two
schemes coincide, and, for the free-energy correction, F = -grad (V - sum_a DF(l_a)) with
DF integrated in numpy from the tabulated dDF/dl.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1806_10841_gb300 import inputs

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def hybrid_system(M=24, box=(7.0, 5.0, 5.0), at=1.6, hy=1.8, seed=3, **kw):
    F, V = inputs.lj_cg_table(dr=1e-5)
    s = inputs.tetra_system(M, box, at, hy, seed=seed, **kw)
    s.cg_F, s.cg_V, s.cg_dr = F, V, 1e-5
    s.scheme = 1
    x, v = inputs.tetra_state(s)
    return s, x, v


def potential(o, x, w_override=None):
    _, e = o.forces(x, w_override=w_override)
    return e["E_at"] + e["E_cg"] + e["E_bond"]


def fd_check(o, x, f, idx, h, rel, w_override=None):
    fmax = np.abs(f).max()
    for i in idx:
        for d in range(3):
            xp, xm = x.copy(), x.copy()
            xp[i, d] += h
            xm[i, d] -= h
            g = -(potential(o, xp, w_override) - potential(o, xm, w_override)) / (2 * h)
            assert f[i, d] == pytest.approx(g, rel=rel, abs=rel * (1 + fmax * 1e-3)), (i, d)


def test_one_site_potential_equals_per_molecule_sums():
    """One-site molecules: atoms are the centres, so H's potential is written out directly
    as sum_a l_a V_AT_a + (1 - l_a) V_CG_a with the WCA pair and the tabulated CG pair."""
    rng = np.random.default_rng(11)
    M, L = 90, np.array([12.0, 6.0, 6.0])
    s = inputs.tetra_system(M, tuple(L), 3.0, 2.0)
    s.na, s.mass, s.bonds = 1, np.ones(1), np.zeros((0, 2), np.int32)
    s.scheme = 1
    # spread points on a jittered lattice so that no pair sits deep in the WCA core
    g = np.stack(np.meshgrid(np.arange(9), np.arange(5), np.arange(2), indexing="ij"), -1).reshape(-1, 3)
    x = (g + 0.5) * np.array([12 / 9, 6 / 5, 3.0]) + rng.uniform(-0.15, 0.15, (M, 3))
    x = np.mod(x, L)
    d = np.abs(x[:, 0] - 0.5 * L[0])
    lam = np.where(d < s.d_at, 1.0, np.where(d >= s.d_at + s.d_hy, 0.0,
                   np.cos(0.5 * math.pi * (d - s.d_at) / s.d_hy) ** 2))
    assert ((lam > 0) & (lam < 1)).sum() > 10
    r = x[:, None] - x[None]
    r -= L * np.rint(r / L)
    r = np.sqrt((r ** 2).sum(-1))
    np.fill_diagonal(r, np.inf)
    rc = 2 ** (1 / 6)
    vat = np.where(r < rc, 4 * (r ** -12.0 - r ** -6.0) + 1.0, 0.0)
    grid = np.arange(len(s.cg_V)) * s.cg_dr
    vcg = np.where(r < s.rc_cg, np.interp(np.minimum(r, s.rc_cg), grid, s.cg_V), 0.0)
    Vat, Vcg = 0.5 * vat.sum(1), 0.5 * vcg.sum(1)
    _, e = oracle.Oracle(s).forces(x)
    assert e["E_at"] == pytest.approx((lam * Vat).sum(), rel=1e-12, abs=1e-12)
    # the oracle interpolates the CG table linearly in the force and integrates it for V:
    # compare with the table's own V within its interpolation error
    assert e["E_cg"] == pytest.approx(((1 - lam) * Vcg).sum(), rel=1e-6, abs=1e-8)


@pytest.mark.parametrize("seed", [1, 2])
def test_forces_are_gradient_at_fixed_lambda_with_mean_pair_weight(seed):
    s, x, _ = hybrid_system(seed=seed)
    s.mass = np.array([1.0, 2.0, 0.5, 1.5])
    rng = np.random.default_rng(seed)
    wfix = rng.uniform(0, 1, s.M)
    wfix[:3] = [0.0, 1.0, 0.0]
    o = oracle.Oracle(s)
    f, _ = o.forces(x, w_override=wfix)
    fd_check(o, x, f, rng.choice(s.N, 12, replace=False), 1e-6, 2e-4, w_override=wfix)
    # the pair weight differs from force interpolation's l_a l_b
    s0, _, _ = hybrid_system(seed=seed)
    s0.mass, s0.scheme = s.mass, 0
    f0, _ = oracle.Oracle(s0).forces(x, w_override=wfix)
    assert np.abs(f - f0).max() > 1e-3 * np.abs(f).max()


@pytest.mark.parametrize("seed", [4, 5, 6])
def test_forces_are_gradient_of_the_hamiltonian_slab(seed):
    """lambda follows the centres of mass: the drift force -(V_AT_a - V_CG_a) grad l_a
    closes the gap between the pair forces and -grad H."""
    s, x, _ = hybrid_system(seed=seed)
    s.mass = np.array([1.0, 2.0, 0.5, 1.5])
    o = oracle.Oracle(s)
    R, _, w = o.com_lambda(x)
    hyb = np.flatnonzero((w > 0.02) & (w < 0.98))
    assert len(hyb) >= 3
    f, _ = o.forces(x)
    # without the drift force the same check fails: the fixed-lambda forces differ
    f_fix, _ = o.forces(x, w_override=w)
    assert np.abs(f - f_fix).max() > 1e-3 * np.abs(f).max()
    rng = np.random.default_rng(seed)
    idx = np.concatenate([4 * hyb[:4] + rng.integers(0, 4, min(4, len(hyb))), rng.choice(s.N, 4, replace=False)])
    fd_check(o, x, f, idx, 1e-6, 2e-4)


@pytest.mark.parametrize("seed", [7, 8])
def test_forces_are_gradient_of_the_hamiltonian_spheres(seed):
    """Resolution centres (one of them near a periodic face): the drift force points along
    the direction from the nearest centre."""
    s, x, _ = hybrid_system(M=40, box=(7.0, 7.0, 6.0), at=1.2, hy=1.5, seed=seed)
    s.centers = np.array([[2.0, 2.5, 3.0], [6.6, 5.0, 0.3]])
    o = oracle.Oracle(s)
    _, _, w = o.com_lambda(x)
    hyb = np.flatnonzero((w > 0.02) & (w < 0.98))
    assert len(hyb) >= 3
    f, _ = o.forces(x)
    rng = np.random.default_rng(seed)
    idx = 4 * hyb[:6] + rng.integers(0, 4, min(6, len(hyb)))
    fd_check(o, x, f, idx, 1e-6, 2e-4)


def _total(o, x, v, s):
    return 0.5 * (np.repeat(s.mass[None, :], s.M, 0).reshape(-1, 1) * v ** 2).sum() + potential(o, x)


def _nve_error(scheme, dt, T=3.2, chunks=32):
    s, x, v = hybrid_system(M=64, box=(12.9, 7.0, 7.0), at=2.0, hy=2.0, seed=13, gamma=0.0, dt=dt)
    s.scheme = scheme
    o = oracle.Oracle(s)
    _, _, w0 = o.com_lambda(x)
    f, _ = o.forces(x)
    E0 = _total(o, x, v, s)
    Es = []
    for _ in range(chunks):
        x, v, f = o.run(x, v, f, 0, int(round(T / dt)) // chunks)
        Es.append(_total(o, x, v, s))
    _, _, w1 = o.com_lambda(x)
    return np.abs(np.array(Es) - E0).max() / s.N, int((np.abs(w1 - w0) > 0.05).sum())


def test_velocity_verlet_conserves_the_hamiltonian_in_a_hybrid_system():
    """No thermostat, no thermodynamic force: H is conserved with an error that shrinks like
    dt^2 while molecules cross the hybrid layer; force interpolation, which has no
    Hamiltonian, keeps an error that does not shrink with dt."""
    amp1, crossed = _nve_error(1, 0.001)
    amp2, _ = _nve_error(1, 0.0005)
    assert crossed >= 5
    assert amp2 < 1e-3
    assert 3.0 < amp1 / amp2 < 5.0  # 4 for a second-order integrator
    amp_fi, _ = _nve_error(0, 0.0005)
    assert amp_fi > 10 * amp2


@pytest.mark.parametrize("at,hy", [(1e3, 1.0), (0.0, 0.0)])
def test_schemes_coincide_at_full_and_zero_resolution(at, hy):
    s, x, _ = hybrid_system(M=27, box=(6.8, 6.8, 6.8), at=at, hy=hy, seed=9)
    f1, e1 = oracle.Oracle(s).forces(x)
    s.scheme = 0
    f0, e0 = oracle.Oracle(s).forces(x)
    assert np.array_equal(f1, f0)
    for k in ("E_at", "E_cg", "E_bond"):
        assert e1[k] == e0[k]


def free_energy(g, lam):
    """DF(l) = int_0^l g for g linear between equidistant nodes on [0, 1] (exact)."""
    n = len(g)
    u = np.asarray(lam) * (n - 1)
    k = np.minimum(np.floor(u).astype(int), n - 2)
    t = u - k
    cum = np.concatenate([[0.0], np.cumsum(0.5 * (g[:-1] + g[1:]))]) / (n - 1)
    gk = g[k] + (g[k + 1] - g[k]) * t
    return cum[k] + 0.5 * (g[k] + gk) * t / (n - 1)


def test_free_energy_integral_helper():
    g = np.array([1.0, 3.0, -2.0, 0.5])
    assert free_energy(g, 0.0) == 0.0
    assert free_energy(g, 1.0) == pytest.approx((0.5 * (1 + 3) + 0.5 * (3 - 2) + 0.5 * (-2 + 0.5)) / 3)
    lam = np.linspace(0, 1, 3001)
    gl = np.interp(lam, np.linspace(0, 1, 4), g)
    num = np.concatenate([[0.0], np.cumsum(0.5 * (gl[1:] + gl[:-1]) * np.diff(lam))])
    assert np.allclose(free_energy(g, lam), num, atol=1e-12)


@pytest.mark.parametrize("seed,centers", [(21, None), (22, [[2.0, 2.5, 3.0], [6.6, 5.0, 0.3]])])
def test_free_energy_correction_is_gradient_of_its_potential(seed, centers):
    """With a tabulated dDF/dl the forces are -grad (V - sum_a DF(l_a)): the correction adds
    +g(l_a) grad l_a to the drift force, in the slab and the sphere geometry."""
    if centers is None:
        s, x, _ = hybrid_system(seed=seed)
    else:
        s, x, _ = hybrid_system(M=40, box=(7.0, 7.0, 6.0), at=1.2, hy=1.5, seed=seed)
        s.centers = np.array(centers)
    rng = np.random.default_rng(seed)
    s.fec = rng.uniform(-20, 20, 9)
    o = oracle.Oracle(s)
    _, _, w = o.com_lambda(x)
    hyb = np.flatnonzero((w > 0.02) & (w < 0.98))
    assert len(hyb) >= 3
    f, _ = o.forces(x)
    f_nofec, _ = oracle.Oracle(_without_fec(s)).forces(x)
    assert np.abs(f - f_nofec).max() > 1e-2

    def pot(xx):
        _, _, ww = o.com_lambda(xx)
        return potential(o, xx) - free_energy(s.fec, ww).sum()

    fmax = np.abs(f).max()
    for i in 4 * hyb[:6] + rng.integers(0, 4, min(6, len(hyb))):
        for d in range(3):
            xp, xm = x.copy(), x.copy()
            xp[i, d] += 1e-6
            xm[i, d] -= 1e-6
            gnum = -(pot(xp) - pot(xm)) / 2e-6
            assert f[i, d] == pytest.approx(gnum, rel=2e-4, abs=2e-4 * (1 + fmax * 1e-3)), (i, d)


def _without_fec(s):
    import copy

    s2 = copy.copy(s)
    s2.fec = None
    return s2


# --- uniform lambda and Kirkwood thermodynamic integration --------------------------------

def one_site_fluid(M=125, L=6.0, seed=4, cg_scale=1.0, **kw):
    """One-site molecules on a jittered lattice; the CG table is cg_scale x WCA (the force-
    shifted LJ at its minimum is WCA), so AT and CG differ by a known factor."""
    rc = 2 ** (1 / 6)
    n = 112246
    F, V = inputs.lj_cg_table(1.0, 1.0, rc, rc / n, r_min=0.5)
    s = inputs.tetra_system(M, (L, L, L), 2.0, 1.0, rc_cg=rc, cg_dr=rc / n, seed=seed, **kw)
    s.na, s.mass, s.bonds = 1, np.ones(1), np.zeros((0, 2), np.int32)
    s.cg_F, s.cg_V = cg_scale * F, cg_scale * V
    s.scheme = 1
    k = round(M ** (1 / 3))
    g = np.stack(np.meshgrid(*[np.arange(k)] * 3, indexing="ij"), -1).reshape(-1, 3)
    rng = np.random.default_rng(seed)
    x = np.mod((g + 0.5) * (L / k) + rng.uniform(-0.12, 0.12, (M, 3)), L)
    v = rng.normal(0, 1, (M, 3))
    v -= v.mean(0)
    return s, x, v


def _wca_all_pairs(x, L):
    r = x[:, None] - x[None]
    r -= L * np.rint(r / L)
    r2 = (r ** 2).sum(-1)
    np.fill_diagonal(r2, np.inf)
    inside = r2 < 2 ** (1 / 3)
    ir6 = np.where(inside, 1 / np.where(inside, r2, 1) ** 3, 0)
    V = 0.5 * np.where(inside, 4 * (ir6 ** 2 - ir6) + 1, 0).sum()
    F = (np.where(inside, 24 * (2 * ir6 ** 2 - ir6) / np.where(inside, r2, 1), 0)[:, :, None] * r).sum(1)
    return F, V


@pytest.mark.parametrize("lam", [0.2, 0.5, 0.9])
def test_uniform_lambda_mixes_the_two_models_linearly(lam):
    """Every molecule at l = lam: H's potential is lam V_AT + (1 - lam) V_CG and the force
    the same mix of the plain all-atom and all-CG forces (numpy, WCA and 0.5 x WCA), with
    no thermodynamic force, drift force or correction although all three are configured."""
    s, x, _ = one_site_fluid(cg_scale=0.5)
    s.tf = np.full(8, 3.0)
    s.fec = np.linspace(-5, 5, 6)
    o = oracle.Oracle(s)
    o.set_uniform_lambda(lam)
    _, _, w = o.com_lambda(x)
    assert np.all(w == lam)
    f, e = o.forces(x)
    F, V = _wca_all_pairs(x, np.array(s.box))
    assert e["E_at"] == pytest.approx(lam * V, rel=1e-12)
    assert e["E_cg"] == pytest.approx((1 - lam) * 0.5 * V, rel=1e-8)
    assert np.allclose(f, (lam + 0.5 * (1 - lam)) * F, rtol=1e-8, atol=1e-8 * np.abs(F).max())
    # dH/dl at fixed configuration = V_AT - V_CG
    assert e["E_at"] / lam - e["E_cg"] / (1 - lam) == pytest.approx(0.5 * V, rel=1e-8)


def test_kirkwood_integrand_vanishes_for_identical_models():
    """AT and CG the same potential: dH/dl = V_AT - V_CG = 0 at every l and every sampled
    configuration (up to the CG table's interpolation error)."""
    s, x, v = one_site_fluid(cg_scale=1.0, gamma=1.0, dt=0.002)
    o = oracle.Oracle(s)
    g, x1, v1, step = o.kirkwood(x, v, [0.25, 0.5, 0.75], n_equil=20, n_samples=4, every=10)
    assert step == 3 * (20 + 40)
    _, V = _wca_all_pairs(x1, np.array(s.box))
    assert np.abs(g).max() < 1e-8 * (1 + V / s.M)
    assert np.abs(x1 - x).max() > 1e-3  # the configurations moved


def test_kirkwood_integrand_for_half_strength_cg_model():
    """CG = 0.5 x AT: the integrand is half the AT energy per molecule of the sampled
    configurations, and the dynamics at l samples the potential ((1 + l)/2) V_WCA."""
    s, x, v = one_site_fluid(cg_scale=0.5, gamma=1.0, dt=0.002)
    o = oracle.Oracle(s)
    g, x1, _, _ = o.kirkwood(x, v, [0.6], n_equil=0, n_samples=1, every=15)
    _, V = _wca_all_pairs(x1, np.array(s.box))
    assert g[0] == pytest.approx(0.5 * V / s.M, rel=1e-8)
