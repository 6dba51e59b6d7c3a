"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: closed forms,
finite-difference gradients of its own energies (force = -grad V), library routines
(numpy.interp, numpy.histogram), the published Philox4x32-10 known-answer vectors, the reductions of Eq. 1 at lambda = 1
and lambda = 0, Newton's third law (which force interpolation preserves exactly),
energy conservation of velocity Verlet in the pure-AT limit, and the Langevin
equipartition / friction limits.
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_1806_10841_gb300 import inputs

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def small_system(M=27, box=(9.0, 6.5, 6.5), at=2.0, hy=1.5, seed=3, **kw):
    s = inputs.tetra_system(M, box, at, hy, seed=seed, **kw)
    x, v = inputs.tetra_state(s)
    return s, x, v


def point_system(n, box, d_at, d_hy, **kw):
    """n single-atom molecules (na = 1, no bonds)."""
    s = inputs.tetra_system(n, box, 2 * d_at, d_hy, **kw)
    s.na, s.mass, s.bonds = 1, np.ones(1), np.zeros((0, 2), np.int32)
    return s


# --- Philox4x32-10 against its published known-answer vectors ----------------------

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def kat_vectors():
    rows = []
    for line in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        w = [int(t, 16) for t in line.split()]
        rows.append((w[0:4], w[4:6], w[6:10]))
    return rows


@pytest.mark.parametrize("ctr,key,expect", kat_vectors())
def test_philox4x32_known_answers(ctr, key, expect):
    assert list(map(int, oracle.philox4x32(ctr, key))) == expect


def test_uniform3_bits_and_distribution():
    """Each component joins 32 bits of the first block and the top 21 bits of the second;
    draws are uniform on [0,1) and independent across atoms, steps and replicas."""
    seed, rep, gid, step = 0x1234567890ABCDEF, 3, 77, 2**33 + 5
    key = [seed & 0xFFFFFFFF, seed >> 32]
    hi = oracle.philox4x32([gid, step & 0xFFFFFFFF, step >> 32, 2 * rep], key)
    lo = oracle.philox4x32([gid, step & 0xFFFFFFFF, step >> 32, 2 * rep + 1], key)
    u = oracle.uniform3(seed, rep, gid, step)
    for d in range(3):
        assert u[d] == ((int(hi[d]) << 21) | (int(lo[d]) >> 11)) * 2.0 ** -53
    draws = np.array([oracle.uniform3(7, 0, g, s) for g in range(200) for s in range(20)]).ravel()
    assert draws.min() >= 0 and draws.max() < 1
    hist, _ = np.histogram(draws, bins=20, range=(0, 1))
    chi2 = ((hist - draws.size / 20) ** 2 / (draws.size / 20)).sum()
    assert chi2 < 45  # 19 degrees of freedom, p ~ 1e-3
    assert abs(np.corrcoef(draws[:-1], draws[1:])[0, 1]) < 0.05
    assert not np.array_equal(oracle.uniform3(7, 0, 5, 1), oracle.uniform3(7, 1, 5, 1))


# --- resolution function ------------------------------------------------------------

def test_weight_closed_form():
    s = point_system(2, (20, 10, 10), 2.5, 2.5)
    o = oracle.Oracle(s)
    assert o.weight(0.0) == 1.0
    assert o.weight(2.4999) == 1.0
    assert o.weight(2.5) == 1.0
    assert o.weight(5.0) == 0.0
    assert o.weight(9.0) == 0.0
    assert o.weight(3.75) == pytest.approx(0.5, abs=1e-15)
    assert o.weight(2.5 + 2.5 / 3) == pytest.approx(0.75, abs=1e-15)
    assert o.weight(2.5 + 2 * 2.5 / 3) == pytest.approx(0.25, abs=1e-15)
    # C1 at both ends: one-sided slopes vanish like O(h)
    for h in (1e-3, 1e-4):
        assert abs(o.weight(2.5 + h) - 1.0) / h < 2 * h
        assert abs(o.weight(5.0 - h)) / h < 2 * h
    # monotone non-increasing
    d = np.linspace(0, 6, 601)
    w = np.array([o.weight(t) for t in d])
    assert np.all(np.diff(w) <= 1e-15)


def test_weight_zero_hybrid_is_step():
    s = point_system(2, (20, 10, 10), 2.5, 0.0)
    o = oracle.Oracle(s)
    assert o.weight(2.4999999) == 1.0 and o.weight(2.5) == 0.0 and o.weight(7.0) == 0.0


# --- centre of mass ------------------------------------------------------------------

def test_com_straddling_boundary():
    s, x, _ = small_system(M=8, box=(10.0, 8.0, 8.0))
    L = np.array(s.box)
    # put molecule 0 astride the x = 0 face and molecule 1 astride a corner
    body = inputs.tetra_sites()
    x[0:4] = np.mod(np.array([0.05, 4.0, 4.0]) + body, L)
    x[4:8] = np.mod(np.array([9.9, 7.95, 0.02]) + body, L)
    o = oracle.Oracle(s)
    R, dxc, w = o.com_lambda(x)
    assert np.allclose(R[0], [0.05, 4.0, 4.0], atol=1e-14)
    assert np.allclose(R[1], [9.9, 7.95, 0.02], atol=1e-14)
    assert np.all((R >= 0) & (R < L))
    # signed distance to the slab centre under the minimum image
    assert dxc[0] == pytest.approx(0.05 - 5.0, abs=1e-14)
    assert dxc[1] == pytest.approx(9.9 - 5.0, abs=1e-14)


# --- pair potentials against closed forms ---------------------------------------------

def test_wca_closed_form():
    s = point_system(2, (10.0, 10.0, 10.0), 100.0, 0.0)  # all AT
    o = oracle.Oracle(s)
    for r, V, F in [(1.0, 1.0, 24.0), (2 ** (1 / 6), 0.0, 0.0), (0.9, None, None), (1.2, 0.0, 0.0)]:
        x = np.array([[3.0, 5.0, 5.0], [3.0 + r, 5.0, 5.0]])
        f, e = o.forces(x)
        if V is None:
            sr6 = (1 / r) ** 6
            V = 4 * (sr6 * sr6 - sr6) + 1
            F = 24 * (2 * sr6 * sr6 - sr6) / r
        assert e["E_at"] == pytest.approx(V, abs=1e-12)
        assert f[1, 0] == pytest.approx(F, abs=1e-12) and f[0, 0] == pytest.approx(-F, abs=1e-12)
        assert e["virial"] == pytest.approx(F * r, abs=1e-12)


def test_fene_closed_form():
    s = point_system(1, (10.0, 10.0, 10.0), 100.0, 0.0)
    s.na, s.mass, s.bonds = 2, np.ones(2), np.array([[0, 1]], np.int32)
    o = oracle.Oracle(s)
    for r in (0.97, 1.0, 1.3):
        x = np.array([[3.0, 5.0, 5.0], [3.0, 5.0 + r, 5.0]])
        f, e = o.forces(x)
        Vf = -0.5 * 30 * 1.5 ** 2 * math.log(1 - (r / 1.5) ** 2)
        Ff = -30 * r / (1 - (r / 1.5) ** 2)
        if r < 2 ** (1 / 6):
            sr6 = r ** -6
            Vf += 4 * (sr6 * sr6 - sr6) + 1
            Ff += 24 * (2 * sr6 * sr6 - sr6) / r
        assert e["E_bond"] == pytest.approx(Vf, rel=1e-13)
        assert f[1, 1] == pytest.approx(Ff, rel=1e-12) and f[0, 1] == pytest.approx(-Ff, rel=1e-12)
    with pytest.raises(RuntimeError):
        o.forces(np.array([[3.0, 5.0, 5.0], [3.0, 6.6, 5.0]]))  # beyond R0: bond broken


def test_cg_table_matches_analytic_lj_within_interpolation_bound():
    F, V = inputs.lj_cg_table()
    eps, sig, rc, dr = 1.0, 1.75, 2.3, 0.001
    s = point_system(2, (10.0, 10.0, 10.0), 0.0, 0.0)  # all CG
    o = oracle.Oracle(s)

    def Fa(r):
        s6 = (sig / r) ** 6
        return 24 * eps * (2 * s6 * s6 - s6) / r - 24 * eps * (2 * (sig / rc) ** 12 - (sig / rc) ** 6) / rc

    rng = np.random.default_rng(0)
    for r in rng.uniform(1.2, 2.299, 40):
        x = np.array([[3.0, 5.0, 5.0], [3.0 + r, 5.0, 5.0]])
        f, e = o.forces(x)
        # |F_lin - F| <= h^2/8 max|F''| on the interval
        h = dr
        rr = np.linspace(r - h, r + h, 5)
        F2 = np.abs(np.gradient(np.gradient(Fa(rr), rr), rr)).max() * 2
        assert abs(f[1, 0] - Fa(r)) <= h * h / 8 * F2 + 1e-12
        # table force is what numpy.interp gives on the same nodes
        assert f[1, 0] == pytest.approx(np.interp(r, np.arange(len(F)) * dr, F), rel=1e-13, abs=1e-13)
        assert e["E_cg"] == pytest.approx(np.interp(r, np.arange(len(V)) * dr, V), rel=1e-13, abs=1e-13)
    # beyond the cutoff: nothing
    f, e = o.forces(np.array([[3.0, 5.0, 5.0], [5.31, 5.0, 5.0]]))
    assert np.all(f == 0) and e["E_cg"] == 0


# --- finite-difference gradient of the fixed-lambda energy -------------------------------

@pytest.mark.parametrize("seed", [1, 2])
def test_forces_are_gradient_at_fixed_lambda(seed):
    """With every lambda held fixed, Eq. 1 is the gradient of
    E = sum_ab [l_a l_b V_AT + (1 - l_a l_b) V_CG] + V_bond; this pins the atom sums,
    the COM mass-fraction redistribution of F_CG, the signs and the bonded terms."""
    F, V = inputs.lj_cg_table(dr=1e-5)
    s, x, _ = small_system(M=16, box=(6.0, 5.0, 5.0), seed=seed)
    s.cg_F, s.cg_V, s.cg_dr = F, V, 1e-5
    s.mass = np.array([1.0, 2.0, 0.5, 1.5])  # unequal masses exercise m_i / M
    rng = np.random.default_rng(seed)
    wfix = rng.uniform(0, 1, s.M)
    wfix[:3] = [0.0, 1.0, 1.0]
    o = oracle.Oracle(s)
    f, _ = o.forces(x, w_override=wfix)

    def energy(xx):
        _, e = o.forces(xx, w_override=wfix)
        return e["E_at"] + e["E_cg"] + e["E_bond"]

    h = 1e-6
    idx = rng.choice(s.N, 12, replace=False)
    for i in idx:
        for d in range(3):
            xp, xm = x.copy(), x.copy()
            xp[i, d] += h
            xm[i, d] -= h
            g = -(energy(xp) - energy(xm)) / (2 * h)
            assert f[i, d] == pytest.approx(g, rel=2e-4, abs=2e-4 * (1 + np.abs(f).max() * 1e-3))


# --- reductions of Eq. 1 -----------------------------------------------------------------

def _plain_atomistic(s, x):
    """Plain WCA + FENE molecular dynamics forces (no resolution, no COMs)."""
    L = np.array(s.box)
    N = s.N
    mol = np.arange(N) // s.na
    r = x[:, None, :] - x[None, :, :]
    r -= L * np.rint(r / L)
    r2 = (r ** 2).sum(-1)
    np.fill_diagonal(r2, np.inf)
    inter = (mol[:, None] != mol[None, :]) & (r2 < s.rc_at ** 2)
    sr6 = np.where(inter, 1.0 / np.where(inter, r2, 1.0) ** 3, 0.0)
    fr = np.where(inter, 24 * (2 * sr6 ** 2 - sr6) / np.where(inter, r2, 1.0), 0.0)
    f = (fr[:, :, None] * r).sum(1)
    for a in range(s.M):
        for p, q in s.bonds:
            i, j = a * s.na + p, a * s.na + q
            rij = x[i] - x[j]
            rij -= L * np.rint(rij / L)
            rr2 = rij @ rij
            g = -s.fene_k / (1 - rr2 / s.fene_r0 ** 2)
            if rr2 < s.rc_at ** 2:
                s6 = 1 / rr2 ** 3
                g += 24 * (2 * s6 * s6 - s6) / rr2
            f[i] += g * rij
            f[j] -= g * rij
    return f


def _plain_cg(s, x):
    """Plain COM-COM tabulated model: forces on molecule centres spread by mass fraction."""
    L = np.array(s.box)
    xm = x.reshape(s.M, s.na, 3)
    un = xm[:, :1] + (xm - xm[:, :1]) - L * np.rint((xm - xm[:, :1]) / L)
    R = (s.mass[None, :, None] * un).sum(1) / s.mass.sum()
    d = R[:, None] - R[None, :]
    d -= L * np.rint(d / L)
    r = np.sqrt((d ** 2).sum(-1))
    np.fill_diagonal(r, np.inf)
    within = r < s.rc_cg
    Fm = np.where(within, np.interp(np.where(within, r, 0), np.arange(len(s.cg_F)) * s.cg_dr, s.cg_F), 0)
    FR = (np.where(within, Fm / np.where(within, r, 1), 0)[:, :, None] * d).sum(1)
    f = (s.mass[None, :, None] / s.mass.sum() * FR[:, None, :]).reshape(-1, 3)
    s2 = inputs.tetra_system(s.M, s.box, 1e6, 0.0)  # bonded part alone: an all-AT copy, no partners
    return f, R


@pytest.mark.parametrize("seed", [4, 5])
def test_lambda_one_reduces_to_plain_atomistic(seed):
    s, x, _ = small_system(M=27, box=(6.8, 6.8, 6.8), at=1e3, hy=1.0, seed=seed)
    o = oracle.Oracle(s)
    _, _, w = o.com_lambda(x)
    assert np.all(w == 1.0)
    f, e = o.forces(x)
    assert e["E_cg"] == 0.0
    ref = _plain_atomistic(s, x)
    assert np.allclose(f, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())


@pytest.mark.parametrize("seed", [6, 7])
def test_lambda_zero_reduces_to_plain_cg(seed):
    s, x, _ = small_system(M=27, box=(6.8, 6.8, 6.8), at=0.0, hy=0.0, seed=seed)
    o = oracle.Oracle(s)
    _, _, w = o.com_lambda(x)
    assert np.all(w == 0.0)
    f, e = o.forces(x)
    assert e["E_at"] == 0.0
    # remove the bonded part, which is not interpolated: evaluate it with an isolated copy
    fb = np.zeros_like(f)
    for a in range(s.M):
        sa = inputs.tetra_system(1, s.box, 0.0, 0.0)
        fa, _ = oracle.Oracle(sa).forces(x[a * 4:(a + 1) * 4])
        fb[a * 4:(a + 1) * 4] = fa
    ref, R = _plain_cg(s, x)
    R_or, _, _ = o.com_lambda(x)
    assert np.allclose(np.mod(R, s.box), R_or, atol=1e-12)
    assert np.allclose(f - fb, ref, rtol=1e-11, atol=1e-11 * np.abs(ref).max())


# --- Newton's third law and the cell scan -------------------------------------------------

@pytest.mark.parametrize("seed", [8, 9, 10])
def test_newton_third_law_in_hybrid_system(seed):
    s, x, _ = small_system(M=64, box=(14.0, 6.0, 6.0), at=3.0, hy=2.0, seed=seed)
    o = oracle.Oracle(s)
    _, _, w = o.com_lambda(x)
    assert (w == 1).any() and (w == 0).any() and ((w > 0) & (w < 1)).any()
    f, _ = o.forces(x)
    assert np.abs(f.sum(0)).max() <= 1e-12 * np.abs(f).sum()


@pytest.mark.parametrize("M,box", [(64, (14.0, 6.0, 6.0)), (27, (6.0, 5.0, 5.0)), (216, (20.0, 9.0, 9.0))])
def test_cell_scan_equals_all_pairs(M, box):
    s, x, _ = small_system(M=M, box=box, at=3.0, hy=2.0, seed=M)
    o = oracle.Oracle(s)
    f0, e0 = o.forces(x, method=0)
    f1, e1 = o.forces(x, method=1)
    assert np.allclose(f0, f1, rtol=1e-13, atol=1e-13 * np.abs(f0).max())
    for k in e0:
        assert e0[k] == pytest.approx(e1[k], rel=1e-13, abs=1e-13)


# --- thermodynamic force ------------------------------------------------------------------

def test_tf_zero_table_is_no_tf_and_constant_table_adds_known_force():
    s, x, _ = small_system(M=64, box=(14.0, 6.0, 6.0), at=3.0, hy=2.0, seed=11)
    s.mass = np.array([1.0, 2.0, 0.5, 1.5])
    o = oracle.Oracle(s)
    f0, _ = o.forces(x)
    o.set_tf(np.zeros_like(s.tf))
    fz, _ = o.forces(x)
    assert np.array_equal(f0, fz)
    c = 0.37
    o.set_tf(np.full_like(s.tf, c))
    fc, _ = o.forces(x)
    _, dxc, _ = o.com_lambda(x)
    hy = (np.abs(dxc) >= s.d_at) & (np.abs(dxc) < s.d_at + s.d_hy)
    assert hy.any()
    expect = np.zeros_like(f0)
    for a in np.nonzero(hy)[0]:
        expect[a * 4:(a + 1) * 4, 0] = c * np.sign(dxc[a]) * s.mass / s.mass.sum()
    assert np.allclose(fc - f0, expect, atol=1e-14 * np.abs(f0).max())
    # a table linear in d is reproduced exactly between nodes
    slope = 0.2
    o.set_tf(slope * np.arange(len(s.tf)) * s.tf_dx)
    fl, _ = o.forces(x)
    for a in np.nonzero(hy)[0]:
        tot = (fl - f0)[a * 4:(a + 1) * 4, 0].sum()
        assert tot == pytest.approx(slope * abs(dxc[a]) * np.sign(dxc[a]), rel=1e-12, abs=1e-14 * np.abs(f0).max())


def test_tf_update_closed_forms():
    s = inputs.tetra_system(10, (20.0, 4.0, 5.0), 4.0, 4.0)  # d_at = 2, d_hy = 4
    o = oracle.Oracle(s)
    n = len(s.tf)
    # uniform profile: no gradient, no change
    tf = o.tf_update(np.full(n, 0.3), np.full(n, 50), nsamples=5, alpha=2.0)
    assert np.array_equal(tf, np.full(n, 0.3))
    # linear profile counts_k = a + b k: interior gradient b / (vol dx) on every node
    a_, b_ = 40, 3
    counts = a_ + b_ * np.arange(n)
    ns, alpha = 4.0, 0.7
    vol = ns * 2 * s.tf_dx * 4.0 * 5.0
    tf = o.tf_update(np.zeros(n), counts, nsamples=ns, alpha=alpha)
    g = b_ / vol / s.tf_dx
    dk = np.arange(n) * s.tf_dx
    inside = (dk >= s.d_at) & (dk <= s.d_at + s.d_hy)
    interior = inside & (np.arange(n) >= 2) & (np.arange(n) <= n - 2)
    assert np.allclose(tf[interior], -alpha * g, rtol=1e-12)
    assert np.all(tf[~inside] == 0.0)


# --- density histogram against numpy.histogram ----------------------------------------------

def test_density_histogram_matches_numpy():
    s, x, _ = small_system(M=216, box=(20.0, 9.0, 9.0), seed=12)
    o = oracle.Oracle(s)
    R, dxc, _ = o.com_lambda(x)
    nd, nx = 20, 40
    cd, cx = o.density(x, nd, nx)
    ref_d, _ = np.histogram(np.abs(dxc), bins=nd, range=(0, nd * s.tf_dx))
    ref_x, _ = np.histogram(R[:, 0], bins=nx, range=(0, s.box[0]))
    assert np.array_equal(cd, ref_d) and np.array_equal(cx, ref_x)


# --- integrator ---------------------------------------------------------------------------

def _total_energy(o, x, v):
    _, e = o.forces(x)
    ke, _ = o.kinetic(v)
    return ke + e["E_at"] + e["E_cg"] + e["E_bond"]


def test_velocity_verlet_conserves_energy_pure_at_second_order():
    """lambda = 1 everywhere and no thermostat: the scheme is plain MD and velocity Verlet
    keeps the energy bounded with fluctuations that shrink like dt^2."""
    amp = {}
    for dt in (0.004, 0.002):
        s, x, v = small_system(M=64, box=(8.6, 8.6, 8.6), at=1e3, hy=1.0, seed=13, gamma=0.0, dt=dt)
        o = oracle.Oracle(s)
        f, _ = o.forces(x)
        E0 = _total_energy(o, x, v)
        Es = []
        nsteps = int(round(2.0 / dt))
        for _ in range(20):
            x, v, f = o.run(x, v, f, 0, nsteps // 20)
            Es.append(_total_energy(o, x, v))
        Es = np.array(Es)
        amp[dt] = np.abs(Es - E0).max() / s.N
    assert amp[0.002] < 1e-3
    assert 3.0 < amp[0.004] / amp[0.002] < 5.0  # 4 for a second-order integrator


def test_momentum_conserved_without_thermostat():
    s, x, v = small_system(M=72, box=(17.2, 6.45, 6.45), at=3.0, hy=2.0, seed=14, gamma=0.0)
    o = oracle.Oracle(s)
    f, _ = o.forces(x)
    _, p0 = o.kinetic(v)
    x, v, f = o.run(x, v, f, 0, 200)
    _, p1 = o.kinetic(v)
    assert np.abs(p1 - p0).max() < 1e-10


def test_langevin_free_particle_friction_and_noise_amplitude():
    # kT = 0: v decays as exp(-gamma t) up to O(dt) discretisation error
    s = point_system(1, (50.0, 50.0, 50.0), 0.0, 0.0, gamma=0.5, kT=0.0, dt=0.005)
    o = oracle.Oracle(s)
    x = np.array([[10.0, 10.0, 10.0]])
    v = np.array([[1.0, -2.0, 0.5]])
    f = np.zeros((1, 3))
    x, v2, f = o.run(x, v, f, 0, 400)
    assert np.allclose(v2, v * math.exp(-0.5 * 2.0), rtol=2e-3)
    # noise force: mean 0, variance 2 gamma kT m / dt per component
    s2 = point_system(4096, (50.0, 50.0, 50.0), 0.0, 0.0, gamma=0.5, kT=1.3, dt=0.005)
    o2 = oracle.Oracle(s2)
    fl = o2.langevin_force(np.zeros((4096, 3)), step=7)
    var = 2 * 0.5 * 1.3 * 1.0 / 0.005
    assert abs(fl.mean()) < 4 * math.sqrt(var / fl.size)
    assert fl.var() == pytest.approx(var, rel=0.05)
    assert np.abs(fl).max() <= math.sqrt(24 * 0.5 * 1.3 / 0.005) / 2
    # different steps give independent draws, same step the same draw
    assert np.array_equal(fl, o2.langevin_force(np.zeros((4096, 3)), step=7))
    assert not np.allclose(fl, o2.langevin_force(np.zeros((4096, 3)), step=8))


@pytest.mark.slow
def test_langevin_equipartition():
    s, x, v = small_system(M=27, box=(6.45, 6.45, 6.45), at=1e3, hy=1.0, seed=15, gamma=0.5, kT=1.0)
    o = oracle.Oracle(s)
    f, _ = o.forces(x)
    x, v, f = o.run(x, v, f, 0, 2000)
    kes = []
    step = 2000
    for _ in range(200):
        x, v, f = o.run(x, v, f, step, 50)
        step += 50
        kes.append(o.kinetic(v)[0])
    T = np.mean(kes) / (1.5 * s.N)
    assert T == pytest.approx(1.0, abs=0.04)
