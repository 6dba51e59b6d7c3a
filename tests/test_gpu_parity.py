"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances: per-atom force relative RMS  sqrt(sum|F - F_ref|^2 / sum|F_ref|^2)
<= 1e-10 for the FP64 path and <= 2e-5 for the FP32 mixed path; next to it a per-atom
bound max_i |F_i - F_ref_i| / (|F_ref_i| + rms|F_ref|) (each atom's error relative to its
own force, with the RMS force as the floor for atoms whose contributions cancel) of
MAXTOL; integer outputs (density histogram) bit-exact.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1806_10841_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "fp32": 2e-5}
ETOL = {"fp64": 1e-10, "fp32": 2e-5}
MAXTOL = {"fp64": 1e-12, "fp32": 5e-5}  # measured on GB300: <= 7.3e-14 and <= 6.4e-6 (800k atoms)


def rel_rms(a, b):
    return math.sqrt(((a - b) ** 2).sum() / (b ** 2).sum())


def per_atom_max(a, b):
    """max_i |a_i - b_i| / (|b_i| + rms|b|) over atoms (rows of (N, 3) arrays)."""
    d = np.linalg.norm(a - b, axis=1)
    n = np.linalg.norm(b, axis=1)
    return float((d / (n + math.sqrt((n ** 2).mean()))).max())


def make(name):
    if name == "c1_literal":
        s = inputs.c1_literal()
        x, v = inputs.tetra_state(s, min_contact=0.0)
    elif name == "c1_stable":
        s = inputs.c1_stable()
        x, v = inputs.tetra_state(s)
    elif name == "hybrid_216":
        s = inputs.tetra_system(216, (25.8, 12.9, 6.45), 5.0, 2.5, seed=5)
        x, v = inputs.tetra_state(s)
    elif name == "scaled_20k":
        s = inputs.scaled_c2(20_000)
        x, v = inputs.tetra_state(s)
    elif name == "c2_800k":
        s = inputs.c2_800k()
        x, v = inputs.tetra_state(s)
    else:
        raise KeyError(name)
    return s, x, v


_cache = {}


def case(name):
    if name not in _cache:
        s, x, v = make(name)
        f, e = oracle.Oracle(s).forces(x)
        _cache[name] = (s, x, v, f, e)
    return _cache[name]


def gpu(s, precision, **kw):
    from paper_1806_10841_gb300 import adress

    return adress.AdResS(s, precision=precision, **kw)


def check_forces(s, x, f_ref, e_ref, precision):
    sim = gpu(s, precision)
    sim.set_state(x)
    f, e = sim.forces()
    sim.check()
    r = rel_rms(f, f_ref)
    m = per_atom_max(f, f_ref)
    print(f"PARITY {precision} N={len(f)} rms={r:.3e} max={m:.3e}")
    assert r <= TOL[precision], f"{precision}: force rel RMS {r:.3e}"
    assert m <= MAXTOL[precision], f"{precision}: per-atom max {m:.3e}"
    scale = abs(e_ref["E_at"]) + abs(e_ref["E_cg"]) + abs(e_ref["E_bond"])
    for k in ("E_at", "E_cg", "E_bond"):
        assert abs(e[k] - e_ref[k]) <= ETOL[precision] * scale, (k, e[k], e_ref[k])
    assert abs(e["virial"] - e_ref["virial"]) <= ETOL[precision] * (abs(e_ref["virial"]) + scale)
    sim.close()
    return r


# ---- step-0 forces ---------------------------------------------------------------------

@pytest.mark.parametrize("name", ["c1_literal", "c1_stable", "hybrid_216", "scaled_20k"])
def test_forces_fp64(name):
    s, x, v, f, e = case(name)
    check_forces(s, x, f, e, "fp64")


@pytest.mark.parametrize("name", ["c1_stable", "hybrid_216", "scaled_20k"])
def test_forces_fp32(name):
    s, x, v, f, e = case(name)
    check_forces(s, x, f, e, "fp32")


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_forces_full_size_800k_atoms(precision):
    """The benchmark's workload (200k tetrahedra, 800k atoms), every atom compared."""
    s, x, v, f, e = case("c2_800k")
    check_forces(s, x, f, e, precision)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_com_and_resolution(precision):
    s, x, v, f, e = case("hybrid_216")
    R, dxc, w = oracle.Oracle(s).com_lambda(x)
    sim = gpu(s, precision)
    sim.set_state(x)
    com, wg = sim.com_lambda()
    d = com - R
    d -= np.array(s.box) * np.rint(d / np.array(s.box))
    assert np.abs(d).max() < 1e-12
    assert np.abs(wg - w).max() < (1e-14 if precision == "fp64" else 2e-6)
    assert ((w > 0) & (w < 1)).any() and (w == 1).any() and (w == 0).any()


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_thermodynamic_force_table(precision):
    s, x, v, _, _ = case("hybrid_216")
    o = oracle.Oracle(s)
    tf = 0.8 * np.sin(np.arange(len(s.tf)) * 0.7)
    o.set_tf(tf)
    f_ref, e_ref = o.forces(x)
    sim = gpu(s, precision)
    sim.set_tf(tf)
    assert np.array_equal(sim.get_tf(), tf)
    sim.set_state(x)
    f, _ = sim.forces()
    assert rel_rms(f, f_ref) <= TOL[precision]


# ---- limits of Eq. 1 and conservation -------------------------------------------------

@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("geom", ["all_at", "all_cg", "step", "two_cells"])
def test_edge_geometries(precision, geom):
    if geom == "all_at":
        s = inputs.tetra_system(216, (25.8, 12.9, 6.45), 1e3, 1.0, seed=6)
    elif geom == "all_cg":
        s = inputs.tetra_system(216, (25.8, 12.9, 6.45), 0.0, 0.0, seed=7)
    elif geom == "step":
        s = inputs.tetra_system(216, (25.8, 12.9, 6.45), 8.0, 0.0, seed=8)
    else:  # 2 cells along y and z: the 27-cell stencil must not double count
        s = inputs.tetra_system(64, (17.2, 6.0, 6.0), 5.0, 2.0, seed=9)
    x, v = inputs.tetra_state(s)
    f_ref, e_ref = oracle.Oracle(s).forces(x)
    check_forces(s, x, f_ref, e_ref, precision)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_point_particles(precision):
    """One atom per molecule: AT and CG act between the same points."""
    s = inputs.tetra_system(400, (20.0, 10.0, 10.0), 6.0, 2.0, seed=10)
    s.na, s.mass, s.bonds = 1, np.ones(1), np.zeros((0, 2), np.int32)
    rng = np.random.default_rng(10)
    g = np.stack(np.meshgrid(np.arange(10), np.arange(5), np.arange(8), indexing="ij"), -1).reshape(-1, 3)
    x = (g + 0.5) * np.array([2.0, 2.0, 1.25]) + rng.uniform(-0.1, 0.1, g.shape)
    f_ref, e_ref = oracle.Oracle(s).forces(x)
    check_forces(s, x, f_ref, e_ref, precision)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_newton_third_law(precision):
    s, x, v, f, e = case("hybrid_216")
    sim = gpu(s, precision)
    sim.set_state(x)
    fg, _ = sim.forces()
    tol = 1e-12 if precision == "fp64" else 1e-6
    assert np.abs(fg.sum(0)).max() <= tol * np.abs(fg).sum()


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_deterministic(precision):
    s, x, v, f, e = case("scaled_20k")
    sim = gpu(s, precision)
    sim.set_state(x, v)
    f1, _ = sim.forces()
    f2, _ = sim.forces()
    assert np.array_equal(f1, f2)
    sim.set_state(x, v, f1)
    sim.step(20)
    a = sim.get_state()
    sim.set_state(x, v, f1)
    sim.set_step(0)
    sim.build_lists()
    sim.step(20)
    b = sim.get_state()
    for p, q in zip(a, b):
        assert np.array_equal(p, q)


# ---- trajectories -----------------------------------------------------------------------

@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_trajectory_divergence_100_steps(precision):
    """Langevin velocity Verlet with identical Philox noise: the GPU trajectory follows the
    oracle's; the divergence curve stays below a precision-dependent envelope."""
    s, x, v, f0, _ = case("c1_stable")
    o = oracle.Oracle(s)
    sim = gpu(s, precision)
    sim.set_state(x, v)
    sim.compute_forces(energies=False)
    _, _, fg = sim.get_state()
    xo, vo, fo = x, v, f0
    L = np.array(s.box)
    curve = []
    for k in range(10):
        sim.step(10)
        xo, vo, fo = o.run(xo, vo, fo, 10 * k, 10)
        xg, vg, fg = sim.get_state()
        dx = xg - xo
        dx -= L * np.rint(dx / L)
        curve.append((np.abs(dx).max(), np.abs(vg - vo).max()))
    sim.check()
    assert sim.get_step() == 100
    env = {"fp64": (1e-11, 1e-9), "fp32": (1e-5, 1e-3)}[precision]
    print(precision, "divergence curve", [f"{a:.1e}" for a, _ in curve], [f"{b:.1e}" for _, b in curve])
    assert curve[0][0] < env[0] / 10
    # every point of the curve (positions and velocities) stays inside the envelope
    assert max(a for a, _ in curve) < env[0] and max(b for _, b in curve) < env[1]
    stats = sim.list_stats()
    assert stats["rebuilds"] >= 2 and stats["n_hr"] + stats["n_cg"] == s.M


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_kinetic_energy_and_momentum(precision):
    s, x, v, f, e = case("scaled_20k")
    o = oracle.Oracle(s)
    sim = gpu(s, precision)
    sim.set_state(x, v)
    ke, p = sim.kinetic()
    ke_ref, p_ref = o.kinetic(v)
    assert ke == pytest.approx(ke_ref, rel=1e-13)
    assert np.allclose(p, p_ref, atol=1e-10)


# ---- density profile and thermodynamic-force iteration -------------------------------------

@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_density_histogram_bit_exact_and_tf_update(precision):
    s, x, v, f, e = case("scaled_20k")
    o = oracle.Oracle(s)
    sim = gpu(s, precision)
    sim.set_state(x)
    sim.density_accumulate()
    sim.density_accumulate()
    counts, ns = sim.density_get()
    ref_d, _ = o.density(x, len(s.tf), 10)
    assert ns == 2
    assert np.array_equal(counts, 2 * ref_d)
    tf0 = 0.1 * np.cos(np.arange(len(s.tf)))
    sim.set_tf(tf0)
    sim.tf_update(alpha=3.0)
    tf_gpu = sim.get_tf()
    tf_ref = o.tf_update(tf0, 2 * ref_d, nsamples=2, alpha=3.0)
    assert np.allclose(tf_gpu, tf_ref, rtol=1e-13, atol=1e-15)
    counts, ns = sim.density_get()
    assert ns == 0 and not counts.any()


# ---- radial distribution function -------------------------------------------------------

@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_rdf_counts_bit_exact(precision):
    """COM pair-distance histogram (0..5 sigma, 0.02 bins) equals the oracle's all-pairs
    count on 80k atoms; bins are decided in FP64 on both sides."""
    s, x, v, f, e = case("scaled_20k")
    sim = gpu(s, precision)
    sim.set_state(x)
    c = sim.rdf_counts(250, 0.02)[0]
    ref = oracle.Oracle(s).rdf_counts(x, 250, 0.02)
    assert np.array_equal(c, ref)
    assert ref.sum() > 100_000
    from paper_1806_10841_gb300 import adress

    with pytest.raises(adress.AdressError):
        sim.rdf_counts(5000, 0.02)  # beyond half the box
    sim.close()


# ---- host-visible error paths (no GPU fault: device flags read back by the host) ----------

def test_list_capacity_grows_automatically():
    s, x, v, f, e = case("hybrid_216")
    sim = gpu(s, "fp64", max_neighbors=4)
    sim.set_state(x)
    fg, _ = sim.forces()
    assert rel_rms(fg, f) <= TOL["fp64"]
    st = sim.list_stats()
    assert st["capacity"] >= st["max_nn"] > 4


def test_broken_bond_is_reported():
    from paper_1806_10841_gb300 import adress

    s = inputs.scaled_c2(2000)
    s.r_ext = 1.2  # wide enough lists that the stretched molecule is still listed
    x, v = inputs.tetra_state(s)
    x[1] = np.mod(x[0] + np.array([1.6, 0.0, 0.0]), s.box)  # beyond R0 = 1.5
    sim = gpu(s, "fp32")
    sim.set_state(x)
    sim.compute_forces(energies=False)
    with pytest.raises(adress.AdressError) as ei:
        sim.check()
    assert ei.value.status == 5
    sim.check()  # cleared


def test_invalid_configs_are_rejected():
    from paper_1806_10841_gb300 import adress

    s = inputs.tetra_system(8, (4.0, 4.0, 4.0), 1.0, 1.0)  # box shorter than twice r_list
    with pytest.raises(adress.AdressError) as ei:
        gpu(s, "fp32")
    assert ei.value.status == 1
    s = inputs.tetra_system(1, (20.0, 20.0, 20.0), 1.0, 1.0)
    with pytest.raises(adress.AdressError):
        gpu(s, "fp64")


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_run_block_matches_oracle_sequence(precision):
    """adress_run: 20 steps with a density sample every 5 and one thermodynamic-force update,
    against the oracle doing the same sequence."""
    s, x, v, f0, _ = case("scaled_20k")
    o = oracle.Oracle(s)
    sim = gpu(s, precision)
    sim.set_state(x, v)
    sim.compute_forces(energies=False)
    sim.run(20, sample_every=5, tf_update=True, alpha=2.0)
    sim.check()
    xg, vg, _ = sim.get_state()
    xo, vo, fo = x, v, f0
    counts = np.zeros(len(s.tf), dtype=np.int64)
    for k in range(4):
        xo, vo, fo = o.run(xo, vo, fo, 5 * k, 5)
        cd, _ = o.density(xo, len(s.tf), 4)
        counts += cd
    tf_ref = o.tf_update(np.zeros(len(s.tf)), counts, nsamples=4, alpha=2.0)
    L = np.array(s.box)
    dx = xg - xo
    dx -= L * np.rint(dx / L)
    assert np.abs(dx).max() < (1e-10 if precision == "fp64" else 1e-4)
    tf_gpu = sim.get_tf()
    assert np.allclose(tf_gpu, tf_ref, rtol=1e-9, atol=1e-12)
    assert sim.get_step() == 20
    counts_g, ns = sim.density_get()
    assert ns == 0 and not counts_g.any()  # reset by the update


@pytest.mark.parametrize("name", ["hybrid_216", "c1_stable"])
def test_neighbour_lists_are_complete_and_exact(name):
    """Every molecule pair within its list cutoff is listed (both directions), no pair beyond
    it: r_list = max(rc_cg, rc_at + 2 r_ext) + skin between two high-resolution work items,
    rc_cg + skin when either is a coarse-grained item (weight 0 until the next build)."""
    s, x, v, f, e = case(name)
    sim = gpu(s, "fp64")
    sim.set_state(x)
    sim.build_lists()
    st = sim.list_stats()
    items, _, _ = sim.neighbour_lists()
    hr = np.zeros(s.M, dtype=bool)
    hr[items[:st["n_hr"]]] = True
    assert 0 < st["n_hr"] < s.M  # both kinds present
    com, _ = sim.com_lambda()
    L = np.array(s.box)
    d = com[:, None, :] - com[None, :, :]
    d -= L * np.rint(d / L)
    r = np.sqrt((d ** 2).sum(-1))
    r_list = max(s.rc_cg, s.rc_at + 2 * s.r_ext) + s.skin
    cut = np.where(hr[:, None] & hr[None, :], r_list, s.rc_cg + s.skin)
    assert r_list > s.rc_cg + s.skin  # the two cutoffs differ in this geometry
    off = ~np.eye(s.M, dtype=bool)
    expect = {(int(a), int(b_)) for a, b_ in zip(*np.nonzero(off & (r < cut - 1e-6)))}
    maybe = {(int(a), int(b_)) for a, b_ in zip(*np.nonzero(off & (np.abs(r - cut) <= 1e-6)))}
    assert st["max_nn"] <= st["capacity"]
    assert expect  # non-trivial
    got = sim.neighbour_pairs()
    assert expect <= got and got <= expect | maybe
    # symmetric: the mirror slots of the network force rely on it
    assert {(b_, a) for a, b_ in got} == got


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_energy_trace_of_all_atomistic_nve_follows_the_oracle(precision):
    """lambda = 1, no thermostat: the total energy after every 10 of 100 velocity-Verlet steps
    equals the oracle's (FP64: 1e-10 relative), and stays conserved."""
    s = inputs.tetra_system(1000, (34.20, 17.10, 17.10), 1e3, 1.0, gamma=0.0, dt=0.001)
    x, v = inputs.tetra_state(s)
    o = oracle.Oracle(s)
    sim = gpu(s, precision)
    sim.set_state(x, v)
    sim.compute_forces(energies=False)
    f = o.forces(x)[0]
    xo, vo = x, v

    def total_ref(xx, vv):
        _, e = o.forces(xx)
        return o.kinetic(vv)[0] + e["E_at"] + e["E_cg"] + e["E_bond"]

    def total_gpu():
        _, e = sim.forces()
        return sim.kinetic()[0] + e["E_at"] + e["E_cg"] + e["E_bond"]

    E0 = total_ref(x, v)
    tol = {"fp64": 1e-10, "fp32": 1e-5}[precision]
    for k in range(10):
        sim.step(10)
        xo, vo, f = o.run(xo, vo, f, 10 * k, 10)
        Eg, Er = total_gpu(), total_ref(xo, vo)
        assert abs(Eg - Er) <= tol * abs(Er), (k, Eg, Er)
        assert abs(Er - E0) <= 1e-3 * s.N
    sim.check()
    sim.close()
