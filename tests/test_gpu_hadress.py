"""Energy interpolation (H-AdResS, Eq. Hmix) on the GPU against the FP64 oracle.

Tolerances as for force interpolation: per-atom force relative RMS <= 1e-10 (FP64 path) and
<= 2e-5 (FP32 path), energies (which here are the Hamiltonian's potential terms) to the
same relative bound.  Cases: slab and sphere geometry, with and without a free-energy
correction, the water-like model, the 800k-atom workload, a batch of replicas, trajectories
with the thermostat, and conservation of H without it.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1806_10841_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "fp32": 2e-5}


def rel_rms(a, b):
    return math.sqrt(((a - b) ** 2).sum() / (b ** 2).sum())


def sim_of(s, precision, **kw):
    from paper_1806_10841_gb300 import adress

    return adress.AdResS(s, precision=precision, **kw)


def hadress(s, fec=False, seed=0):
    s.scheme = 1
    if fec:
        s.fec = np.random.default_rng(seed).uniform(-3.0, 3.0, 17)
    return s


def tetra_case(geom, fec, M=8000, seed=3):
    s = inputs.scaled_c2(M, seed=seed)
    if geom == "spheres":
        L = np.array(s.box)
        s.d_at, s.d_hy = 4.0, 4.0
        s.centers = np.array([[0.2 * L[0], 0.5 * L[1], 0.5 * L[2]], [0.97 * L[0], 0.03 * L[1], 0.9 * L[2]],
                              [0.6 * L[0], 0.3 * L[1], 0.7 * L[2]]])
        s.tf = np.zeros(int(math.ceil((s.d_at + s.d_hy) / s.tf_dx)) + 2)
    s = hadress(s, fec, seed)
    x, v = inputs.tetra_state(s)
    return s, x, v


def check(s, x, precision):
    o = oracle.Oracle(s)
    f_ref, e_ref = o.forces(x)
    _, _, w = o.com_lambda(x)
    assert ((w > 0) & (w < 1)).sum() > 20
    sim = sim_of(s, precision)
    sim.set_state(x)
    f, e = sim.forces()
    sim.check()
    assert rel_rms(f, f_ref) <= TOL[precision], rel_rms(f, f_ref)
    scale = abs(e_ref["E_at"]) + abs(e_ref["E_cg"]) + abs(e_ref["E_bond"])
    for k in ("E_at", "E_cg", "E_bond"):
        assert abs(e[k] - e_ref[k]) <= TOL[precision] * scale, (k, e[k], e_ref[k])
    return sim, f, f_ref


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("geom,fec", [("slab", False), ("slab", True), ("spheres", False), ("spheres", True)])
def test_forces_and_hamiltonian_terms_match_oracle(precision, geom, fec):
    s, x, _ = tetra_case(geom, fec)
    sim, f, f_ref = check(s, x, precision)
    # the drift force matters: force interpolation's forces differ from these
    s.scheme, s.fec = 0, None
    f_fi, _ = oracle.Oracle(s).forces(x)
    assert rel_rms(f_fi, f_ref) > 100 * TOL[precision]
    st = sim.list_stats()
    assert st["n_hr"] + st["n_cg"] == s.M and st["n_cg"] > 0
    sim.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_water_model_with_energy_interpolation(precision):
    s = hadress(inputs.scaled_c3(3000), fec=True, seed=5)
    x, _ = inputs.water_state(s)
    sim, _, _ = check(s, x, precision)
    sim.close()


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_full_size_800k_atoms(precision):
    s = hadress(inputs.c2_800k())
    x, _ = inputs.tetra_state(s)
    sim, _, _ = check(s, x, precision)
    sim.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_trajectory_follows_the_oracle(precision):
    s, x, v = tetra_case("slab", True, M=2000, seed=7)
    sim = sim_of(s, precision)
    sim.set_state(x, v)
    sim.compute_forces(energies=False)
    sim.step(40)
    sim.check()
    xg, vg, _ = sim.get_state()
    o = oracle.Oracle(s)
    f0, _ = o.forces(x)
    xo, vo, _ = o.run(x, v, f0, 0, 40)
    L = np.array(s.box)
    dx = xg - xo
    dx -= L * np.rint(dx / L)
    env = {"fp64": (1e-9, 1e-7), "fp32": (1e-3, 1e-1)}[precision]
    assert np.abs(dx).max() < env[0]
    assert np.abs(vg - vo).max() < env[1]
    sim.close()


def test_batch_replicas_equal_single_systems():
    systems = [tetra_case("slab", False, M=M)[0] for M in (2000, 3000)]
    nt = max(len(s.tf) for s in systems)  # replicas share the thermodynamic-force grid
    for s in systems:
        s.tf = np.zeros(nt)
    x, v = inputs.replica_states(systems)
    sim = sim_of(systems, "fp32")
    sim.set_state(x)
    f, _ = sim.forces()
    sim.check()
    for r, s in enumerate(systems):
        a0, a1 = sim.atom0[r], sim.atom0[r + 1]
        one = sim_of(s, "fp32", replica=r)
        one.set_state(x[a0:a1])
        f1, _ = one.forces()
        one.close()
        assert np.array_equal(f[a0:a1], f1), r
        f_ref, _ = oracle.Oracle(s, replica=r).forces(x[a0:a1])
        assert rel_rms(f[a0:a1], f_ref) <= TOL["fp32"]
    sim.close()


def _hamiltonian(sim):
    _, e = sim.forces()
    return sim.kinetic()[0] + e["E_at"] + e["E_cg"] + e["E_bond"]


def test_hamiltonian_is_conserved_without_thermostat():
    """FP64, gamma = 0, no thermodynamic force: over 4000 molecules crossing the hybrid
    layer, |H - H0| shrinks like dt^2 (velocity Verlet on a Hamiltonian system)."""
    amp = {}
    for dt in (0.001, 0.0005):
        s = inputs.scaled_c2(4000, seed=11)
        s.gamma, s.dt = 0.0, dt
        s = hadress(s)
        x, v = inputs.tetra_state(s)
        sim = sim_of(s, "fp64")
        sim.set_state(x, v)
        H0 = _hamiltonian(sim)
        dev = 0.0
        for _ in range(10):
            sim.step(int(round(0.2 / dt)))
            sim.check()
            dev = max(dev, abs(_hamiltonian(sim) - H0))
        amp[dt] = dev / s.N
        sim.close()
    assert amp[0.0005] < 5e-4
    assert 3.0 < amp[0.001] / amp[0.0005] < 5.0


def test_learned_cg_force_is_refused_with_energy_interpolation():
    from paper_1806_10841_gb300 import adress

    s, x, _ = tetra_case("slab", False, M=2000)
    sim = sim_of(s, "fp32")
    params = adress.AdResS.mlp_unflatten(np.random.default_rng(0).normal(0, 0.1, adress.AdResS.MLP_NPAR))
    sim.mlp_set(params, np.zeros(9), np.ones(9), 1.0)
    with pytest.raises(adress.AdressError):
        sim.set_cg_mode(1)
    sim.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("lam", [0.0, 0.35, 1.0])
def test_uniform_lambda_forces_match_oracle(precision, lam):
    """Kirkwood mode: every molecule at the same l; the thermodynamic force and the
    free-energy correction configured on the system must not act."""
    s, x, _ = tetra_case("slab", True, M=4000, seed=9)
    s.tf = np.full(len(s.tf), 2.0)
    o = oracle.Oracle(s)
    o.set_uniform_lambda(lam)
    f_ref, e_ref = o.forces(x)
    sim = sim_of(s, precision)
    sim.set_state(x)
    sim.set_uniform_lambda(lam)
    f, e = sim.forces()
    sim.check()
    assert rel_rms(f, f_ref) <= TOL[precision]
    scale = abs(e_ref["E_at"]) + abs(e_ref["E_cg"]) + abs(e_ref["E_bond"])
    for k in ("E_at", "E_cg", "E_bond"):
        assert abs(e[k] - e_ref[k]) <= TOL[precision] * scale, k
    _, w = sim.com_lambda()
    assert np.all(w == (lam if precision == "fp64" else np.float32(lam)))
    st = sim.list_stats()
    assert st["n_hr"] == (s.M if lam > 0 else 0)
    sim.set_uniform_lambda(None)
    sim.build_lists()
    _, w = sim.com_lambda()
    assert ((w > 0) & (w < 1)).any()
    sim.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_kirkwood_integration_follows_the_oracle_protocol(precision):
    s, x, v = tetra_case("slab", False, M=1000, seed=12)
    lams = [0.3, 0.7]
    o = oracle.Oracle(s)
    g_ref, x_ref, _, step_ref = o.kirkwood(x, v, lams, n_equil=10, n_samples=3, every=5)
    sim = sim_of(s, precision)
    sim.set_state(x, v)
    sim.compute_forces(energies=False)
    g = sim.kirkwood(lams, n_equil=10, n_samples=3, every=5)
    sim.check()
    assert sim.get_step() == step_ref
    tol = 1e-8 if precision == "fp64" else 1e-3
    assert np.allclose(g, g_ref, rtol=tol, atol=tol * np.abs(g_ref).max())
    xg, _, _ = sim.get_state()
    L = np.array(s.box)
    dx = xg - x_ref
    dx -= L * np.rint(dx / L)
    assert np.abs(dx).max() < (1e-9 if precision == "fp64" else 1e-2)
    # resolution follows the geometry again
    _, w = sim.com_lambda()
    assert ((w > 0) & (w < 1)).any() and (w == 1).any()
    sim.close()
