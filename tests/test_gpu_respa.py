"""Multiple time stepping (impulse r-RESPA, CG forces as the slow part) on the GPU against
the FP64 oracle: forces at inner and outer time levels, trajectories, and conservation of
the Hamiltonian with energy interpolation.  Tolerances as for the single-step integrator:
force relative RMS <= 1e-10 (FP64) and <= 2e-5 (FP32)."""
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


def case(scheme, n, M=6000, seed=4, **kw):
    s = inputs.scaled_c2(M, seed=seed, **kw)
    s.scheme, s.respa_n = scheme, n
    s.tf = np.linspace(0.4, -0.4, len(s.tf))
    if scheme == 1:
        s.fec = np.random.default_rng(seed).uniform(-2.0, 2.0, 9)
    x, v = inputs.tetra_state(s)
    return s, x, v


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("scheme", [0, 1])
def test_forces_at_inner_and_outer_levels(precision, scheme):
    s, x, _ = case(scheme, 3)
    o = oracle.Oracle(s)
    sim = sim_of(s, precision)
    sim.set_state(x)
    for level in (0, 1, 2, 3, 7):
        sim.set_step(level)
        f, e = sim.forces()
        f_ref, e_ref = o.forces(x, step=level)
        assert rel_rms(f, f_ref) <= TOL[precision], (level, rel_rms(f, f_ref))
        scale = abs(e_ref["E_at"]) + abs(e_ref["E_cg"]) + abs(e_ref["E_bond"])
        for k in ("E_at", "E_cg", "E_bond"):
            assert abs(e[k] - e_ref[k]) <= TOL[precision] * scale, (level, k)
    sim.check()
    sim.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("scheme", [0, 1])
def test_trajectory_follows_the_oracle(precision, scheme):
    s, x, v = case(scheme, 4, M=2000, seed=6)
    sim = sim_of(s, precision)
    sim.set_state(x, v)
    sim.compute_forces(energies=False)
    sim.step(41)
    sim.check()
    xg, vg, _ = sim.get_state()
    o = oracle.Oracle(s)
    f0, _ = o.forces(x, step=0)
    xo, vo, _ = o.run(x, v, f0, 0, 41)
    L = np.array(s.box)
    dx = xg - xo
    dx -= L * np.rint(dx / L)
    env = {"fp64": (1e-9, 1e-7), "fp32": (1e-3, 1e-1)}[precision]
    assert np.abs(dx).max() < env[0]
    assert np.abs(vg - vo).max() < env[1]
    sim.close()


def test_hamiltonian_conserved_with_multiple_time_steps():
    """Energy interpolation, FP64, no thermostat or thermodynamic force, 3 inner steps per
    outer step: |H - H0| shrinks like the outer step squared."""
    amp = {}
    for dt_out in (0.003, 0.0015):
        s = inputs.scaled_c2(4000, seed=11)
        s.gamma, s.dt, s.scheme, s.respa_n = 0.0, dt_out / 3, 1, 3
        x, v = inputs.tetra_state(s)
        sim = sim_of(s, "fp64")
        sim.set_state(x, v)
        _, e = sim.forces()
        H0 = sim.kinetic()[0] + e["E_at"] + e["E_cg"] + e["E_bond"]
        dev = 0.0
        for _ in range(8):
            sim.step(3 * int(round(0.25 / dt_out)))
            sim.check()
            _, e = sim.forces()
            dev = max(dev, abs(sim.kinetic()[0] + e["E_at"] + e["E_cg"] + e["E_bond"] - H0))
        amp[dt_out] = dev / s.N
        sim.close()
    assert amp[0.0015] < 1e-3
    assert 3.0 < amp[0.003] / amp[0.0015] < 5.0


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_combinations_water_spheres_and_batches(precision):
    """Multiple time stepping combined with the water model, with energy interpolation in the
    sphere geometry, and with batched replicas: forces at an inner and an outer level."""
    from paper_1806_10841_gb300 import adress

    w = inputs.scaled_c3(2000)
    w.respa_n, w.scheme = 2, 1
    xw, _ = inputs.water_state(w)
    sp = inputs.scaled_c2(6000, seed=8)
    L = np.array(sp.box)
    sp.d_at, sp.d_hy = 4.0, 4.0
    sp.centers = np.array([[0.25 * L[0], 0.5 * L[1], 0.5 * L[2]], [0.98 * L[0], 0.1 * L[1], 0.9 * L[2]]])
    sp.tf = np.linspace(0.3, -0.3, int(math.ceil((sp.d_at + sp.d_hy) / sp.tf_dx)) + 2)
    sp.respa_n, sp.scheme, sp.fec = 3, 1, np.linspace(-1.0, 1.0, 5)
    xs, _ = inputs.tetra_state(sp)
    for s, x in ((w, xw), (sp, xs)):
        o = oracle.Oracle(s)
        sim = sim_of(s, precision)
        sim.set_state(x)
        for level in (0, 1):
            sim.set_step(level)
            f, _ = sim.forces()
            f_ref, _ = o.forces(x, step=level)
            assert rel_rms(f, f_ref) <= TOL[precision], (s.na, level)
        sim.check()
        sim.close()
    systems = [case(0, 2, M=M, seed=sd)[0] for M, sd in ((1500, 1), (2500, 1))]
    nt = max(len(s.tf) for s in systems)
    for s in systems:
        s.tf = np.zeros(nt)
    x, _ = inputs.replica_states(systems)
    sim = adress.AdResS(systems, precision=precision)
    sim.set_state(x)
    for level in (1, 2):
        sim.set_step(level)
        f, _ = sim.forces()
        for r, s in enumerate(systems):
            a0, a1 = sim.atom0[r], sim.atom0[r + 1]
            f_ref, _ = oracle.Oracle(s, replica=r).forces(x[a0:a1], step=level)
            assert rel_rms(f[a0:a1], f_ref) <= TOL[precision], (r, level)
    sim.check()
    sim.close()
