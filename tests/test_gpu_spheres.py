"""The self-adjusting geometry on the GPU (AT region = union of spheres around resolution
centres; Sec. "Self-adjusting adaptive resolution simulations") against the FP64 oracle.

Tolerances as for the slab: force relative RMS <= 1e-10 (FP64) and <= 2e-5 (FP32); density
counts bit-exact.  Centres overlap and straddle periodic faces; the thermodynamic-force cases
use well-separated centres (the nearest centre, hence the force direction, is then unique).
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


def sphere_system(centers, at=8.0, hy=4.0, M=8000, tf=None, seed=3):
    s = inputs.scaled_c2(M, seed=seed)
    s.d_at, s.d_hy = 0.5 * at, hy
    s.tf = np.zeros(int(math.ceil((s.d_at + s.d_hy) / s.tf_dx)) + 2) if tf is None else tf
    s.centers = np.asarray(centers, dtype=np.float64)
    return s


def overlapping_centers(s):
    L = np.array(s.box)
    return np.array([[0.1 * L[0], 0.5 * L[1], 0.5 * L[2]], [0.1 * L[0] + 3.0, 0.5 * L[1] + 2.0, 0.5 * L[2]],
                     [0.99 * L[0], 0.02 * L[1], 0.97 * L[2]], [0.6 * L[0], 0.3 * L[1], 0.8 * L[2]]])


def sim_of(s, precision):
    from paper_1806_10841_gb300 import adress

    return adress.AdResS(s, precision=precision)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_forces_and_resolution_with_overlapping_spheres(precision):
    s0 = sphere_system(np.zeros((1, 3)))
    s = sphere_system(overlapping_centers(s0))
    x, _ = inputs.tetra_state(s)
    o = oracle.Oracle(s)
    f_ref, e_ref = o.forces(x)
    _, _, w_ref = o.com_lambda(x)
    assert (w_ref == 1).any() and ((w_ref > 0) & (w_ref < 1)).any() and (w_ref == 0).any()
    sim = sim_of(s, precision)
    sim.set_state(x)
    f, e = sim.forces()
    sim.check()
    assert rel_rms(f, f_ref) <= TOL[precision]
    _, w = sim.com_lambda()
    assert np.abs(w - w_ref).max() <= (1e-14 if precision == "fp64" else 1e-5)
    sim.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_thermodynamic_force_along_the_nearest_centre(precision):
    s0 = sphere_system(np.zeros((1, 3)))
    L = np.array(s0.box)
    c = np.array([[0.25 * L[0], 0.5 * L[1], 0.5 * L[2]], [0.75 * L[0], 0.5 * L[1], 0.5 * L[2]]])
    nb = int(math.ceil((4.0 + 4.0) / s0.tf_dx)) + 2
    tf = 0.3 * np.sin(np.arange(nb))
    s = sphere_system(c, tf=tf)
    x, _ = inputs.tetra_state(s)
    f_ref, _ = oracle.Oracle(s).forces(x)
    sim = sim_of(s, precision)
    sim.set_state(x)
    f, _ = sim.forces()
    assert rel_rms(f, f_ref) <= TOL[precision]
    sim.close()


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_density_counts_and_tf_update_with_spheres(precision):
    s0 = sphere_system(np.zeros((1, 3)))
    L = np.array(s0.box)
    c = np.array([[0.25 * L[0], 0.5 * L[1], 0.5 * L[2]], [0.75 * L[0], 0.4 * L[1], 0.6 * L[2]]])
    s = sphere_system(c)
    x, _ = inputs.tetra_state(s)
    o = oracle.Oracle(s)
    sim = sim_of(s, precision)
    sim.set_state(x)
    sim.density_accumulate()
    counts, ns = sim.density_get()
    ref_d, _ = o.density(x, len(s.tf), 10)
    assert ns == 1 and np.array_equal(counts, ref_d)
    tf0 = 0.05 * np.cos(np.arange(len(s.tf)))
    sim.set_tf(tf0)
    sim.tf_update(alpha=4.0)
    assert np.allclose(sim.get_tf(), o.tf_update(tf0, ref_d, nsamples=1, alpha=4.0), rtol=1e-13, atol=1e-15)
    sim.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_run_block_and_moving_centres_follow_the_oracle(precision):
    s0 = sphere_system(np.zeros((1, 3)))
    L = np.array(s0.box)
    c = np.array([[0.3 * L[0], 0.5 * L[1], 0.5 * L[2]], [0.8 * L[0], 0.5 * L[1], 0.2 * L[2]]])
    s = sphere_system(c)
    x, v = inputs.tetra_state(s)
    o = oracle.Oracle(s)
    f0, _ = o.forces(x)
    sim = sim_of(s, precision)
    sim.set_state(x, v)
    sim.compute_forces(energies=False)
    sim.run(20, sample_every=5, tf_update=True, alpha=1.0)
    sim.check()
    xo, vo, fo = x, v, f0
    counts = np.zeros(len(s.tf), dtype=np.int64)
    for k in range(4):
        xo, vo, fo = o.run(xo, vo, fo, 5 * k, 5)
        counts += o.density(xo, len(s.tf), 4)[0]
    xg, _, _ = sim.get_state()
    dx = xg - xo
    dx -= L * np.rint(dx / L)
    assert np.abs(dx).max() < (1e-10 if precision == "fp64" else 1e-4)
    assert np.allclose(sim.get_tf(), o.tf_update(np.zeros(len(s.tf)), counts, nsamples=4, alpha=1.0),
                       rtol=1e-9, atol=1e-12)
    # the AT region follows moved centres
    c2 = c + np.array([5.0, -3.0, 2.0])
    sim.set_centers(c2)
    o.set_centers(np.mod(c2, L))
    _, w = sim.com_lambda()
    _, _, w_ref = o.com_lambda(xg if precision == "fp64" else xo)
    assert np.abs(w - w_ref).max() <= (1e-12 if precision == "fp64" else 1e-3)
    # stepping on: the lists are rebuilt for the moved region (no molecule listed as CG may
    # find itself in the new hybrid shells), and the run follows the oracle's
    import copy

    s2 = copy.copy(s)
    s2.centers, s2.tf = np.mod(c2, L), sim.get_tf()
    sim.step(10)
    sim.check()
    xo2, _, _ = oracle.Oracle(s2).run(xo, vo, fo, 20, 10)
    dx = sim.get_state()[0] - xo2
    dx -= L * np.rint(dx / L)
    assert np.abs(dx).max() < (1e-9 if precision == "fp64" else 1e-3)
    sim.close()


def test_batches_with_centres_are_rejected():
    from paper_1806_10841_gb300 import adress

    s = sphere_system(np.array([[5.0, 5.0, 5.0]]), M=2000)
    with pytest.raises(adress.AdressError) as ei:
        adress.AdResS([s, s], precision="fp32")
    assert ei.value.status == 1
