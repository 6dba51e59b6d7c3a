"""Batched replicas: independent systems of uneven size and slab geometry stepped by the
same kernels in one handle, against single-system handles and the FP64 oracle.

Each replica's lists hold only its own molecules, its cells and neighbour order are those
of a single-system handle, and its thermostat noise is keyed by its own replica id and
atom index within the replica; so step-0 forces are bit-identical to the single-system
path, and trajectories agree with the oracle run with the same replica id.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1806_10841_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "fp32": 2e-5}
TF_BINS = 48


def rel_rms(a, b):
    return math.sqrt(((a - b) ** 2).sum() / (b ** 2).sum())


def small_batch():
    """Five replicas: a small hybrid box, the c1-stable fluid, a 2000-molecule scaled fluid,
    an all-atomistic box (slab wider than the box) and an all-coarse-grained one."""
    systems = [
        inputs.tetra_system(216, (25.8, 12.9, 6.45), 5.0, 2.5, tf_bins=TF_BINS),
        inputs.tetra_system(1000, (34.20, 17.10, 17.10), 5.0, 2.5, tf_bins=TF_BINS),
        inputs.tetra_system(2000, (58.48, 29.24, 29.24), 11.7, 2.9, tf_bins=TF_BINS),
        inputs.tetra_system(400, (20.0, 14.0, 14.0), 40.0, 1.0, tf_bins=TF_BINS),
        inputs.tetra_system(300, (20.0, 12.0, 12.5), 0.0, 0.0, tf_bins=TF_BINS),
    ]
    x, v = inputs.replica_states(systems)
    return systems, x, v


_cache = {}


def batch_case():
    if "b" not in _cache:
        _cache["b"] = small_batch()
    return _cache["b"]


def sim_of(systems, precision, **kw):
    from paper_1806_10841_gb300 import adress

    return adress.AdResS(systems, precision=precision, **kw)


def split(arr, sim):
    return [arr[sim.atom0[r]:sim.atom0[r + 1]] for r in range(sim.n_replicas)]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_batch_forces_equal_single_system_forces_and_oracle(precision):
    systems, x, v = batch_case()
    sim = sim_of(systems, precision)
    sim.set_state(x)
    f, e = sim.forces()
    sim.check()
    xs, fs = split(x, sim), split(f, sim)
    e_sum = {k: 0.0 for k in ("E_at", "E_cg", "E_bond", "virial")}
    for r, s in enumerate(systems):
        single = sim_of(s, precision, replica=r)
        single.set_state(xs[r])
        f1, e1 = single.forces()
        single.close()
        assert np.array_equal(fs[r], f1), r  # same lists, same order, same arithmetic
        for k in e_sum:
            e_sum[k] += e1[k]
        f_ref, _ = oracle.Oracle(s, replica=r).forces(xs[r])
        assert rel_rms(fs[r], f_ref) <= TOL[precision], r
    for k in e_sum:
        assert e[k] == pytest.approx(e_sum[k], rel=1e-12, abs=1e-12)
    st = sim.list_stats()
    assert st["n_hr"] + st["n_cg"] == sim.M
    sim.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_batch_trajectories_follow_the_oracle_per_replica(precision):
    """40 Langevin steps of the whole batch; each replica against the oracle run with its
    replica id (the noise differs between replicas)."""
    systems, x, v = batch_case()
    sim = sim_of(systems, precision)
    sim.set_state(x, v)
    sim.compute_forces(energies=False)
    sim.step(40)
    sim.check()
    assert sim.get_step() == 40
    xg, vg, _ = sim.get_state()
    xs, vs = split(x, sim), split(v, sim)
    xgs, vgs = split(xg, sim), split(vg, sim)
    env = {"fp64": (1e-9, 1e-7), "fp32": (1e-3, 1e-1)}[precision]
    for r, s in enumerate(systems):
        o = oracle.Oracle(s, replica=r)
        f0, _ = o.forces(xs[r])
        xo, vo, _ = o.run(xs[r], vs[r], f0, 0, 40)
        L = np.array(s.box)
        dx = xgs[r] - xo
        dx -= L * np.rint(dx / L)
        assert np.abs(dx).max() < env[0], (r, np.abs(dx).max())
        assert np.abs(vgs[r] - vo).max() < env[1], (r, np.abs(vgs[r] - vo).max())
    # replicas with different ids draw different noise
    o0 = oracle.Oracle(systems[0], replica=1)
    f0, _ = o0.forces(xs[0])
    xo, _, _ = o0.run(xs[0], vs[0], f0, 0, 40)
    assert np.abs(xgs[0] - xo).max() > 1e-6
    sim.close()


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_batch_density_histograms_and_tf_update_per_replica(precision):
    systems, x, v = batch_case()
    sim = sim_of(systems, precision)
    sim.set_state(x)
    sim.density_accumulate()
    counts, ns = sim.density_get()
    assert ns == 1
    counts = counts.reshape(len(systems), TF_BINS)
    xs = split(x, sim)
    tf0 = np.stack([0.05 * (r + 1) * np.cos(np.arange(TF_BINS)) for r in range(len(systems))])
    sim.set_tf(tf0.reshape(-1))
    sim.tf_update(alpha=2.0)
    tf_gpu = sim.get_tf().reshape(len(systems), TF_BINS)
    for r, s in enumerate(systems):
        o = oracle.Oracle(s, replica=r)
        ref_d, _ = o.density(xs[r], TF_BINS, 10)
        assert np.array_equal(counts[r], ref_d), r
        tf_ref = o.tf_update(tf0[r], ref_d, nsamples=1, alpha=2.0)
        assert np.allclose(tf_gpu[r], tf_ref, rtol=1e-13, atol=1e-15), r
    counts, ns = sim.density_get()
    assert ns == 0 and not counts.any()
    sim.close()


def test_batch_rdf_counts_per_replica_bit_exact():
    systems, x, v = batch_case()
    sim = sim_of(systems, "fp32")
    sim.set_state(x)
    c = sim.rdf_counts(150, 0.02)
    xs = split(x, sim)
    for r, s in enumerate(systems):
        assert np.array_equal(c[r], oracle.Oracle(s, replica=r).rdf_counts(xs[r], 150, 0.02)), r
    sim.close()


def test_batch_run_block_with_tf_iteration_matches_single_handles():
    """adress_run over the batch (density samples + one TF update) gives each replica the
    thermodynamic-force table its own single-system handle gets."""
    systems, x, v = batch_case()
    sim = sim_of(systems, "fp64")
    sim.set_state(x, v)
    sim.compute_forces(energies=False)
    sim.run(20, sample_every=5, tf_update=True, alpha=2.0)
    sim.check()
    tf_b = sim.get_tf().reshape(len(systems), TF_BINS)
    xs, vs = split(x, sim), split(v, sim)
    for r, s in enumerate(systems):
        one = sim_of(s, "fp64", replica=r)
        one.set_state(xs[r], vs[r])
        one.compute_forces(energies=False)
        one.run(20, sample_every=5, tf_update=True, alpha=2.0)
        one.check()
        assert np.allclose(tf_b[r], one.get_tf(), rtol=1e-9, atol=1e-12), r
        one.close()
    sim.close()


def test_autotune_restores_the_state_and_keeps_the_fastest():
    systems, x, v = batch_case()
    sim = sim_of(systems, "fp32")
    sim.set_state(x, v)
    sim.compute_forces(energies=False)
    sim.step(5)
    before = sim.get_state()
    step0 = sim.get_step()
    blk0, skin0 = sim.get_tuning()
    rows = sim.autotune(nsteps=10)
    assert len(rows) >= 9
    assert all(r[3] <= r[2] <= r[4] for r in rows)  # median inside the runs' range
    blk, skin = sim.get_tuning()
    best = min(rows, key=lambda r: r[2])
    start = [r for r in rows if (r[0], r[1]) == (blk0, skin0)][0]
    # the fastest median wins only when it beats every run of the starting setting
    expect = (best[0], best[1]) if best[2] < start[3] else (blk0, skin0)
    assert (blk, skin) == expect
    after = sim.get_state()
    for a, b in zip(before, after):
        assert np.array_equal(a, b)
    assert sim.get_step() == step0
    # forces with the tuned configuration still match the oracle
    f, _ = sim.forces()
    xs, fs = split(before[0], sim), split(f, sim)
    for r, s in enumerate(systems):
        f_ref, _ = oracle.Oracle(s, replica=r).forces(xs[r])
        assert rel_rms(fs[r], f_ref) <= TOL["fp32"], r
    sim.close()


@pytest.mark.parametrize("block,skin", [(32, 0.15), (64, 0.6)])
def test_tuning_changes_no_result_beyond_rounding(block, skin):
    systems, x, v = batch_case()
    ref = sim_of(systems, "fp64")
    ref.set_state(x, v)
    f_ref, _ = ref.forces()
    sim = sim_of(systems, "fp64")
    sim.set_tuning(block, skin)
    sim.set_state(x, v)
    f, _ = sim.forces()
    assert rel_rms(f, f_ref) < 1e-14
    ref.compute_forces(energies=False)
    sim.compute_forces(energies=False)
    ref.step(30)
    sim.step(30)
    assert np.abs(sim.get_state()[0] - ref.get_state()[0]).max() < 1e-9
    ref.close()
    sim.close()


def test_64_replica_workload_full_size():
    """The 64-replica workload (log-uniform 500..20000 molecules, ~1.5M atoms): FP32 forces of
    sampled replicas equal their single-system forces and match the oracle; 50 steps run
    clean."""
    systems = inputs.replica_batch(64)
    x, v = inputs.replica_states(systems)
    sim = sim_of(systems, "fp32")
    sim.set_state(x, v)
    f, _ = sim.forces()
    sim.check()
    xs, fs = split(x, sim), split(f, sim)
    sizes = [s.M for s in systems]
    picks = sorted({int(np.argmin(sizes)), int(np.argmax(sizes)), 17})
    for r in picks:
        one = sim_of(systems[r], "fp32", replica=r)
        one.set_state(xs[r])
        f1, _ = one.forces()
        one.close()
        assert np.array_equal(fs[r], f1), r
    r = int(np.argmin(sizes))
    f_ref, _ = oracle.Oracle(systems[r], replica=r).forces(xs[r])
    assert rel_rms(fs[r], f_ref) <= TOL["fp32"]
    sim.step(50)
    sim.check()
    _, vg, _ = sim.get_state()
    assert np.isfinite(vg).all()
    sim.close()
