"""Force-matched CG table on the GPU (adress_cg_fit) against the oracle's
force_matched_table on the same samples, and the fitted table in use."""
import math

import numpy as np
import pytest

import oracle
from paper_1806_10841_gb300 import inputs

pytestmark = pytest.mark.gpu


def all_atomistic(M, seed):
    s = inputs.scaled_c2(M, seed=seed)
    s.d_at = 1e3  # every molecule atomistic: the samples come from the atomistic model
    x, v = inputs.tetra_state(s)
    return s, x, v


def fit_both(sim, s, feat, t, h, n_min, install=False):
    F, V = sim.cg_fit(h, n_min, install=install)
    Fo, Vo = oracle.force_matched_table(feat[:, 0].astype(np.float64), t.astype(np.float64), h, n_min, s.cg_dr,
                                        len(s.cg_F) - 1, s.rc_cg)
    return F, V, Fo, Vo


@pytest.mark.parametrize("h,n_min", [(0.02, 5), (0.005, 1)])
def test_cg_fit_matches_oracle(h, n_min):
    from paper_1806_10841_gb300 import adress

    s, x, _ = all_atomistic(2000, 21)
    feat, t, _ = oracle.Oracle(s).collect_pairs(x, s.rc_cg)
    feat, t = feat.astype(np.float32), t.astype(np.float32)  # the library holds float samples
    sim = adress.AdResS(s, precision="fp64")
    sim.mlp_load_samples(feat, t)
    F, V, Fo, Vo = fit_both(sim, s, feat, t, h, n_min)
    print(f"CGFIT h={h} max|dF|={np.abs(F - Fo).max():.2e} max|F|={np.abs(Fo).max():.2e}")
    assert np.abs(F - Fo).max() <= 1e-12 * np.abs(Fo).max()
    assert np.abs(V - Vo).max() <= 1e-12 * np.abs(Vo).max()
    assert np.abs(Fo).max() > 1.0  # a non-trivial table
    sim.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_installed_table_drives_the_cg_force(precision):
    """install=True: the fitted table becomes the CG force of the handle; the forces of an
    all-CG box then equal the oracle's with the oracle's own fitted table."""
    import copy

    from paper_1806_10841_gb300 import adress

    s, x, _ = all_atomistic(2000, 22)
    feat, t, _ = oracle.Oracle(s).collect_pairs(x, s.rc_cg)
    feat, t = feat.astype(np.float32), t.astype(np.float32)
    s_cg = copy.copy(s)
    s_cg.d_at, s_cg.d_hy = 0.0, 0.0  # every molecule coarse-grained
    sim = adress.AdResS(s_cg, precision=precision)
    sim.mlp_load_samples(feat, t)
    F, V, Fo, Vo = fit_both(sim, s, feat, t, 0.02, 5, install=True)
    s_ref = copy.copy(s_cg)
    s_ref.cg_F, s_ref.cg_V = Fo, Vo
    f_ref, e_ref = oracle.Oracle(s_ref).forces(x)
    sim.set_state(x)
    f, e = sim.forces()
    sim.check()
    rel = math.sqrt(((f - f_ref) ** 2).sum() / (f_ref ** 2).sum())
    assert rel <= (1e-10 if precision == "fp64" else 2e-5), rel
    assert e["E_cg"] == pytest.approx(e_ref["E_cg"], rel=1e-10 if precision == "fp64" else 2e-5)
    sim.close()


def test_cg_fit_full_size_800k_atoms():
    """The benchmark's fluid, all atomistic: every pair within rc_cg of the 800k-atom state
    collected on the GPU (~0.5M samples), fitted on the GPU and by the oracle from the same
    samples."""
    from paper_1806_10841_gb300 import adress

    s = inputs.c2_800k()
    s.d_at = 1e4
    x, v = inputs.tetra_state(s)
    sim = adress.AdResS(s, precision="fp64")
    sim.set_state(x, v)
    n = sim.mlp_collect(cap=2_000_000)
    assert n > 300_000
    feat, t, _ = sim.mlp_samples(n)
    F, V, Fo, Vo = fit_both(sim, s, feat, t, 0.01, 20)
    assert np.abs(F - Fo).max() <= 1e-12 * np.abs(Fo).max()
    assert np.abs(V - Vo).max() <= 1e-12 * np.abs(Vo).max()
    sim.close()


def test_water_samples_and_table_match_oracle():
    """The water-like fluid, all atomistic: the GPU's samples (features, and the site-pair
    Lennard-Jones + reaction-field force between two molecules projected on their axis) and
    the force-matched table from them against the oracle's."""
    from paper_1806_10841_gb300 import adress

    s = inputs.scaled_c3(3000)
    s.d_at = 1e3
    x, v = inputs.water_state(s)
    feat_o, t_o, ids_o = oracle.Oracle(s).collect_pairs(x, s.rc_cg)
    sim = adress.AdResS(s, precision="fp32")
    sim.set_state(x, v)
    n = sim.mlp_collect(cap=2_000_000)
    feat, t, ids = sim.mlp_samples(n)
    key_o = {tuple(map(int, p)): k for k, p in enumerate(ids_o)}
    assert {tuple(map(int, p)) for p in ids} == set(key_o)
    order = np.array([key_o[tuple(map(int, p))] for p in ids])
    assert np.abs(feat - feat_o[order]).max() < 2e-5
    scale = np.abs(t_o).max()
    print(f"WATER samples={n} max|dt|={np.abs(t - t_o[order]).max():.2e} scale={scale:.2e}")
    assert np.abs(t - t_o[order]).max() <= 1e-4 * scale
    h = 0.01
    F, V, Fo, Vo = fit_both(sim, s, feat, t, h, 5)
    assert np.abs(F - Fo).max() <= 1e-12 * np.abs(Fo).max()
    assert np.abs(V - Vo).max() <= 1e-12 * np.abs(Vo).max()
    sim.close()
