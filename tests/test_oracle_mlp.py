"""Pins of the oracle's learned CG pair force (features, targets, network, gradients).

Checked against: numpy matmuls and an independent numpy bfloat16 rounding (forward),
central finite differences of the loss (gradients), rotation / permutation / exchange
invariances of the features, and the total intermolecular force of a two-molecule
system from the (separately pinned) force oracle (targets).
"""
import numpy as np
import pytest

import oracle
from paper_1806_10841_gb300 import inputs


def random_params(nh=64, seed=0, scale=0.3):
    rng = np.random.default_rng(seed)
    return dict(W1=rng.normal(0, scale, (nh, 9)), b1=rng.normal(0, 0.1, nh), W2=rng.normal(0, scale, (nh, nh)),
                b2=rng.normal(0, 0.1, nh), w3=rng.normal(0, scale, nh), b3=0.2,
                in_mean=rng.normal(0, 0.5, 9), in_std=rng.uniform(0.5, 2.0, 9), out_scale=3.0)


def np_bf16(a):
    """Round float64 values to bfloat16 (nearest even) through float32 bit patterns."""
    f = np.asarray(a, dtype=np.float32).copy()
    u = f.view(np.uint32)
    r = (u + np.uint32(0x7FFF) + ((u >> np.uint32(16)) & np.uint32(1))) & np.uint32(0xFFFF0000)
    return r.view(np.float32).astype(np.float64)


def np_forward(p, feat, bf16=False):
    rnd = np_bf16 if bf16 else (lambda a: a)
    x = rnd((feat - p["in_mean"]) / p["in_std"])
    silu = lambda z: z / (1 + np.exp(-z))
    h1 = rnd(silu(x @ rnd(p["W1"]).T + p["b1"]))
    h2 = silu(h1 @ rnd(p["W2"]).T + p["b2"])
    return h2 @ p["w3"] + p["b3"]


@pytest.mark.parametrize("bf16", [False, True])
def test_forward_matches_numpy(bf16):
    p = random_params(seed=1)
    feat = np.random.default_rng(2).normal(0, 1, (200, 9))
    m = oracle.OracleMLP(p, bf16=bf16)
    y = m.forward(feat)
    ref = np_forward(p, feat, bf16=bf16)
    # the bfloat16 case can differ where FP64 sums land on the other side of a rounding tie
    assert np.median(np.abs(y - ref)) < 1e-12
    assert np.mean(np.abs(y - ref) < 1e-10) > 0.98


def test_bf16_rounding_matches_numpy():
    vals = np.random.default_rng(3).normal(0, 10, 1000)
    assert all(oracle.bf16(v) == r for v, r in zip(vals, np_bf16(vals)))
    assert oracle.bf16(1.0 + 2 ** -9) == 1.0 and oracle.bf16(1.0 + 3 * 2 ** -9) == 1.0 + 2 ** -7


def test_gradients_match_finite_differences():
    p = random_params(nh=16, seed=4)
    rng = np.random.default_rng(5)
    feat = rng.normal(0, 1, (30, 9))
    target = rng.normal(0, 2, 30)
    loss, g = oracle.OracleMLP(p).loss_grad(feat, target)
    y = np_forward(p, feat)
    assert loss == pytest.approx(np.mean((y - target / p["out_scale"]) ** 2), rel=1e-12)
    h = 1e-6
    for name in ("W1", "b1", "W2", "b2", "w3", "b3"):
        arr = np.asarray(p[name], dtype=np.float64)
        flat = arr.reshape(-1)
        for idx in rng.choice(flat.size, min(6, flat.size), replace=False):
            pp, pm = dict(p), dict(p)
            a1, a2 = flat.copy(), flat.copy()
            a1[idx] += h
            a2[idx] -= h
            pp[name] = a1.reshape(arr.shape) if arr.ndim else float(a1[0])
            pm[name] = a2.reshape(arr.shape) if arr.ndim else float(a2[0])
            lp = np.mean((np_forward(pp, feat) - target / p["out_scale"]) ** 2)
            lm = np.mean((np_forward(pm, feat) - target / p["out_scale"]) ** 2)
            gnum = (lp - lm) / (2 * h)
            gana = np.asarray(g[name]).reshape(-1)[idx] if name != "b3" else g["b3"]
            assert gana == pytest.approx(gnum, rel=1e-5, abs=1e-8), (name, idx)


def test_pair_force_is_symmetric_in_the_two_molecules():
    p = random_params(seed=6)
    feat = np.random.default_rng(7).normal(0, 1, (50, 9))
    sw = feat.copy()
    sw[:, 1:5], sw[:, 5:9] = feat[:, 5:9], feat[:, 1:5]
    m = oracle.OracleMLP(p)
    assert np.array_equal(m.pair_force(feat), m.pair_force(sw))
    y1, y2 = m.forward(feat), m.forward(sw)
    assert np.allclose(m.pair_force(feat), 0.5 * p["out_scale"] * (y1 + y2), rtol=1e-14)


def two_molecules(seed=0, dist=1.6):
    """Two tetrahedra near the middle of a large box, all atomistic, random orientations."""
    s = inputs.tetra_system(2, (30.0, 30.0, 30.0), 1e3, 1.0)
    rng = np.random.default_rng(seed)
    body = inputs.tetra_sites()
    rot = inputs.random_rotations(rng, 2)
    c = np.array([[15.0, 15.0, 15.0], [15.0 + dist, 15.2, 14.9]])
    x = np.concatenate([c[0] + body @ rot[0].T, c[1] + body @ rot[1].T])
    return s, x, rot


def test_target_is_the_total_intermolecular_force_along_the_axis():
    for seed in range(5):
        s, x, _ = two_molecules(seed)
        o = oracle.Oracle(s)
        feat, t = o.pair_features(x, 0, 1)
        f, _ = o.forces(x)  # bonded forces cancel inside each molecule
        R = x.reshape(2, 4, 3).mean(1)
        e = (R[1] - R[0]) / np.linalg.norm(R[1] - R[0])
        assert feat[0] == pytest.approx(np.linalg.norm(R[1] - R[0]), rel=1e-14)
        assert t == pytest.approx(-(f[:4].sum(0) @ e), rel=1e-10, abs=1e-10)
        _, t_ba = o.pair_features(x, 1, 0)
        assert t_ba == pytest.approx(t, rel=1e-12, abs=1e-12)
    assert any(oracle.Oracle(two_molecules(k, 1.4)[0]).pair_features(two_molecules(k, 1.4)[1], 0, 1)[1] != 0
               for k in range(5))


def test_features_are_invariant_under_rotation_permutation_and_exchange():
    s, x, _ = two_molecules(11)
    o = oracle.Oracle(s)
    feat, t = o.pair_features(x, 0, 1)
    # rigid rotation about the box centre
    Q = inputs.random_rotations(np.random.default_rng(12), 1)[0]
    xr = (x - 15.0) @ Q.T + 15.0
    fr, tr = o.pair_features(xr, 0, 1)
    assert np.allclose(fr, feat, atol=1e-12) and tr == pytest.approx(t, rel=1e-12)
    # permuting the atoms inside a molecule
    xp = x.copy()
    xp[:4] = x[[2, 0, 3, 1]]
    fp, _ = o.pair_features(xp, 0, 1)
    assert np.allclose(fp, feat, atol=1e-14)
    # exchanging the two molecules swaps the two halves
    fe, _ = o.pair_features(x, 1, 0)
    assert fe[0] == feat[0] and np.allclose(fe[1:5], feat[5:9]) and np.allclose(fe[5:9], feat[1:5])
    # projections are sorted and bounded by the atom-to-COM distances
    assert np.all(np.diff(feat[1:5]) >= 0) and np.all(np.abs(feat[1:]) <= 0.6)


def test_collect_pairs_matches_pairwise_definition():
    s = inputs.tetra_system(64, (17.2, 6.45, 6.45), 3.0, 2.0, seed=13)
    x, _ = inputs.tetra_state(s)
    o = oracle.Oracle(s)
    feat, t, ids = o.collect_pairs(x, 2.3)
    R, _, _ = o.com_lambda(x)
    L = np.array(s.box)
    d = R[:, None] - R[None]
    d -= L * np.rint(d / L)
    r = np.sqrt((d ** 2).sum(-1))
    expect = {(a, b) for a in range(s.M) for b in range(a + 1, s.M) if r[a, b] < 2.3}
    assert {tuple(map(int, p)) for p in ids} == expect
    for k in range(0, len(ids), 17):
        f1, t1 = o.pair_features(x, *ids[k])
        assert np.array_equal(f1, feat[k]) and t1 == t[k]


def test_forces_with_learned_cg_force_all_cg_reduce_to_pair_sums_and_conserve_momentum():
    """lambda = 0 everywhere: the total force on each molecule is the sum over partners of
    the symmetrised network force along the COM axis (bonded terms cancel in the sum)."""
    s = inputs.tetra_system(64, (17.2, 6.45, 6.45), 0.0, 0.0, seed=14)
    x, _ = inputs.tetra_state(s)
    o = oracle.Oracle(s)
    net = oracle.OracleMLP(random_params(seed=15, scale=0.2))
    o.set_mlp(net)
    f, e = o.forces(x)
    assert e["E_cg"] == 0.0
    assert np.abs(f.sum(0)).max() <= 1e-12 * np.abs(f).sum()
    feat, _, ids = o.collect_pairs(x, s.rc_cg)
    fp = net.pair_force(feat)
    R, _, _ = o.com_lambda(x)
    L = np.array(s.box)
    Fm = np.zeros((s.M, 3))
    for (a, b), fab in zip(ids, fp):
        d = R[a] - R[b]
        d -= L * np.rint(d / L)
        u = d / np.linalg.norm(d)
        Fm[a] += fab * u
        Fm[b] -= fab * u
    assert np.allclose(f.reshape(s.M, 4, 3).sum(1), Fm, rtol=1e-9, atol=1e-9 * np.abs(Fm).max())
    o.set_mlp(None)
    f_tab, e_tab = o.forces(x)
    assert e_tab["E_cg"] != 0.0 and not np.allclose(f_tab, f)
