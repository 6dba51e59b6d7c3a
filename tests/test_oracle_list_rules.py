"""The list rules of the CUDA path, checked against the oracle's own dynamics (CPU).

At a list build the library classifies work items (high-resolution when |dxc| < d_at + d_hy
+ skin/2), lists a pair within r_list = max(rc_cg, rc_at + 2 r_ext) + skin when both are
high-resolution items and within rc_cg + skin otherwise, and (network mode) records as
candidates the pairs within rc_cg + skin that are not made of two deep-atomistic molecules
(|dxc| < d_at - skin/2).  Until the next build (triggered once a centre has moved more than
skin/2) these must cover every interaction of Eq. 1: here the oracle runs the Langevin
dynamics of a hybrid box step by step, and at every step before the rebuild condition each
pair that needs a CG force (centres within rc_cg, weight below 1) is listed and is a
candidate, and each pair that can need atomistic forces (weight above 0, centres within
rc_at + 2 * the largest atom-to-centre distance) is listed.  The premises are checked too:
coarse-grained items keep weight 0, deep-atomistic molecules weight 1.
"""
import numpy as np
import pytest

import oracle
from paper_1806_10841_gb300 import inputs


def pair_distances(R, L):
    d = R[:, None, :] - R[None, :, :]
    d -= L * np.rint(d / L)
    return np.sqrt((d ** 2).sum(-1))


def max_extent(o, x, R, L, na):
    off = x.reshape(-1, na, 3) - R[:, None, :]
    off -= L * np.rint(off / L)
    return float(np.sqrt((off ** 2).sum(-1)).max())


@pytest.mark.parametrize("seed", [1, 2, 3, 4])
def test_lists_and_candidates_cover_every_interaction_until_the_rebuild(seed):
    s = inputs.tetra_system(1000, (34.20, 17.10, 17.10), 5.0, 2.5)
    x, v = inputs.tetra_state(s, seed=seed)
    o = oracle.Oracle(s)
    L = np.array(s.box)
    f, _ = o.forces(x)
    R0, dxc0, _ = o.com_lambda(x)
    r_list = max(s.rc_cg, s.rc_at + 2 * s.r_ext) + s.skin
    r_cg_list = s.rc_cg + s.skin
    hr = np.abs(dxc0) < s.d_at + s.d_hy + 0.5 * s.skin
    deep = np.abs(dxc0) < s.d_at - 0.5 * s.skin - 1e-3
    assert hr.any() and (~hr).any() and deep.any()
    r0 = pair_distances(R0, L)
    off = ~np.eye(s.M, dtype=bool)
    listed = off & (r0 < np.where(hr[:, None] & hr[None, :], r_list, r_cg_list))
    cand = off & (r0 < r_cg_list) & ~(deep[:, None] & deep[None, :])
    assert (listed == listed.T).all() and (cand == cand.T).all()
    steps = 0
    for k in range(400):
        x, v, f = o.run(x, v, f, k, 1)
        R, dxc, w = o.com_lambda(x)
        disp = R - R0
        disp -= L * np.rint(disp / L)
        if np.sqrt((disp ** 2).sum(-1)).max() > 0.5 * s.skin:
            break  # the library rebuilds here
        steps += 1
        assert (w[~hr] == 0.0).all()
        assert (w[deep] == 1.0).all()
        r = pair_distances(R, L)
        wab = w[:, None] * w[None, :]
        need_cg = off & (r < s.rc_cg) & (wab < 1.0)
        assert (~need_cg | listed).all()
        assert (~need_cg | cand).all()
        reach = s.rc_at + 2.0 * max_extent(o, x, R, L, s.na)
        assert reach + 2 * 0.5 * s.skin <= r_list + 1e-12  # the extent rule of the rebuild decision
        need_at = off & (r < reach) & (wab > 0.0)
        assert (~need_at | listed).all()
    assert steps >= 10  # a real stretch of dynamics before the rebuild condition


def test_classification_margins_hold_for_any_move_below_half_the_skin():
    """A centre moves by less than skin/2 before the rebuild: a coarse-grained item (|dxc| at
    least d_at + d_hy + skin/2 at the build) keeps weight 0, a deep-atomistic molecule (|dxc|
    below d_at - skin/2) weight 1, whatever the move (the oracle's weight function)."""
    s = inputs.tetra_system(1000, (34.20, 17.10, 17.10), 5.0, 2.5)
    o = oracle.Oracle(s)
    half = 0.5 * s.skin
    moves = np.linspace(-half, half, 41)[1:-1]
    for d0 in np.linspace(0.0, s.d_at + s.d_hy + 2.0, 801):
        cg_item = not d0 < s.d_at + s.d_hy + half
        deep = d0 < s.d_at - half - 1e-3
        for dm in moves:
            w = o.weight(abs(d0 + dm))
            if cg_item:
                assert w == 0.0, (d0, dm)
            if deep:
                assert w == 1.0, (d0, dm)
