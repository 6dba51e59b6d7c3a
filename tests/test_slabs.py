"""Spatial slab decomposition (paper_1806_10841_gb300.slabs) on the CPU with gloo ranks:
slab boundaries balanced by resolution-class cost, ownership and ghost bands against their
plain definitions (bit for bit), and forces assembled from the ranks (half shell with
reverse force accumulation, and full shell) against a single-domain oracle evaluation of
the whole box.  The local force engine is the oracle on each rank's molecules."""
import copy
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def _case():
    from paper_1806_10841_gb300 import inputs

    s = inputs.scaled_c2(2000, seed=11)
    x, v = inputs.tetra_state(s)
    return s, x, v


def _sub(s, m):
    t = copy.copy(s)
    t.M = int(m)
    return t


def oracle_engine(s, mode):
    """Local forces from the oracle.  Half shell: the ghost rows keep only the pair forces
    from owned molecules (forces of owned + ghosts minus forces of the ghosts alone, which
    removes ghost-ghost pairs and the ghosts' own bonded and thermodynamic terms)."""
    import oracle

    na = s.na

    def engine(x_local, owned):
        m = len(owned)
        f_all, _ = oracle.Oracle(_sub(s, m)).forces(x_local)
        out = f_all.reshape(m, na * 3).copy()
        g = ~owned
        if mode == "half_shell" and g.any():
            xg = x_local.reshape(m, na, 3)[g].reshape(-1, 3)
            f_g, _ = oracle.Oracle(_sub(s, int(g.sum()))).forces(xg)
            out[g] -= f_g.reshape(-1, na * 3)
        return out.reshape(-1, 3)

    return engine


def _worker(rank, world, port, mode, q):
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist

    from paper_1806_10841_gb300 import slabs

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        s, x, v = _case()
        L = float(s.box[0])
        cx = slabs.com_x(x, s.na, s.mass, L)
        cls = slabs.resolution_class(cx, L, s.xc, s.d_at, s.d_hy)
        halo = slabs.halo_width(s)
        bounds = slabs.balance_bounds(cx, cls, L, world, slabs.cost_per_class(8.0, 1.0), halo)
        dec = slabs.SlabDecomposition(s, bounds, halo, mode=mode)
        owner = slabs.owner_of(cx, bounds)
        mine = np.nonzero(owner == rank)[0]
        xm = x.reshape(s.M, s.na, 3)
        f_own, loc = dec.forces(mine, xm[mine].reshape(-1, 3), oracle_engine(s, mode))
        # migration after a displacement that carries molecules across the boundaries
        shift = np.array([1.7, 0.0, 0.0])
        x2 = np.mod(xm[mine] + shift, s.box).reshape(-1, 3)
        v2 = v.reshape(s.M, s.na, 3)[mine].reshape(-1, 3)
        ids2, (x2n, v2n) = dec.migrate(mine, x2, v2)
        # gather to rank 0 (test plumbing)
        payload = dict(rank=rank, owned=mine, ghosts=loc.ids[loc.n_owned:], f=f_own, ids2=ids2, x2=x2n, v2=v2n,
                       bounds=bounds)
        out = [None] * world
        dist.all_gather_object(out, payload)
        if rank == 0:
            q.put(out)
    finally:
        dist.barrier()
        dist.destroy_process_group()


def _run(world, mode):
    import torch.multiprocessing as mp

    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, mode, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = q.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    return out


@pytest.mark.parametrize("world,mode", [(2, "half_shell"), (2, "full_shell"), (3, "half_shell")])
def test_decomposed_forces_equal_the_single_domain_oracle(world, mode):
    import oracle
    from paper_1806_10841_gb300 import slabs

    out = _run(world, mode)
    s, x, v = _case()
    L = float(s.box[0])
    cx = slabs.com_x(x, s.na, s.mass, L)
    bounds = out[0]["bounds"]
    halo = slabs.halo_width(s)
    # ownership: the slab holding the centre, every molecule exactly once
    owned = [o["owned"] for o in out]
    assert np.array_equal(np.sort(np.concatenate(owned)), np.arange(s.M))
    for r, o in enumerate(out):
        assert np.array_equal(o["owned"], np.nonzero((cx >= bounds[r]) & (cx < bounds[r + 1]))[0])
        # ghosts: the plain definition of the bands (centre x within the halo above the upper
        # face; full shell: and below the lower face), periodic, not owned
        up = (cx - bounds[r + 1]) % L < halo
        lo = (bounds[r] - cx) % L <= halo
        lo &= (bounds[r] - cx) % L > 0
        want = up | (lo if mode == "full_shell" else False)
        want &= ~((cx >= bounds[r]) & (cx < bounds[r + 1]))
        assert np.array_equal(o["ghosts"], np.nonzero(want)[0]), r
    # forces of every atom against the whole box evaluated at once
    f_ref, _ = oracle.Oracle(s).forces(x)
    f = np.zeros_like(f_ref)
    for o in out:
        f.reshape(s.M, s.na, 3)[o["owned"]] = o["f"].reshape(-1, s.na, 3)
    rel = np.sqrt(((f - f_ref) ** 2).sum() / (f_ref ** 2).sum())
    assert rel < 1e-12, rel
    # migration: after the shift every molecule sits on the rank owning its new centre, with
    # its own positions and velocities
    shift = np.array([1.7, 0.0, 0.0])
    x2 = np.mod(x + shift, s.box)
    cx2 = slabs.com_x(x2, s.na, s.mass, L)
    own2 = slabs.owner_of(cx2, bounds)
    allids = np.sort(np.concatenate([o["ids2"] for o in out]))
    assert np.array_equal(allids, np.arange(s.M))
    for r, o in enumerate(out):
        assert np.array_equal(o["ids2"], np.nonzero(own2 == r)[0])
        assert np.array_equal(o["x2"].reshape(-1, s.na, 3), x2.reshape(s.M, s.na, 3)[o["ids2"]])
        assert np.array_equal(o["v2"].reshape(-1, s.na, 3), v.reshape(s.M, s.na, 3)[o["ids2"]])


def test_balanced_bounds_follow_the_cost_density():
    """Equal estimated cost per slab: with atomistic molecules 8x the cost of coarse-grained
    ones the slabs over the atomistic region are narrower; the slab costs agree to the
    cost of the molecules within one bin; every slab is at least the halo width (with six
    slabs the ideal ones over the atomistic region would be narrower than the halo, so the
    width bound decides there)."""
    from paper_1806_10841_gb300 import slabs

    s, x, _ = _case()
    L = float(s.box[0])
    cx = slabs.com_x(x, s.na, s.mass, L)
    cls = slabs.resolution_class(cx, L, s.xc, s.d_at, s.d_hy)
    cost = slabs.cost_per_class(8.0, 1.0)
    b6 = slabs.balance_bounds(cx, cls, L, 6, cost, slabs.halo_width(s))
    assert np.all(np.diff(b6) >= slabs.halo_width(s) * (1 - 1e-12))
    assert np.isclose(np.diff(b6), slabs.halo_width(s)).any()
    for n in (2, 4):
        b = slabs.balance_bounds(cx, cls, L, n, cost, slabs.halo_width(s))
        assert b[0] == 0.0 and b[-1] == L and np.all(np.diff(b) >= slabs.halo_width(s))
        own = slabs.owner_of(cx, b)
        per = np.array([cost[cls[own == r]].sum() for r in range(n)])
        binw = L / 4096
        slack = cost.max() * (np.abs(cx[:, None] - b[None, 1:-1]) < binw).sum() + cost.max()
        assert per.max() - per.min() <= 2 * slack, (n, per)
    b4 = slabs.balance_bounds(cx, cls, L, 4, cost, slabs.halo_width(s))
    widths = np.diff(b4)
    # the slabs whose middle lies in the high-resolution band are narrower than the others
    mid = 0.5 * (b4[1:] + b4[:-1])
    hr = np.abs(mid - s.xc) < s.d_at + s.d_hy
    assert hr.any() and (~hr).any() and widths[hr].max() < widths[~hr].min()
    with pytest.raises(ValueError):
        slabs.balance_bounds(cx, cls, L, 100, cost, slabs.halo_width(s))


def test_owner_and_band_edges():
    from paper_1806_10841_gb300 import slabs

    b = np.array([0.0, 10.0, 25.0, 40.0])
    cx = np.array([0.0, 9.999, 10.0, 24.9, 25.0, 39.99])
    assert np.array_equal(slabs.owner_of(cx, b), [0, 0, 1, 1, 2, 2])
    assert np.array_equal(slabs.in_band(np.array([39.0, 1.0, 2.0]), 38.5, 3.0, 40.0), [True, True, False])
