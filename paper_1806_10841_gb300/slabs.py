"""Spatial slab decomposition of the AdResS step across ranks (one GPU per rank).

The paper's code scales by spatial domain decomposition with halo exchange over a linked-cell
list, and balances the unequal cost of atomistic and coarse-grained regions with non-uniform
domains (Sec. "Heterogeneous Spatial Domain Decomposition Algorithm").  Here the box is cut
into slabs along x (the slab geometry's resolution axis):

* ``balance_bounds`` places the slab boundaries so that every rank gets the same estimated
  cost, the cost of a molecule depending on its resolution class (atomistic, hybrid,
  coarse-grained) with per-class costs measured on the GPU; narrow slabs where the
  expensive atomistic region is, wide ones in the cheap coarse-grained region.
* ``SlabDecomposition`` owns one rank's part of a step.  Every molecule belongs to the
  rank whose slab holds its centre of mass.  A rank needs as ghosts the molecules within
  the halo width (the neighbour-list cutoff) beyond its faces.  Two ways of exchanging:

  - ``half_shell`` (the communication-saving one): a rank receives ghosts from the rank
    above only and computes every pair with at least one of its own molecules; the forces
    its ghosts received are sent back to their owner and added there (reverse force
    accumulation), so each pair is computed once;
  - ``full_shell``: ghosts from both sides, every rank computes all pairs of its own
    molecules with any neighbour, nothing goes back (each cross-boundary pair is computed on
    both ranks).

  Positions, velocities and forces move with their molecules when a centre crosses a
  boundary (``migrate``).

The local force evaluation is injected (``engine``): it receives the local molecules'
positions and an owned mask and returns forces for every local molecule.  For the half shell
the ghost rows must hold only the pair forces from owned molecules (bonded, thermodynamic and
ghost-ghost terms excluded); for the full shell only the owned rows are used.  Communication
is plain ``torch.distributed`` point-to-point messages of host tensors (gloo) or device tensors
(NCCL), never a collective on the data path beyond the halo and force messages.

Molecule ids are global; within a rank the local order is owned molecules (ascending id)
followed by ghosts (ascending id), so every list is deterministic.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

CLASS_AT, CLASS_HY, CLASS_CG = 0, 1, 2


def com_x(x, na: int, mass, L: float):
    """x component of every molecule's centre of mass (minimum-image unwrap relative to its
    first atom, wrapped into [0, L)); x: (N, 3) or (N,) x coordinates."""
    xs = np.asarray(x, dtype=np.float64)
    xs = xs[:, 0] if xs.ndim == 2 else xs
    xm = xs.reshape(-1, na)
    d = xm - xm[:, :1]
    d -= L * np.rint(d / L)
    m = np.asarray(mass, dtype=np.float64)
    r = xm[:, 0] + (d * m[None, :]).sum(1) / m.sum()
    r -= L * np.floor(r / L)
    return np.where(r >= L, r - L, r)


def resolution_class(cx, L: float, x_center: float, d_at: float, d_hy: float):
    """AT / hybrid / CG class of molecules from their centre x (slab geometry)."""
    d = cx - x_center
    d -= L * np.rint(d / L)
    d = np.abs(d)
    return np.where(d < d_at, CLASS_AT, np.where(d < d_at + d_hy, CLASS_HY, CLASS_CG)).astype(np.int8)


def balance_bounds(cx, cls, L: float, n_ranks: int, cost, min_width: float, nbins: int = 4096):
    """Slab boundaries b_0 = 0 < b_1 < ... < b_n = L with equal estimated cost per slab.

    The cost density along x is the sum of cost[class] over the molecules of each of nbins
    bins; boundary k is where the cumulative cost reaches k/n of the total (linear within a
    bin).  Slabs narrower than min_width (the halo width: ghosts must come from the next
    rank only) are widened by moving their upper boundary, in order, and the last slab keeps
    what remains (ValueError if that is narrower than min_width)."""
    if n_ranks < 1:
        raise ValueError("n_ranks >= 1")
    if n_ranks * min_width > L:
        raise ValueError("the box is too short for that many slabs of the halo width")
    cost = np.asarray(cost, dtype=np.float64)
    h = L / nbins
    j = np.minimum((np.asarray(cx) / h).astype(np.int64), nbins - 1)
    dens = np.bincount(j, weights=cost[np.asarray(cls, dtype=np.int64)], minlength=nbins)
    cum = np.concatenate([[0.0], np.cumsum(dens)])
    total = cum[-1]
    b = np.zeros(n_ranks + 1)
    b[-1] = L
    for k in range(1, n_ranks):
        target = total * k / n_ranks
        i = int(np.searchsorted(cum, target, side="left"))
        i = min(max(i, 1), nbins)
        lo, hi = cum[i - 1], cum[i]
        frac = 0.0 if hi <= lo else (target - lo) / (hi - lo)
        b[k] = (i - 1 + frac) * h
    for k in range(1, n_ranks):
        if b[k] - b[k - 1] < min_width:
            b[k] = b[k - 1] + min_width
    for k in range(n_ranks - 1, 0, -1):
        if b[k + 1] - b[k] < min_width:
            b[k] = b[k + 1] - min_width
    if np.any(np.diff(b) < min_width * (1 - 1e-12)):
        raise ValueError("no slab layout with every slab at least the halo width")
    return b


def owner_of(cx, bounds):
    """Rank owning each molecule: the slab [b_k, b_{k+1}) holding its centre's x."""
    r = np.searchsorted(bounds, cx, side="right") - 1
    return np.clip(r, 0, len(bounds) - 2).astype(np.int64)


def in_band(cx, lo: float, width: float, L: float):
    """Molecules whose centre x lies in [lo, lo + width) (periodic)."""
    d = (np.asarray(cx) - lo) % L
    return d < width


@dataclass
class Local:
    """One rank's molecules: ids (owned first, then ghosts, each ascending) and how many are
    owned."""
    ids: np.ndarray
    n_owned: int


class SlabDecomposition:
    """One rank's view of the decomposition (see the module docstring).

    system: the single-system description of the whole box (its M, na, mass, box, slab
    geometry); bounds: slab boundaries (``balance_bounds``); halo: ghost band width (at
    least the neighbour-list cutoff of the force engine); mode: "half_shell" or
    "full_shell"; group: a torch.distributed process group (or None for the default)."""

    def __init__(self, system, bounds, halo: float, mode: str = "half_shell", group=None):
        import torch.distributed as dist

        if mode not in ("half_shell", "full_shell"):
            raise ValueError(mode)
        self.s = system
        self.dist = dist
        self.group = group
        self.rank = dist.get_rank(group)
        self.n = dist.get_world_size(group)
        self.bounds = np.asarray(bounds, dtype=np.float64)
        if len(self.bounds) != self.n + 1:
            raise ValueError("one slab per rank")
        self.L = float(system.box[0])
        self.halo = float(halo)
        if np.any(np.diff(self.bounds) < self.halo * (1 - 1e-12)):
            raise ValueError("every slab must be at least the halo width")
        self.mode = mode
        self.na = int(system.na)
        self.mass = np.asarray(system.mass, dtype=np.float64)

    # -- geometry ---------------------------------------------------------------------------
    def ghost_bands(self, rank: int):
        """(lo, width) bands of centre x a rank needs as ghosts: above its upper face (both
        modes) and below its lower face (full shell only)."""
        lo, hi = self.bounds[rank], self.bounds[rank + 1]
        bands = [(hi % self.L, self.halo)]
        if self.mode == "full_shell":
            bands.append(((lo - self.halo) % self.L, self.halo))
        return bands

    def needed_by(self, rank: int, cx, ids):
        """Which of the molecules (ids, centres cx) lie in a ghost band of `rank` and are not
        owned by it (a molecule can be a ghost of a rank once, even if two bands cover it)."""
        sel = np.zeros(len(ids), dtype=bool)
        for lo, w in self.ghost_bands(rank):
            sel |= in_band(cx, lo, w, self.L)
        own = owner_of(cx, self.bounds) == rank
        return sel & ~own

    # -- messages ----------------------------------------------------------------------------
    def _exchange(self, send: dict, dtype):
        """Point-to-point exchange: send[r] = 2-D float64 array for rank r (r != self); returns
        recv[r] from every rank that sent (sizes first, then payloads)."""
        import torch

        dist = self.dist
        me = self.rank
        reqs, sizes_out = [], {}
        for r in range(self.n):
            if r == me:
                continue
            a = send.get(r, np.zeros((0, 1)))
            sizes_out[r] = torch.tensor([a.shape[0], a.shape[1] if a.ndim == 2 else 1], dtype=torch.int64)
            reqs.append(dist.isend(sizes_out[r], dst=r, group=self.group))
        sizes_in = {}
        for r in range(self.n):
            if r == me:
                continue
            t = torch.zeros(2, dtype=torch.int64)
            dist.recv(t, src=r, group=self.group)
            sizes_in[r] = (int(t[0]), int(t[1]))
        for q in reqs:
            q.wait()
        reqs, keep = [], []
        for r in range(self.n):
            if r == me:
                continue
            a = np.ascontiguousarray(send.get(r, np.zeros((0, 1))), dtype=dtype)
            if a.size:
                ta = torch.from_numpy(a.reshape(a.shape[0], -1).copy())
                keep.append(ta)
                reqs.append(dist.isend(ta, dst=r, group=self.group))
        recv = {}
        for r in range(self.n):
            if r == me:
                continue
            n0, n1 = sizes_in[r]
            if n0 == 0:
                recv[r] = np.zeros((0, n1), dtype=dtype)
                continue
            t = torch.zeros((n0, n1), dtype=torch.float64 if dtype == np.float64 else torch.int64)
            dist.recv(t, src=r, group=self.group)
            recv[r] = t.numpy()
        for q in reqs:
            q.wait()
        return recv

    # -- a force evaluation ---------------------------------------------------------------------
    def forces(self, owned_ids, x_owned, engine):
        """Forces on this rank's molecules.

        owned_ids: ascending global ids of the owned molecules; x_owned: (len * na, 3) their
        atom positions.  Sends this rank's molecules that other ranks need as ghosts, receives
        its own ghosts, evaluates ``engine(x_local, owned_mask)`` on owned + ghosts, and in the
        half shell sends the ghost rows back to their owners and adds the rows it receives.
        Returns (forces of the owned atoms, Local)."""
        na = self.na
        owned_ids = np.asarray(owned_ids, dtype=np.int64)
        x_owned = np.asarray(x_owned, dtype=np.float64).reshape(-1, 3)
        cx = com_x(x_owned, na, self.mass, self.L)
        send = {}
        for r in range(self.n):
            if r == self.rank:
                continue
            sel = self.needed_by(r, cx, owned_ids)
            if sel.any():
                rows = np.concatenate([owned_ids[sel][:, None].astype(np.float64),
                                       x_owned.reshape(-1, na * 3)[sel]], axis=1)
                send[r] = rows
        recv = self._exchange(send, np.float64)
        g_ids = [owned_ids[:0]]
        g_x = [np.zeros((0, na * 3))]
        for r in sorted(recv):
            if len(recv[r]):
                g_ids.append(recv[r][:, 0].astype(np.int64))
                g_x.append(recv[r][:, 1:])
        g_ids = np.concatenate(g_ids)
        g_x = np.concatenate(g_x)
        order = np.argsort(g_ids, kind="stable")
        g_ids, g_x = g_ids[order], g_x[order]
        ids = np.concatenate([owned_ids, g_ids])
        x_local = np.concatenate([x_owned.reshape(-1, na * 3), g_x]).reshape(-1, 3)
        mask = np.zeros(len(ids), dtype=bool)
        mask[:len(owned_ids)] = True
        f = np.asarray(engine(x_local, mask), dtype=np.float64).reshape(len(ids), na * 3)
        f_owned = f[:len(owned_ids)].copy()
        if self.mode == "half_shell":
            # reverse force accumulation: ghost rows back to their owners
            g_owner = owner_of(com_x(g_x.reshape(-1, 3), na, self.mass, self.L), self.bounds) if len(g_ids) else g_ids
            back = {}
            for r in range(self.n):
                if r == self.rank:
                    continue
                sel = g_owner == r
                if sel.any():
                    back[r] = np.concatenate([g_ids[sel][:, None].astype(np.float64), f[len(owned_ids):][sel]], axis=1)
            got = self._exchange(back, np.float64)
            pos = {int(a): k for k, a in enumerate(owned_ids)}
            for r in sorted(got):
                for row in got[r]:
                    f_owned[pos[int(row[0])]] += row[1:]
        return f_owned.reshape(-1, 3), Local(ids=ids, n_owned=len(owned_ids))

    # -- migration -------------------------------------------------------------------------------
    def migrate(self, owned_ids, *arrays):
        """Hand molecules whose centre left this rank's slab to their new owner.  arrays:
        per-atom (len * na, 3) arrays of the owned molecules (positions first).  Returns the
        new ascending owned ids and the arrays in that order."""
        na = self.na
        owned_ids = np.asarray(owned_ids, dtype=np.int64)
        rows = [np.asarray(a, dtype=np.float64).reshape(-1, na * 3) for a in arrays]
        cx = com_x(rows[0].reshape(-1, 3), na, self.mass, self.L)
        dest = owner_of(cx, self.bounds)
        send = {}
        for r in range(self.n):
            if r == self.rank:
                continue
            sel = dest == r
            if sel.any():
                send[r] = np.concatenate([owned_ids[sel][:, None].astype(np.float64)] + [a[sel] for a in rows], axis=1)
        got = self._exchange(send, np.float64)
        keep = dest == self.rank
        ids = [owned_ids[keep]]
        parts = [[a[keep]] for a in rows]
        for r in sorted(got):
            if len(got[r]):
                ids.append(got[r][:, 0].astype(np.int64))
                for k in range(len(rows)):
                    parts[k].append(got[r][:, 1 + k * na * 3:1 + (k + 1) * na * 3])
        ids = np.concatenate(ids)
        order = np.argsort(ids, kind="stable")
        out = [np.concatenate(p)[order].reshape(-1, 3) for p in parts]
        return ids[order], out


class LibraryEngine:
    """Local force engine on the GPU through the library: the rank's molecules (owned, then
    ghosts) as one system in the global box (the resolution geometry and thermodynamic force
    are those of the whole box), conservative forces from adress_compute_forces.  A handle is
    kept per local molecule count (the two most recent).  Half shell: the forces of owned +
    ghosts and of the ghosts alone; the ghost rows are their difference, i.e. the pair forces
    the ghosts receive from owned molecules."""

    def __init__(self, system, mode: str = "half_shell", precision: str = "fp32", device: str = "cuda:0"):
        if mode not in ("half_shell", "full_shell"):
            raise ValueError(mode)
        self.s, self.mode, self.precision, self.device = system, mode, precision, device
        self.na = int(system.na)
        self._handles = {}

    def _sim(self, m: int):
        import copy

        from . import adress

        sim = self._handles.pop(m, None)
        if sim is None:
            sub = copy.copy(self.s)
            sub.M = int(m)
            sim = adress.AdResS(sub, precision=self.precision, device=self.device)
        self._handles[m] = sim
        while len(self._handles) > 2:
            old = next(iter(self._handles))
            self._handles.pop(old).close()
        return sim

    def _forces(self, x):
        sim = self._sim(len(x) // self.na)
        sim.set_state(x)
        f, _ = sim.forces()
        sim.check()
        return f

    def __call__(self, x_local, owned):
        m = len(owned)
        na = self.na
        out = self._forces(np.asarray(x_local, dtype=np.float64)).reshape(m, na * 3)
        g = ~np.asarray(owned, dtype=bool)
        if self.mode == "half_shell" and g.sum() >= 2:
            xg = np.asarray(x_local, dtype=np.float64).reshape(m, na, 3)[g].reshape(-1, 3)
            out[g] -= self._forces(xg).reshape(-1, na * 3)
        elif self.mode == "half_shell" and g.any():
            raise ValueError("a half-shell ghost band needs at least two molecules")
        return out.reshape(-1, 3)

    def close(self):
        for sim in self._handles.values():
            sim.close()
        self._handles.clear()


def measure_class_costs(system, molecules: int = 20000, precision: str = "fp32", device: str = "cuda:0"):
    """Per-molecule cost (ms) of the fused step kernel for high-resolution and for
    coarse-grained molecules, measured on the GPU: the same fluid at `molecules` molecules,
    once all atomistic and once all coarse-grained (adress_time_kernels); returns the
    per-class cost vector for balance_bounds."""
    import copy

    from . import adress, inputs

    out = []
    for d_at, d_hy in ((1e4, 0.0), (0.0, 0.0)):
        s = inputs.scaled_c2(molecules, seed=int(system.seed))
        s = copy.copy(s)
        s.d_at, s.d_hy = d_at, d_hy
        x, v = inputs.tetra_state(s)
        sim = adress.AdResS(s, precision=precision, device=device)
        sim.set_state(x, v)
        sim.compute_forces(energies=False)
        ms = sim.time_kernels(reps=10)["step"]
        sim.close()
        out.append(ms / s.M)
    return cost_per_class(out[0], out[1])


def cost_per_class(ms_hr_item: float, ms_cg_item: float):
    """Per-class molecule cost for balance_bounds from measured per-item times (hybrid
    molecules cost as much as atomistic ones: both run the high-resolution loop)."""
    return np.array([ms_hr_item, ms_hr_item, ms_cg_item], dtype=np.float64)


def halo_width(system) -> float:
    """Neighbour cutoff between molecule centres of the force model: max(rc_cg, rc_at +
    2 r_ext) (the list cutoff without its skin; forces are exact with this halo)."""
    return max(float(system.rc_cg), float(system.rc_at) + 2.0 * float(system.r_ext))


def slab_count_limit(system) -> int:
    return int(math.floor(float(system.box[0]) / halo_width(system)))
