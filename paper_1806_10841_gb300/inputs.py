"""Seeded synthetic inputs for the tetrahedral AdResS fluid and the water-like fluid.

This module only *builds inputs*: the molecular geometry, the initial lattice with
jitter, Maxwell-Boltzmann velocities, the tabulated coarse-grained (CG) pair potential
and the run parameters.  It contains none of the method's arithmetic (no centre-of-mass
mapping, no resolution function, no force interpolation, no integration).  Both the
CUDA path and the FP64 oracle receive the arrays produced here.

Workload shapes (sizes, densities, slab widths, interaction constants) follow the
tetrahedral-fluid configurations that accompany the paper's force-interpolation
scheme (Sec. "Force interpolation", Eq. 1): four atoms per molecule, all six
intramolecular pairs bonded by FENE, WCA between atoms of different molecules, a
tabulated Lennard-Jones-like COM-COM potential for the CG model, a slab-shaped
atomistic region with hybrid layers on both sides, and a Langevin thermostat.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

WCA_RC = 2.0 ** (1.0 / 6.0)


@dataclasses.dataclass
class System:
    """Static description of one AdResS system (molecules of identical topology).

    Layout conventions: atoms of molecule ``a`` are ``a*na .. a*na+na-1``;
    positions/velocities are returned by the generators as ``(N, 3)`` float64.
    """

    M: int                      # molecules
    na: int                     # atoms per molecule
    box: tuple                  # (Lx, Ly, Lz)
    mass: np.ndarray            # (na,) per-site masses
    bonds: np.ndarray           # (nb, 2) int32 local atom indices
    xc: float                   # slab centre (x)
    d_at: float                 # atomistic half-width
    d_hy: float                 # hybrid-layer width (each side)
    eps: float = 1.0            # WCA epsilon
    sigma: float = 1.0          # WCA sigma
    rc_at: float = WCA_RC       # atomistic cutoff
    fene_k: float = 30.0
    fene_r0: float = 1.5
    intra_wca: int = 1          # WCA also on bonded intramolecular pairs
    cg_F: np.ndarray = None     # CG force table, F(r_k), k = 0..cg_n (positive = repulsive)
    cg_V: np.ndarray = None     # CG energy table
    cg_dr: float = 0.001
    rc_cg: float = 2.3
    tf: np.ndarray = None       # thermodynamic-force table on nodes d_k = k * tf_dx
    tf_dx: float = 0.5
    kT: float = 1.0
    gamma: float = 0.5
    dt: float = 0.005
    seed: int = 20180628
    skin: float = 0.3
    r_ext: float = 0.75         # bound on atom-to-COM distance used for list cutoffs
    # water-like molecules: nb_model 1 = Lennard-Jones (per-site eps/sigma, Lorentz-Berthelot)
    # + reaction-field Coulomb between atoms of different molecules, cutoff rc_at;
    # bond_model 1 = harmonic bonds (bond_k, bond_r0); harmonic angles
    nb_model: int = 0
    charge: np.ndarray = None   # (na,) site charges (e)
    lj_eps: np.ndarray = None   # (na,) site LJ epsilon
    lj_sig: np.ndarray = None   # (na,) site LJ sigma
    coulomb_f: float = 0.0      # 1/(4 pi eps0) in the model's units
    eps_rf: float = 1.0         # reaction-field dielectric constant
    bond_model: int = 0
    bond_k: float = 0.0
    bond_r0: float = 0.0
    angles: np.ndarray = None   # (n_angles, 3) int32 local indices (i, vertex, k)
    angle_k: float = 0.0
    angle_theta0: float = 0.0
    # self-adjusting geometry: resolution centres (n, 3); the AT region is the union of
    # spheres of radius d_at around them and the hybrid shells have width d_hy (None: slab)
    centers: np.ndarray = None
    # 0: force interpolation (Eq. 1); 1: energy interpolation (H-AdResS, Eq. Hmix)
    scheme: int = 0
    # energy interpolation's free-energy correction dDF/dl at equidistant nodes on [0, 1]
    fec: np.ndarray = None
    # multiple time stepping: CG (slow) forces every respa_n inner steps of dt (1: off)
    respa_n: int = 1

    @property
    def N(self) -> int:
        return self.M * self.na

    @property
    def cg_n(self) -> int:
        return len(self.cg_F) - 1


def tetra_sites(edge: float = 0.97) -> np.ndarray:
    """Regular tetrahedron of the given edge, centred at the origin, shape (4, 3)."""
    v = np.array([[1, 1, 1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1]], dtype=np.float64)
    return v * (edge / (2.0 * math.sqrt(2.0)))


def tetra_bonds() -> np.ndarray:
    return np.array([[i, j] for i in range(4) for j in range(i + 1, 4)], dtype=np.int32)


def random_rotations(rng: np.random.Generator, n: int) -> np.ndarray:
    """Uniform random rotation matrices (n, 3, 3) from uniform unit quaternions (Shoemake)."""
    u1, u2, u3 = rng.random(n), rng.random(n), rng.random(n)
    a = np.sqrt(1.0 - u1)
    b = np.sqrt(u1)
    qx, qy = a * np.sin(2 * np.pi * u2), a * np.cos(2 * np.pi * u2)
    qz, qw = b * np.sin(2 * np.pi * u3), b * np.cos(2 * np.pi * u3)
    R = np.empty((n, 3, 3))
    R[:, 0, 0] = 1 - 2 * (qy * qy + qz * qz)
    R[:, 0, 1] = 2 * (qx * qy - qz * qw)
    R[:, 0, 2] = 2 * (qx * qz + qy * qw)
    R[:, 1, 0] = 2 * (qx * qy + qz * qw)
    R[:, 1, 1] = 1 - 2 * (qx * qx + qz * qz)
    R[:, 1, 2] = 2 * (qy * qz - qx * qw)
    R[:, 2, 0] = 2 * (qx * qz - qy * qw)
    R[:, 2, 1] = 2 * (qy * qz + qx * qw)
    R[:, 2, 2] = 1 - 2 * (qx * qx + qy * qy)
    return R


def lj_cg_table(eps: float = 1.0, sigma: float = 1.75, rc: float = 2.3, dr: float = 0.001,
                r_min: float = 0.5):
    """Tabulated Lennard-Jones-like COM-COM potential on r_k = k*dr, k = 0..rc/dr.

    The tabulated potential is force-shifted so that both F and V vanish at rc:
      F_s(r) = F(r) - F(rc),  V_s(r) = V(r) - V(rc) + (r - rc) F(rc),
    with F = -dV/dr (positive = repulsive).  Below r_min the force is held at
    F_s(r_min) and V continues linearly, so the table stays finite and consistent.
    Returns (F, V) float64 arrays of length n+1.
    """
    n = int(round(rc / dr))
    r = np.arange(n + 1, dtype=np.float64) * dr

    def V(x):
        s6 = (sigma / x) ** 6
        return 4 * eps * (s6 * s6 - s6)

    def F(x):
        s6 = (sigma / x) ** 6
        return 24 * eps * (2 * s6 * s6 - s6) / x

    Frc, Vrc = F(rc), V(rc)
    kmin = int(round(r_min / dr))
    rr = np.maximum(r, r_min)
    Ft = F(rr) - Frc
    Vt = V(rr) - Vrc + (rr - rc) * Frc
    below = r < r_min
    Vt[below] = Vt[kmin] + Ft[kmin] * (r_min - r[below])
    Ft[-1] = 0.0
    Vt[-1] = 0.0
    return Ft, Vt


def tetra_system(M: int, box, at_width: float, hy_width: float, *, tf_bins: int | None = None,
                 **kw) -> System:
    """Tetrahedral fluid: full AT width `at_width`, hybrid width `hy_width` on each side.

    The AT slab is centred at Lx/2, so d_at = at_width/2 and d_hy = hy_width.
    """
    box = tuple(float(b) for b in box)
    cg_kw = {k: kw.pop(k) for k in ("cg_eps", "cg_sigma") if k in kw}
    rc_cg = kw.get("rc_cg", 2.3)
    dr = kw.get("cg_dr", 0.001)
    F, V = lj_cg_table(cg_kw.get("cg_eps", 1.0), cg_kw.get("cg_sigma", 1.75), rc_cg, dr)
    tf_dx = kw.get("tf_dx", 0.5)
    d_at, d_hy = 0.5 * at_width, hy_width
    if tf_bins is None:
        tf_bins = int(math.ceil((d_at + d_hy) / tf_dx)) + 2
    s = System(M=M, na=4, box=box, mass=np.ones(4), bonds=tetra_bonds(), xc=0.5 * box[0],
               d_at=d_at, d_hy=d_hy, cg_F=F, cg_V=V, tf=np.zeros(tf_bins), **kw)
    return s


def _close_pairs(pos, occ, n, L, active, thr):
    """Molecule pairs on neighbouring lattice sites with some atom-atom distance below thr
    (only pairs touching an `active` molecule are checked).  Returns (a, b) index arrays."""
    idx = np.argwhere(occ >= 0)
    a_all = occ[tuple(idx.T)]
    sel = active[a_all]
    idx, a_all = idx[sel], a_all[sel]
    out_a, out_b = [], []
    offs = [(i, j, k) for i in (-1, 0, 1) for j in (-1, 0, 1) for k in (-1, 0, 1) if (i, j, k) != (0, 0, 0)]
    for o in offs:
        nb = (idx + np.array(o)) % n
        b = occ[tuple(nb.T)]
        ok = (b >= 0) & (b != a_all)
        a, bb = a_all[ok], b[ok]
        if len(a) == 0:
            continue
        d = pos[a][:, :, None, :] - pos[bb][:, None, :, :]
        d -= L * np.rint(d / L)
        r = np.sqrt((d * d).sum(-1)).reshape(len(a), -1).min(1)
        hit = r < thr
        out_a.append(a[hit])
        out_b.append(bb[hit])
    if not out_a:
        return np.zeros(0, np.int64), np.zeros(0, np.int64)
    return np.concatenate(out_a), np.concatenate(out_b)


def tetra_state(s: System, *, edge: float = 0.97, jitter: float = 0.1, seed: int | None = None,
                min_contact: float = 1.0, max_rounds: int = 200, body: np.ndarray | None = None):
    """Initial positions and velocities, both (N, 3) float64.

    Molecule centres sit on a simple-cubic lattice filling the box (M sites chosen at
    random among the lattice sites), each displaced by U(-jitter, jitter) per axis; each
    molecule is a regular tetrahedron under a uniform random rotation.  Orientations (and
    jitters) of molecules with an atom closer than `min_contact` to an atom of a
    neighbouring molecule are redrawn (the higher-index molecule of each close pair), up to
    `max_rounds` times (set min_contact=0 to
    keep the first draw, e.g. for over-dense literal configurations).  Velocities are
    Maxwell-Boltzmann at kT with the total momentum removed.  Positions are wrapped
    into [0, L).
    """
    rng = np.random.default_rng(s.seed if seed is None else seed)
    L = np.asarray(s.box)
    a = (np.prod(L) / s.M) ** (1.0 / 3.0)
    n = np.maximum(1, np.floor(L / a + 1e-9).astype(int))
    while np.prod(n) < s.M:  # grow the axis whose spacing is largest
        n[np.argmax(L / n)] += 1
    grid = np.stack(np.meshgrid(*[np.arange(k) for k in n], indexing="ij"), -1).reshape(-1, 3)
    pick = np.sort(rng.choice(len(grid), size=s.M, replace=False))
    site_idx = grid[pick]
    sites = (site_idx + 0.5) * (L / n)
    occ = -np.ones(tuple(n), dtype=np.int64)
    occ[tuple(site_idx.T)] = np.arange(s.M)
    if body is None:
        body = tetra_sites(edge) if s.na == 4 else np.zeros((s.na, 3))
    com = sites + rng.uniform(-jitter, jitter, size=(s.M, 3))
    pos = com[:, None, :] + np.einsum("mij,kj->mki", random_rotations(rng, s.M), body)
    if min_contact > 0 and s.M > 1:
        active = np.ones(s.M, dtype=bool)
        for _ in range(max_rounds):
            pa, pb = _close_pairs(pos, occ, n, L, active, min_contact)
            if len(pa) == 0:
                break
            # redraw only the higher-index molecule of each close pair (sequential-placement order)
            bad = np.zeros(s.M, dtype=bool)
            bad[np.maximum(pa, pb)] = True
            k = int(bad.sum())
            com[bad] = sites[bad] + rng.uniform(-jitter, jitter, size=(k, 3))
            pos[bad] = com[bad][:, None, :] + np.einsum("mij,kj->mki", random_rotations(rng, k), body)
            # re-check the redrawn molecules against all their neighbours
            active = bad
    x = np.mod(pos.reshape(-1, 3), L)
    x[x >= L] -= np.broadcast_to(L, x.shape)[x >= L]
    m = np.tile(s.mass, s.M)
    v = rng.normal(size=(s.N, 3)) * np.sqrt(s.kT / m)[:, None]
    v -= (m[:, None] * v).sum(0) / m.sum()
    return x, v


# --- named workloads ---------------------------------------------------------------

# --- water-like fluid (flexible three-site model, reaction-field electrostatics) -------
# Units: nm, ps, atomic mass units, kJ/mol, elementary charges.

WATER_MASS = np.array([15.9994, 1.008, 1.008])      # O, H, H
WATER_CHARGE = np.array([-0.8476, 0.4238, 0.4238])
WATER_R0 = 0.1                                      # O-H bond length (nm)
WATER_THETA0 = math.radians(109.47)                 # H-O-H angle
COULOMB_F = 138.935458                              # 1 / (4 pi eps0) in kJ mol^-1 nm e^-2
KB = 0.0083144626                                   # kJ mol^-1 K^-1


def water_sites() -> np.ndarray:
    """O and the two H of the equilibrium geometry, relative to the centre of mass (3, 3)."""
    h = 0.5 * WATER_THETA0
    x = np.array([[0.0, 0.0, 0.0],
                  [WATER_R0 * math.sin(h), WATER_R0 * math.cos(h), 0.0],
                  [-WATER_R0 * math.sin(h), WATER_R0 * math.cos(h), 0.0]])
    return x - (WATER_MASS[:, None] * x).sum(0) / WATER_MASS.sum()


def water_system(M: int, box, at_width: float, hy_width: float, *, tf_bins: int | None = None,
                 **kw) -> System:
    """Flexible three-site water-like fluid: O-H bonds harmonic (k = 345000 kJ mol^-1 nm^-2,
    r0 = 0.1 nm), H-O-H angle harmonic at 109.47 degrees (k_theta = 383 kJ mol^-1 rad^-2),
    Lennard-Jones on O (sigma = 0.3166 nm, eps = 0.65 kJ/mol) and reaction-field Coulomb
    (rc = 0.9 nm, eps_rf = 80) between atoms of different molecules; a tabulated single-bead
    COM potential for the CG model (placeholder Lennard-Jones-like table unless `cg_F`/`cg_V`
    are given); Langevin at 300 K (gamma = 5 / ps), dt = 0.5 fs.  Slab as in tetra_system."""
    box = tuple(float(b) for b in box)
    rc_cg = kw.pop("rc_cg", 0.9)
    dr = kw.pop("cg_dr", 0.0005)
    cg = {k: kw.pop(k) for k in ("cg_F", "cg_V") if k in kw}
    if not cg:
        F, V = lj_cg_table(0.65, 0.3166, rc_cg, dr, r_min=0.2)
        cg = dict(cg_F=F, cg_V=V)
    tf_dx = kw.pop("tf_dx", 0.05)
    d_at, d_hy = 0.5 * at_width, hy_width
    if tf_bins is None:
        tf_bins = int(math.ceil((d_at + d_hy) / tf_dx)) + 2
    params = dict(eps=0.0, sigma=1.0, rc_at=0.9, fene_k=0.0, fene_r0=1.0, intra_wca=0, cg_dr=dr, rc_cg=rc_cg,
                  tf_dx=tf_dx, kT=KB * 300.0, gamma=5.0, dt=0.0005, skin=0.1, r_ext=0.15,
                  nb_model=1, charge=WATER_CHARGE.copy(), lj_eps=np.array([0.65, 0.0, 0.0]),
                  lj_sig=np.array([0.3166, 0.0, 0.0]), coulomb_f=COULOMB_F, eps_rf=80.0,
                  bond_model=1, bond_k=345000.0, bond_r0=WATER_R0,
                  angles=np.array([[1, 0, 2]], dtype=np.int32), angle_k=383.0, angle_theta0=WATER_THETA0)
    params.update(kw)
    return System(M=M, na=3, box=box, mass=WATER_MASS.copy(), bonds=np.array([[0, 1], [0, 2]], dtype=np.int32),
                  xc=0.5 * box[0], d_at=d_at, d_hy=d_hy, tf=np.zeros(tf_bins), **cg, **params)


def water_state(s: System, *, seed: int | None = None, jitter: float = 0.01, min_contact: float = 0.17):
    """Initial state of the water-like fluid: molecules at lattice sites in random
    orientations (orientations redrawn until no atom of another molecule is closer than
    min_contact), Maxwell-Boltzmann velocities at kT."""
    return tetra_state(s, seed=seed, jitter=jitter, min_contact=min_contact, body=water_sites())


def c3_water(**kw) -> System:
    """64,000 water-like molecules (192,000 atoms) at 33.4 molecules/nm^3 in 19.72 x 9.86 x
    9.86 nm; AT width 3 nm, hybrid 1.5 nm each side."""
    return water_system(64_000, (19.72, 9.86, 9.86), 3.0, 1.5, **kw)


def scaled_c3(M: int, **kw) -> System:
    """The water workload's shape (33.4 molecules/nm^3, box 2:1:1, AT 15% / hybrid 2x7.6% of
    Lx) at M molecules."""
    Ly = (M / 33.4 / 2.0) ** (1.0 / 3.0)
    Lx = 2 * Ly
    return water_system(M, (Lx, Ly, Ly), 3.0 / 19.72 * Lx, 1.5 / 19.72 * Lx, **kw)


def c1_literal(**kw) -> System:
    """1000 tetrahedra (4000 atoms) in a 20x10x10 box, AT width 5, hybrid 2.5 (density 0.5/sigma^3)."""
    return tetra_system(1000, (20.0, 10.0, 10.0), 5.0, 2.5, **kw)


def c1_stable(**kw) -> System:
    """The same 1000 tetrahedra at 0.1 molecules/sigma^3 (box 34.20 x 17.10 x 17.10)."""
    return tetra_system(1000, (34.20, 17.10, 17.10), 5.0, 2.5, **kw)


def c2_800k(**kw) -> System:
    """200k tetrahedra (800k atoms) in 200x100x100, AT width 40, hybrid 10 (density 0.1)."""
    return tetra_system(200_000, (200.0, 100.0, 100.0), 40.0, 10.0, **kw)


def scaled_c2(M: int, **kw) -> System:
    """The 800k-atom fluid's shape (density 0.1, box 2:1:1, AT 20% / hybrid 2x5% of Lx) at M molecules."""
    Ly = (M / 0.1 / 2.0) ** (1.0 / 3.0)
    Lx = 2 * Ly
    return tetra_system(M, (Lx, Ly, Ly), 0.2 * Lx, 0.05 * Lx, **kw)


def replica_batch(n: int = 64, *, m_lo: int = 500, m_hi: int = 20000, seed: int = 20180628, **kw):
    """Independent replicas of the tetrahedral fluid: M_r = exp(U(ln m_lo, ln m_hi)) molecules
    in a (2a, a, a) box with a = (M_r / 0.2)^(1/3) (density 0.1), full AT width U(3, 15) and
    hybrid width U(1, 5).  The replicas share every model parameter (including the
    thermostat seed and a common thermodynamic-force grid); initial states come from
    replica_states with seed + r."""
    rng = np.random.default_rng(seed)
    ms = np.exp(rng.uniform(math.log(m_lo), math.log(m_hi), n)).astype(int)
    at = rng.uniform(3.0, 15.0, n)
    hy = rng.uniform(1.0, 5.0, n)
    tf_dx = kw.get("tf_dx", 0.5)
    bins = int(math.ceil(max(0.5 * a + h for a, h in zip(at, hy)) / tf_dx)) + 2
    out = []
    for M, w_at, w_hy in zip(ms, at, hy):
        a = (M / 0.2) ** (1.0 / 3.0)
        out.append(tetra_system(int(M), (2 * a, a, a), float(w_at), float(w_hy), tf_bins=bins, seed=seed, **kw))
    return out


def replica_states(systems, seed: int = 20180628):
    """Initial (x, v) of each replica (tetra_state with seed + r), concatenated in order."""
    xs, vs = [], []
    for r, s in enumerate(systems):
        x, v = tetra_state(s, seed=seed + r)
        xs.append(x)
        vs.append(v)
    return np.concatenate(xs), np.concatenate(vs)
