"""FP64 CPU oracle for force-interpolation AdResS — TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference leg of
``bench.py`` may import this package.  The product path (the CUDA library and its
binding) never imports it and shares no code with it.

The arithmetic lives in ``adress_oracle.c`` (plain C, double precision), compiled
here with gcc into ``oracle/_build/libadress_oracle.so`` and called through ctypes.
Arrays are numpy float64 ``(N, 3)`` row-major.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "adress_oracle.c")
_HDR = os.path.join(_HERE, "adress_oracle.h")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libadress_oracle.so")

ORC_OK, ORC_ERR_BOND = 0, 1


class orc_mlp(C.Structure):
    _fields_ = [("nh", C.c_int), ("W1", C.POINTER(C.c_double)), ("b1", C.POINTER(C.c_double)),
                ("W2", C.POINTER(C.c_double)), ("b2", C.POINTER(C.c_double)), ("w3", C.POINTER(C.c_double)),
                ("b3", C.c_double), ("in_mean", C.POINTER(C.c_double)), ("in_std", C.POINTER(C.c_double)),
                ("out_scale", C.c_double), ("bf16", C.c_int)]


class orc_sys(C.Structure):
    _fields_ = [
        ("M", C.c_int), ("na", C.c_int),
        ("mass", C.POINTER(C.c_double)),
        ("L", C.c_double * 3),
        ("xc", C.c_double), ("d_at", C.c_double), ("d_hy", C.c_double),
        ("eps", C.c_double), ("sig", C.c_double), ("rc_at", C.c_double),
        ("nb", C.c_int), ("bonds", C.POINTER(C.c_int)),
        ("fene_k", C.c_double), ("fene_r0", C.c_double),
        ("intra_wca", C.c_int),
        ("cgF", C.POINTER(C.c_double)), ("cgV", C.POINTER(C.c_double)),
        ("cg_n", C.c_int), ("cg_dr", C.c_double), ("rc_cg", C.c_double),
        ("tf", C.POINTER(C.c_double)), ("tf_n", C.c_int), ("tf_dx", C.c_double),
        ("kT", C.c_double), ("gamma", C.c_double), ("dt", C.c_double),
        ("seed", C.c_uint64), ("replica", C.c_int64),
        ("mlp", C.POINTER(orc_mlp)),
        ("nb_model", C.c_int), ("charge", C.POINTER(C.c_double)), ("lj_eps", C.POINTER(C.c_double)),
        ("lj_sig", C.POINTER(C.c_double)), ("coulomb_f", C.c_double), ("eps_rf", C.c_double),
        ("bond_model", C.c_int), ("bond_k", C.c_double), ("bond_r0", C.c_double),
        ("n_angles", C.c_int), ("angles", C.POINTER(C.c_int)), ("angle_k", C.c_double),
        ("angle_theta0", C.c_double),
        ("n_centers", C.c_int), ("centers", C.POINTER(C.c_double)),
        ("scheme", C.c_int),
        ("fec_n", C.c_int), ("fec", C.POINTER(C.c_double)),
        ("lam_uniform_on", C.c_int), ("lam_uniform", C.c_double),
        ("respa_n", C.c_int),
    ]


def build(force: bool = False, extra_flags: tuple = ()) -> str:
    """Compile the oracle with gcc (plain C, -O2, no fast-math).  Returns the .so path."""
    out = _LIB if not extra_flags else os.path.join(
        _BUILD, "libadress_oracle_" + "_".join(f.strip("-").replace("=", "") for f in extra_flags) + ".so")
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if not force and os.path.exists(out) and os.path.getmtime(out) >= newest:
        return out
    os.makedirs(_BUILD, exist_ok=True)
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", *extra_flags,
           _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


_lib = None


def _load(path: str | None = None):
    global _lib
    if path is not None:
        lib = C.CDLL(path)
    else:
        if _lib is not None:
            return _lib
        lib = C.CDLL(build())
    d, i64, u64 = C.POINTER(C.c_double), C.POINTER(C.c_int64), C.POINTER(C.c_uint64)
    S = C.POINTER(orc_sys)
    u32 = C.POINTER(C.c_uint32)
    lib.orc_philox4x32.argtypes = [u32, u32, u32]
    lib.orc_uniform3.argtypes = [C.c_uint64, C.c_int64, C.c_int64, C.c_int64, d]
    lib.orc_weight.argtypes = [S, C.c_double]
    lib.orc_weight.restype = C.c_double
    lib.orc_com_lambda.argtypes = [S, d, d, d, d]
    lib.orc_forces.argtypes = [S, d, C.c_int, d, d, d]
    lib.orc_forces.restype = C.c_int
    lib.orc_run.argtypes = [S, d, d, d, C.c_int64, C.c_int, C.c_int]
    lib.orc_forces_step.argtypes = [S, d, C.c_int64, d, d]
    lib.orc_run.restype = C.c_int
    lib.orc_langevin_force.argtypes = [S, d, C.c_int64, d]
    lib.orc_kinetic.argtypes = [S, d, d]
    lib.orc_density.argtypes = [S, d, C.c_int, i64, C.c_int, i64]
    lib.orc_tf_update.argtypes = [S, d, C.c_int, i64, C.c_int, C.c_double, C.c_double]
    lib.orc_rdf.argtypes = [S, d, C.c_int, C.c_double, i64]
    lib.orc_bf16.argtypes = [C.c_double]
    lib.orc_bf16.restype = C.c_double
    lib.orc_pair_features.argtypes = [S, d, C.c_int, C.c_int, d, d]
    lib.orc_collect_pairs.argtypes = [S, d, C.c_double, C.c_long, d, d, C.POINTER(C.c_int)]
    lib.orc_collect_pairs.restype = C.c_long
    M = C.POINTER(orc_mlp)
    lib.orc_mlp_forward.argtypes = [M, C.c_long, d, d]
    lib.orc_mlp_pair_force.argtypes = [M, C.c_long, d, d]
    lib.orc_mlp_loss_grad.argtypes = [M, C.c_long, d, d, d, d, d, d, d, d]
    lib.orc_mlp_loss_grad.restype = C.c_double
    if path is None:
        _lib = lib
    return lib


def _ptr(a, ct=C.c_double):
    return a.ctypes.data_as(C.POINTER(ct)) if a is not None else None


class Oracle:
    """Holds one system description and exposes the oracle's functions on numpy arrays.

    `system` is any object with the fields M, na, box, mass, bonds, xc, d_at, d_hy, eps,
    sigma, rc_at, fene_k, fene_r0, intra_wca, cg_F, cg_V, cg_dr, rc_cg, tf, tf_dx, kT,
    gamma, dt and seed (the seeded input generator's system description).
    """

    def __init__(self, system, *, replica: int = 0, lib_path: str | None = None):
        s = system
        self.lib = _load(lib_path)
        self.M, self.na = int(s.M), int(s.na)
        self.N = self.M * self.na
        self._keep = dict(
            mass=np.ascontiguousarray(s.mass, dtype=np.float64),
            bonds=np.ascontiguousarray(np.asarray(s.bonds, dtype=np.int32).reshape(-1)),
            cgF=np.ascontiguousarray(s.cg_F, dtype=np.float64),
            cgV=np.ascontiguousarray(s.cg_V, dtype=np.float64),
            tf=np.ascontiguousarray(s.tf if s.tf is not None else np.zeros(0), dtype=np.float64),
        )
        nb_model = int(getattr(s, "nb_model", 0))
        zeros = np.zeros(self.na)
        self._keep.update(
            charge=np.ascontiguousarray(s.charge if nb_model else zeros, dtype=np.float64),
            lj_eps=np.ascontiguousarray(s.lj_eps if nb_model else zeros, dtype=np.float64),
            lj_sig=np.ascontiguousarray(s.lj_sig if nb_model else zeros, dtype=np.float64),
            angles=np.ascontiguousarray(
                np.asarray(s.angles if getattr(s, "angles", None) is not None else np.zeros((0, 3)),
                           dtype=np.int32).reshape(-1)),
        )
        k = self._keep
        self.sys = orc_sys(
            M=self.M, na=self.na, mass=_ptr(k["mass"]), L=(C.c_double * 3)(*s.box),
            xc=s.xc, d_at=s.d_at, d_hy=s.d_hy, eps=s.eps, sig=s.sigma, rc_at=s.rc_at,
            nb=len(k["bonds"]) // 2, bonds=_ptr(k["bonds"], C.c_int),
            fene_k=s.fene_k, fene_r0=s.fene_r0, intra_wca=int(s.intra_wca),
            cgF=_ptr(k["cgF"]), cgV=_ptr(k["cgV"]), cg_n=len(k["cgF"]) - 1, cg_dr=s.cg_dr,
            rc_cg=s.rc_cg, tf=_ptr(k["tf"]), tf_n=len(k["tf"]), tf_dx=s.tf_dx,
            kT=s.kT, gamma=s.gamma, dt=s.dt, seed=int(s.seed), replica=int(replica),
            nb_model=nb_model, charge=_ptr(k["charge"]), lj_eps=_ptr(k["lj_eps"]), lj_sig=_ptr(k["lj_sig"]),
            coulomb_f=float(getattr(s, "coulomb_f", 0.0)), eps_rf=float(getattr(s, "eps_rf", 1.0)),
            bond_model=int(getattr(s, "bond_model", 0)), bond_k=float(getattr(s, "bond_k", 0.0)),
            bond_r0=float(getattr(s, "bond_r0", 0.0)), n_angles=len(k["angles"]) // 3,
            angles=_ptr(k["angles"], C.c_int), angle_k=float(getattr(s, "angle_k", 0.0)),
            angle_theta0=float(getattr(s, "angle_theta0", 0.0)))
        self.set_centers(getattr(s, "centers", None))
        self.sys.scheme = int(getattr(s, "scheme", 0))
        self.sys.respa_n = int(getattr(s, "respa_n", 1))
        fec = getattr(s, "fec", None)
        self._fec = np.ascontiguousarray(np.asarray(fec if fec is not None else [], dtype=np.float64))
        self.sys.fec_n = len(self._fec)
        self.sys.fec = _ptr(self._fec) if len(self._fec) else None

    def set_mlp(self, net):
        """Use the learned CG pair force of `net` (an OracleMLP) in place of the table, or
        the table again with net=None."""
        self._mlp = net
        self.sys.mlp = C.pointer(net.m) if net is not None else C.POINTER(orc_mlp)()

    def set_tf(self, tf):
        self._keep["tf"] = np.ascontiguousarray(tf, dtype=np.float64)
        self.sys.tf = _ptr(self._keep["tf"])
        self.sys.tf_n = len(self._keep["tf"])

    def set_centers(self, centers):
        """Resolution centres (n, 3) of the self-adjusting geometry, or None for the slab."""
        c = np.zeros((0, 3)) if centers is None else np.asarray(centers, dtype=np.float64).reshape(-1, 3)
        self._keep["centers"] = np.ascontiguousarray(c.reshape(-1))
        self.sys.n_centers = len(c)
        self.sys.centers = _ptr(self._keep["centers"])

    def weight(self, d: float) -> float:
        return self.lib.orc_weight(C.byref(self.sys), float(d))

    def set_uniform_lambda(self, lam):
        """Every molecule at l = lam (None: l follows the geometry again)."""
        self.sys.lam_uniform_on = 0 if lam is None else 1
        self.sys.lam_uniform = 0.0 if lam is None else float(lam)

    def kirkwood(self, x, v, lambdas, n_equil, n_samples, every, step0=0):
        """Kirkwood thermodynamic integration of energy interpolation (Sec. "Free energy
        corrections and the thermodynamic force"): at each uniform l in `lambdas` (strictly
        inside (0, 1)), n_equil Langevin steps, then n_samples samples every `every` steps of
        dH/dl per molecule = (V_AT - V_CG) / M = (E_at / l - E_cg / (1 - l)) / M.  Each sample
        recomputes the conservative force, which the next steps start from.  Returns (g, x,
        v, step) with g[k] the mean at lambdas[k]."""
        g = []
        step = step0
        for lam in lambdas:
            self.set_uniform_lambda(lam)
            f, _ = self.forces(x)
            x, v, f = self.run(x, v, f, step, n_equil)
            step += n_equil
            acc = 0.0
            for _ in range(n_samples):
                x, v, f = self.run(x, v, f, step, every)
                step += every
                f, e = self.forces(x)
                acc += e["E_at"] / lam - e["E_cg"] / (1.0 - lam)
            g.append(acc / (n_samples * self.M))
        self.set_uniform_lambda(None)
        return np.array(g), x, v, step

    def com_lambda(self, x):
        x = np.ascontiguousarray(x, dtype=np.float64)
        R = np.empty((self.M, 3))
        dxc = np.empty(self.M)
        w = np.empty(self.M)
        self.lib.orc_com_lambda(C.byref(self.sys), _ptr(x), _ptr(R), _ptr(dxc), _ptr(w))
        return R, dxc, w

    def forces(self, x, method: int = 1, w_override=None, step=None):
        """Conservative forces (N,3) and energies {E_at, E_cg, E_bond, virial}.  With `step`
        (multiple time stepping) the slow part carries its weight at that time level."""
        x = np.ascontiguousarray(x, dtype=np.float64)
        f = np.empty((self.N, 3))
        e = np.zeros(4)
        wo = None if w_override is None else np.ascontiguousarray(w_override, dtype=np.float64)
        if step is not None:
            st = self.lib.orc_forces_step(C.byref(self.sys), _ptr(x), int(step), _ptr(f), _ptr(e))
        else:
            st = self.lib.orc_forces(C.byref(self.sys), _ptr(x), int(method), _ptr(wo), _ptr(f), _ptr(e))
        if st != ORC_OK:
            raise RuntimeError(f"oracle forces failed with status {st}")
        return f, dict(E_at=e[0], E_cg=e[1], E_bond=e[2], virial=e[3])

    def run(self, x, v, f, step0: int, nsteps: int, method: int = 1):
        """Advance (x, v, f) by nsteps of Langevin velocity Verlet; returns new copies."""
        x = np.array(x, dtype=np.float64, order="C")
        v = np.array(v, dtype=np.float64, order="C")
        f = np.array(f, dtype=np.float64, order="C")
        st = self.lib.orc_run(C.byref(self.sys), _ptr(x), _ptr(v), _ptr(f), int(step0), int(nsteps),
                              int(method))
        if st != ORC_OK:
            raise RuntimeError(f"oracle run failed with status {st}")
        return x, v, f

    def langevin_force(self, v, step: int):
        v = np.ascontiguousarray(v, dtype=np.float64)
        f = np.zeros((self.N, 3))
        self.lib.orc_langevin_force(C.byref(self.sys), _ptr(v), int(step), _ptr(f))
        return f

    def kinetic(self, v):
        v = np.ascontiguousarray(v, dtype=np.float64)
        out = np.zeros(4)
        self.lib.orc_kinetic(C.byref(self.sys), _ptr(v), _ptr(out))
        return out[0], out[1:].copy()

    def density(self, x, nd: int, nx: int):
        x = np.ascontiguousarray(x, dtype=np.float64)
        cd = np.zeros(nd, dtype=np.int64)
        cx = np.zeros(nx, dtype=np.int64)
        self.lib.orc_density(C.byref(self.sys), _ptr(x), nd, _ptr(cd, C.c_int64), nx, _ptr(cx, C.c_int64))
        return cd, cx

    def rdf_counts(self, x, nbins: int, dr: float):
        """Pair counts of COM distances in bins [k dr, (k+1) dr), all pairs a < b."""
        x = np.ascontiguousarray(x, dtype=np.float64)
        c = np.zeros(nbins, dtype=np.int64)
        self.lib.orc_rdf(C.byref(self.sys), _ptr(x), int(nbins), float(dr), _ptr(c, C.c_int64))
        return c

    def pair_features(self, x, a: int, b: int):
        x = np.ascontiguousarray(x, dtype=np.float64)
        feat = np.zeros(9)
        t = np.zeros(1)
        self.lib.orc_pair_features(C.byref(self.sys), _ptr(x), int(a), int(b), _ptr(feat), _ptr(t))
        return feat, float(t[0])

    def collect_pairs(self, x, rc: float, cap: int = 10_000_000):
        """Features [n, 9], targets [n], ids [n, 2] of every pair a < b with COM distance < rc."""
        x = np.ascontiguousarray(x, dtype=np.float64)
        n = self.lib.orc_collect_pairs(C.byref(self.sys), _ptr(x), float(rc), 0, None, None, None)
        feat = np.zeros((n, 9))
        t = np.zeros(n)
        ids = np.zeros((n, 2), dtype=np.int32)
        self.lib.orc_collect_pairs(C.byref(self.sys), _ptr(x), float(rc), n, _ptr(feat), _ptr(t),
                                   ids.ctypes.data_as(C.POINTER(C.c_int)))
        return feat, t, ids

    def tf_update(self, tf, counts_d, nsamples: float, alpha: float):
        tf = np.array(tf, dtype=np.float64, order="C")
        cd = np.ascontiguousarray(counts_d, dtype=np.int64)
        self.lib.orc_tf_update(C.byref(self.sys), _ptr(tf), len(tf), _ptr(cd, C.c_int64), len(cd),
                               float(nsamples), float(alpha))
        return tf


class OracleMLP:
    """FP64 network of the learned CG pair force (see adress_oracle.c).  params: dict with
    W1 [nh, 9], b1 [nh], W2 [nh, nh], b2 [nh], w3 [nh], b3, in_mean [9], in_std [9],
    out_scale."""

    def __init__(self, params, bf16: bool = False):
        self.lib = _load()
        self.nh = int(np.asarray(params["b1"]).size)
        k = {n: np.ascontiguousarray(np.asarray(params[n], dtype=np.float64).reshape(-1))
             for n in ("W1", "b1", "W2", "b2", "w3", "in_mean", "in_std")}
        self._keep = k
        self.m = orc_mlp(nh=self.nh, W1=_ptr(k["W1"]), b1=_ptr(k["b1"]), W2=_ptr(k["W2"]), b2=_ptr(k["b2"]),
                         w3=_ptr(k["w3"]), b3=float(params["b3"]), in_mean=_ptr(k["in_mean"]),
                         in_std=_ptr(k["in_std"]), out_scale=float(params["out_scale"]), bf16=int(bf16))

    def forward(self, feat):
        feat = np.ascontiguousarray(feat, dtype=np.float64)
        y = np.zeros(len(feat))
        self.lib.orc_mlp_forward(C.byref(self.m), len(feat), _ptr(feat), _ptr(y))
        return y

    def pair_force(self, feat):
        feat = np.ascontiguousarray(feat, dtype=np.float64)
        f = np.zeros(len(feat))
        self.lib.orc_mlp_pair_force(C.byref(self.m), len(feat), _ptr(feat), _ptr(f))
        return f

    def loss_grad(self, feat, target):
        feat = np.ascontiguousarray(feat, dtype=np.float64)
        target = np.ascontiguousarray(target, dtype=np.float64)
        nh = self.nh
        g = dict(W1=np.zeros((nh, 9)), b1=np.zeros(nh), W2=np.zeros((nh, nh)), b2=np.zeros(nh), w3=np.zeros(nh))
        gb3 = np.zeros(1)
        loss = self.lib.orc_mlp_loss_grad(C.byref(self.m), len(feat), _ptr(feat), _ptr(target), _ptr(g["W1"]),
                                          _ptr(g["b1"]), _ptr(g["W2"]), _ptr(g["b2"]), _ptr(g["w3"]), _ptr(gb3))
        g["b3"] = float(gb3[0])
        return loss, g


def bf16(v: float) -> float:
    return _load().orc_bf16(float(v))


def philox4x32(ctr, key):
    lib = _load()
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib.orc_philox4x32(_ptr(c, C.c_uint32), _ptr(k, C.c_uint32), _ptr(out, C.c_uint32))
    return out


def uniform3(seed: int, replica: int, gid: int, step: int):
    lib = _load()
    u = np.zeros(3)
    lib.orc_uniform3(int(seed), int(replica), int(gid), int(step), _ptr(u))
    return u


def force_matched_table(d, target, fit_dr: float, n_min: int, cg_dr: float, cg_n: int, rc: float):
    """Force-matched CG table.  The CG force of Eq. 1 acts between centres of mass (Sec.
    "Force interpolation"); matched to the atomistic model it is, per COM distance, the mean
    atomistic pair force projected on the COM axis.  From samples (d_i, t_i) with d the COM
    distance and t that projected force:

      1. bins j = floor(d / fit_dr) for d < rc, j < ceil(rc / fit_dr); mean_j = sum t / count
         over the bins holding at least n_min samples;
      2. F_raw(r) linear between the centres (j + 1/2) fit_dr of those bins, equal to the first
         (last) mean below (above) the first (last) centre;
      3. F(r_k) = F_raw(r_k) - F_raw(rc) on the nodes r_k = k cg_dr < rc (the force vanishes
         continuously at the cutoff), 0 from rc on;
      4. V(r_k) = sum over m >= k of (F_m + F_{m+1}) cg_dr / 2 (trapezoid rule, V = 0 at the
         last node).

    Returns F, V as float64 arrays [cg_n + 1]; raises ValueError when no bin holds n_min
    samples."""
    d = np.asarray(d, dtype=np.float64).reshape(-1)
    t = np.asarray(target, dtype=np.float64).reshape(-1)
    nb = int(math.ceil(rc / fit_dr))
    u = d / fit_dr
    keep = (d >= 0) & (u < nb)
    j = np.floor(u[keep]).astype(np.int64)
    sums = np.bincount(j, weights=t[keep], minlength=nb)
    counts = np.bincount(j, minlength=nb)
    pop = np.nonzero(counts >= n_min)[0]
    if len(pop) == 0:
        raise ValueError("no bin holds n_min samples")
    centre = (pop + 0.5) * fit_dr
    mean = sums[pop] / counts[pop]

    def raw(r):
        if r <= centre[0]:
            return mean[0]
        if r >= centre[-1]:
            return mean[-1]
        k = int(np.searchsorted(centre, r, side="right")) - 1  # centre[k] <= r < centre[k + 1]
        slope = (mean[k + 1] - mean[k]) / (centre[k + 1] - centre[k])
        return slope * (r - centre[k]) + mean[k]

    f_rc = raw(rc)
    r_nodes = np.arange(cg_n + 1, dtype=np.float64) * cg_dr
    F = np.array([raw(r) - f_rc if r < rc else 0.0 for r in r_nodes])
    V = np.zeros(cg_n + 1)
    v = 0.0
    for k in range(cg_n - 1, -1, -1):
        v += 0.5 * (F[k] + F[k + 1]) * cg_dr
        V[k] = v
    return F, V
