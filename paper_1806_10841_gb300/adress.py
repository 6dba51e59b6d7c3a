"""Python binding of the C ABI in ``include/adress.h`` (argument marshalling only).

Every step of the method runs in the CUDA library ``_build/libadress_gb300.so``; this
module only fills the configuration struct, owns the state tensors (PyTorch device
memory) and forwards calls.  There is no CPU fallback: a missing library is an error.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libadress_gb300.so")

ADRESS_FP64, ADRESS_FP32_MIXED = 0, 1
STATUS = {0: "ok", 1: "invalid argument", 2: "CUDA error", 3: "neighbour list overflow",
          4: "non-finite force", 5: "FENE bond broken", 6: "device wait timed out",
          7: "invalid state", 8: "molecule wider than the list cutoff allows"}

# Every symbol include/adress.h declares (checked by the CPU test suite).
EXPORTS = ["adress_init", "adress_init_batch", "adress_rdf", "adress_set_centers", "adress_set_uniform_lambda",
           "adress_kirkwood", "adress_set_tuning", "adress_get_tuning", "adress_autotune",
           "adress_bind_state", "adress_build_lists", "adress_compute_forces",
           "adress_step", "adress_run", "adress_set_step", "adress_get_step", "adress_com_lambda", "adress_kinetic",
           "adress_density_accumulate", "adress_density_get", "adress_density_reset",
           "adress_tf_update", "adress_set_tf", "adress_get_tf", "adress_list_stats", "adress_list_export",
           "adress_time_kernels", "adress_set_limit", "adress_cg_fit",
           "adress_kinetic_noalloc", "adress_check", "adress_mlp_set", "adress_mlp_get", "adress_set_cg_mode",
           "adress_mlp_collect", "adress_mlp_samples", "adress_mlp_load_samples", "adress_mlp_forward",
           "adress_mlp_loss_grad", "adress_mlp_train",
           "adress_last_error", "adress_status_string", "adress_destroy"]


class AdressError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class adress_config(C.Structure):
    _fields_ = [
        ("n_mols", C.c_int32), ("atoms_per_mol", C.c_int32),
        ("mass", C.POINTER(C.c_double)),
        ("box", C.c_double * 3),
        ("x_center", C.c_double), ("d_at_half", C.c_double), ("d_hy", C.c_double),
        ("wca_eps", C.c_double), ("wca_sigma", C.c_double), ("rc_at", C.c_double),
        ("n_bonds", C.c_int32), ("bonds", C.POINTER(C.c_int32)),
        ("fene_k", C.c_double), ("fene_r0", C.c_double),
        ("intra_wca", C.c_int32),
        ("cg_F", C.POINTER(C.c_double)), ("cg_V", C.POINTER(C.c_double)),
        ("cg_n", C.c_int32), ("cg_dr", C.c_double), ("rc_cg", C.c_double),
        ("tf", C.POINTER(C.c_double)), ("tf_n", C.c_int32), ("tf_dx", C.c_double),
        ("kT", C.c_double), ("gamma", C.c_double), ("dt", C.c_double),
        ("seed", C.c_uint64), ("replica", C.c_int64),
        ("skin", C.c_double), ("r_ext", C.c_double),
        ("max_neighbors", C.c_int32), ("precision", C.c_int32),
        ("nb_model", C.c_int32), ("charge", C.POINTER(C.c_double)), ("lj_eps", C.POINTER(C.c_double)),
        ("lj_sigma", C.POINTER(C.c_double)), ("coulomb_f", C.c_double), ("eps_rf", C.c_double),
        ("bond_model", C.c_int32), ("bond_k", C.c_double), ("bond_r0", C.c_double),
        ("n_angles", C.c_int32), ("angles", C.POINTER(C.c_int32)), ("angle_k", C.c_double),
        ("angle_theta0", C.c_double),
        ("n_centers", C.c_int32), ("centers", C.POINTER(C.c_double)),
        ("scheme", C.c_int32), ("fec_n", C.c_int32), ("fec", C.POINTER(C.c_double)),
        ("respa_n", C.c_int32),
    ]


_lib = None


def load_library(path: str = LIB_PATH):
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library {path} is missing: build it with "
                           "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = C.CDLL(path)
    H, vp, d = C.c_void_p, C.c_void_p, C.POINTER(C.c_double)
    i64p = C.POINTER(C.c_int64)
    sig = {
        "adress_init": ([C.POINTER(adress_config), vp, C.POINTER(H)], C.c_int),
        "adress_init_batch": ([C.POINTER(adress_config), C.c_int32, vp, C.POINTER(H)], C.c_int),
        "adress_set_tuning": ([H, C.c_int32, C.c_double], C.c_int),
        "adress_rdf": ([H, C.c_int32, C.c_double, i64p], C.c_int),
        "adress_set_centers": ([H, d, C.c_int32], C.c_int),
        "adress_set_uniform_lambda": ([H, C.c_int32, C.c_double], C.c_int),
        "adress_kirkwood": ([H, d, C.c_int32, C.c_int32, C.c_int32, C.c_int32, d], C.c_int),
        "adress_get_tuning": ([H, C.POINTER(C.c_int32), d], C.c_int),
        "adress_autotune": ([H, C.c_int32, d, C.c_int32, C.POINTER(C.c_int32)], C.c_int),
        "adress_bind_state": ([H, vp, vp, vp], C.c_int),
        "adress_build_lists": ([H], C.c_int),
        "adress_compute_forces": ([H, d], C.c_int),
        "adress_step": ([H, C.c_int32], C.c_int),
        "adress_run": ([H, C.c_int32, C.c_int32, C.c_int32, C.c_double], C.c_int),
        "adress_set_step": ([H, C.c_int64], C.c_int),
        "adress_get_step": ([H, i64p], C.c_int),
        "adress_com_lambda": ([H, vp, vp], C.c_int),
        "adress_kinetic": ([H, d], C.c_int),
        "adress_density_accumulate": ([H], C.c_int),
        "adress_density_get": ([H, i64p, C.c_int32, i64p], C.c_int),
        "adress_density_reset": ([H], C.c_int),
        "adress_tf_update": ([H, C.c_double], C.c_int),
        "adress_set_tf": ([H, d, C.c_int32], C.c_int),
        "adress_get_tf": ([H, d, C.c_int32], C.c_int),
        "adress_list_stats": ([H, i64p], C.c_int),
        "adress_list_export": ([H, C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.POINTER(C.c_int32)], C.c_int),
        "adress_time_kernels": ([H, C.c_int32, C.POINTER(C.c_float)], C.c_int),
        "adress_set_limit": ([H, C.c_int32, C.c_int64], C.c_int),
        "adress_cg_fit": ([H, C.c_double, C.c_int32, C.c_int32, d, d], C.c_int),
        "adress_kinetic_noalloc": ([vp, C.c_int64, C.c_int32, d, vp, vp], C.c_int),
        "adress_check": ([H], C.c_int),
        "adress_mlp_set": ([H, C.POINTER(C.c_float), C.POINTER(C.c_float)], C.c_int),
        "adress_mlp_get": ([H, C.POINTER(C.c_float), C.POINTER(C.c_float)], C.c_int),
        "adress_set_cg_mode": ([H, C.c_int32], C.c_int),
        "adress_mlp_collect": ([H, C.c_int64, i64p], C.c_int),
        "adress_mlp_samples": ([H, C.POINTER(C.c_float), C.POINTER(C.c_float), C.POINTER(C.c_int32), C.c_int64],
                               C.c_int),
        "adress_mlp_load_samples": ([H, C.POINTER(C.c_float), C.POINTER(C.c_float), C.c_int64], C.c_int),
        "adress_mlp_forward": ([H, vp, C.c_int64, vp], C.c_int),
        "adress_mlp_loss_grad": ([H, vp, vp, C.c_int64, C.POINTER(C.c_float)], C.c_int),
        "adress_mlp_train": ([H, C.c_int32, C.c_int32, C.c_float, C.POINTER(C.c_float)], C.c_int),
        "adress_last_error": ([H], C.c_char_p),
        "adress_status_string": ([C.c_int], C.c_char_p),
        "adress_destroy": ([H], None),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def _dptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _config(s, keep, replica, max_neighbors, precision):
    """adress_config of one system; the host arrays it points to are appended to keep."""
    arrs = dict(
        mass=np.ascontiguousarray(s.mass, dtype=np.float64),
        bonds=np.ascontiguousarray(np.asarray(s.bonds, dtype=np.int32).reshape(-1)),
        cgF=np.ascontiguousarray(s.cg_F, dtype=np.float64),
        cgV=np.ascontiguousarray(s.cg_V, dtype=np.float64),
        tf=np.ascontiguousarray(s.tf if s.tf is not None else np.zeros(0), dtype=np.float64),
    )
    nb_model = int(getattr(s, "nb_model", 0))
    ang = getattr(s, "angles", None)
    arrs.update(
        charge=np.ascontiguousarray(s.charge if nb_model else np.zeros(s.na), dtype=np.float64),
        lj_eps=np.ascontiguousarray(s.lj_eps if nb_model else np.zeros(s.na), dtype=np.float64),
        lj_sig=np.ascontiguousarray(s.lj_sig if nb_model else np.zeros(s.na), dtype=np.float64),
        angles=np.ascontiguousarray(np.asarray(ang if ang is not None else np.zeros((0, 3)), dtype=np.int32).reshape(-1)),
        centers=np.ascontiguousarray(np.asarray(getattr(s, "centers", None) if getattr(s, "centers", None) is not None
                                                else np.zeros((0, 3)), dtype=np.float64).reshape(-1)),
        fec=np.ascontiguousarray(np.asarray(getattr(s, "fec", None) if getattr(s, "fec", None) is not None
                                            else np.zeros(0), dtype=np.float64).reshape(-1)),
    )
    keep.append(arrs)
    tf_n = len(arrs["tf"])
    return adress_config(
        n_mols=int(s.M), atoms_per_mol=int(s.na), mass=_dptr(arrs["mass"]), box=(C.c_double * 3)(*s.box),
        x_center=s.xc, d_at_half=s.d_at, d_hy=s.d_hy, wca_eps=s.eps, wca_sigma=s.sigma,
        rc_at=s.rc_at, n_bonds=len(arrs["bonds"]) // 2,
        bonds=arrs["bonds"].ctypes.data_as(C.POINTER(C.c_int32)), fene_k=s.fene_k,
        fene_r0=s.fene_r0, intra_wca=int(s.intra_wca), cg_F=_dptr(arrs["cgF"]), cg_V=_dptr(arrs["cgV"]),
        cg_n=len(arrs["cgF"]) - 1, cg_dr=s.cg_dr, rc_cg=s.rc_cg,
        tf=_dptr(arrs["tf"]) if tf_n else None, tf_n=tf_n, tf_dx=s.tf_dx,
        kT=s.kT, gamma=s.gamma, dt=s.dt, seed=int(s.seed), replica=int(replica), skin=s.skin,
        r_ext=s.r_ext, max_neighbors=int(max_neighbors),
        precision=ADRESS_FP64 if precision == "fp64" else ADRESS_FP32_MIXED,
        nb_model=nb_model, charge=_dptr(arrs["charge"]), lj_eps=_dptr(arrs["lj_eps"]), lj_sigma=_dptr(arrs["lj_sig"]),
        coulomb_f=float(getattr(s, "coulomb_f", 0.0)), eps_rf=float(getattr(s, "eps_rf", 1.0)),
        bond_model=int(getattr(s, "bond_model", 0)), bond_k=float(getattr(s, "bond_k", 0.0)),
        bond_r0=float(getattr(s, "bond_r0", 0.0)), n_angles=len(arrs["angles"]) // 3,
        angles=arrs["angles"].ctypes.data_as(C.POINTER(C.c_int32)), angle_k=float(getattr(s, "angle_k", 0.0)),
        angle_theta0=float(getattr(s, "angle_theta0", 0.0)),
        n_centers=len(arrs["centers"]) // 3, centers=_dptr(arrs["centers"]) if len(arrs["centers"]) else None,
        scheme=int(getattr(s, "scheme", 0)), fec_n=len(arrs["fec"]),
        fec=_dptr(arrs["fec"]) if len(arrs["fec"]) else None, respa_n=int(getattr(s, "respa_n", 1)))


class AdResS:
    """One AdResS system, or a batch of independent replicas, on one GPU.

    State tensors live on the device in structure-of-arrays layout ``[3, N]``:
    ``x``, ``v`` float64 and ``f`` float64 (``precision='fp64'``) or float32
    (``precision='fp32'``, the mixed path).  With a list of systems (``adress_init_batch``)
    replica r's molecules follow those of replicas 0..r-1; ``replica`` is then a list of
    replica ids (default 0, 1, ...), and ``mol0`` / ``atom0`` give each replica's first
    molecule / atom.
    """

    def __init__(self, system, *, precision: str = "fp32", device: str = "cuda:0", stream=None,
                 max_neighbors: int = 0, replica=0):
        import torch

        self.torch = torch
        self.lib = load_library()
        self.system = system
        self.precision = precision
        self.device = torch.device(device)
        batch = isinstance(system, (list, tuple))
        systems = list(system) if batch else [system]
        if batch and isinstance(replica, int):
            replica = list(range(replica, replica + len(systems)))
        reps = list(replica) if batch else [replica]
        self._keep = []
        cfgs = (adress_config * len(systems))(*[_config(s, self._keep, r, max_neighbors, precision)
                                                  for s, r in zip(systems, reps)])
        self.n_replicas = len(systems)
        self.na = int(systems[0].na)
        self.mol0 = np.concatenate([[0], np.cumsum([int(s.M) for s in systems])]).astype(np.int64)
        self.M = int(self.mol0[-1])
        self.atom0 = self.mol0 * self.na
        self.N = self.M * self.na
        self.tf_n = len(self._keep[0]["tf"]) * len(systems)
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
            self.h = C.c_void_p()
            sp = C.c_void_p(self.stream.cuda_stream)
            if batch:
                st = self.lib.adress_init_batch(cfgs, len(systems), sp, C.byref(self.h))
            else:
                st = self.lib.adress_init(C.byref(cfgs[0]), sp, C.byref(self.h))
            if st != 0:
                raise AdressError(st, self.lib.adress_last_error(None).decode())
            fdt = torch.float64 if precision == "fp64" else torch.float32
            self.x = torch.zeros((3, self.N), dtype=torch.float64, device=self.device)
            self.v = torch.zeros((3, self.N), dtype=torch.float64, device=self.device)
            self.f = torch.zeros((3, self.N), dtype=fdt, device=self.device)
            self._call("adress_bind_state", C.c_void_p(self.x.data_ptr()), C.c_void_p(self.v.data_ptr()),
                       C.c_void_p(self.f.data_ptr()))

    # -- plumbing -------------------------------------------------------------------
    def _call(self, name, *args):
        st = getattr(self.lib, name)(self.h, *args)
        if st != 0:
            raise AdressError(st, self.lib.adress_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            self.lib.adress_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- state ------------------------------------------------------------------------
    def set_state(self, x, v=None, f=None):
        """x, v, f: (N, 3) numpy arrays (host) or [3, N] tensors."""
        t = self.torch
        for dst, src in ((self.x, x), (self.v, v), (self.f, f)):
            if src is None:
                continue
            if isinstance(src, np.ndarray):
                src = t.from_numpy(np.ascontiguousarray(np.asarray(src).T))
            with t.cuda.stream(self.stream):
                dst.copy_(src.to(dst.dtype), non_blocking=False)
        self.stream.synchronize()

    def get_state(self):
        self.stream.synchronize()
        return (self.x.T.cpu().numpy().copy(), self.v.T.cpu().numpy().copy(),
                self.f.T.to(self.torch.float64).cpu().numpy().copy())

    # -- C ABI calls --------------------------------------------------------------------
    def build_lists(self):
        self._call("adress_build_lists")

    def compute_forces(self, energies: bool = True):
        e = np.zeros(4)
        self._call("adress_compute_forces", _dptr(e) if energies else None)
        return dict(E_at=e[0], E_cg=e[1], E_bond=e[2], virial=e[3]) if energies else None

    def forces(self):
        """Conservative forces (N, 3) float64 on the host plus energies."""
        e = self.compute_forces(True)
        self.stream.synchronize()
        return self.f.T.to(self.torch.float64).cpu().numpy().copy(), e

    def step(self, nsteps: int):
        self._call("adress_step", C.c_int32(int(nsteps)))

    def run(self, nsteps: int, sample_every: int = 0, tf_update: bool = False, alpha: float = 0.0):
        """One thermodynamic-force iteration block as a single captured graph."""
        self._call("adress_run", C.c_int32(int(nsteps)), C.c_int32(int(sample_every)),
                   C.c_int32(1 if tf_update else 0), C.c_double(float(alpha)))

    def set_step(self, step: int):
        self._call("adress_set_step", C.c_int64(int(step)))

    def get_step(self) -> int:
        v = C.c_int64()
        self._call("adress_get_step", C.byref(v))
        return v.value

    def com_lambda(self):
        t = self.torch
        com = t.empty((3, self.M), dtype=t.float64, device=self.device)
        w = t.empty((self.M,), dtype=t.float64, device=self.device)
        self._call("adress_com_lambda", C.c_void_p(com.data_ptr()), C.c_void_p(w.data_ptr()))
        self.stream.synchronize()
        return com.T.cpu().numpy().copy(), w.cpu().numpy().copy()

    def kinetic(self):
        out = np.zeros(4)
        self._call("adress_kinetic", _dptr(out))
        return out[0], out[1:].copy()

    def rdf_counts(self, nbins: int = 250, dr: float = 0.02):
        """COM pair-distance histogram [n_replicas, nbins] of the current positions."""
        c = np.zeros(self.n_replicas * int(nbins), dtype=np.int64)
        self._call("adress_rdf", C.c_int32(int(nbins)), C.c_double(float(dr)), c.ctypes.data_as(C.POINTER(C.c_int64)))
        return c.reshape(self.n_replicas, int(nbins))

    @staticmethod
    def rdf_normalise(counts, n_mols: int, volume: float, dr: float, n_samples: int = 1):
        """g(r) per bin from pair counts summed over n_samples snapshots: counts divided by
        the ideal-gas pair count of the bin's shell."""
        k = np.arange(len(counts), dtype=np.float64)
        shell = 4.0 / 3.0 * np.pi * ((k + 1) ** 3 - k ** 3) * dr ** 3
        ideal = n_samples * 0.5 * n_mols * (n_mols - 1) * shell / volume
        return np.asarray(counts, dtype=np.float64) / ideal

    def density_accumulate(self):
        self._call("adress_density_accumulate")

    def density_get(self):
        counts = np.zeros(self.tf_n, dtype=np.int64)
        ns = C.c_int64()
        self._call("adress_density_get", counts.ctypes.data_as(C.POINTER(C.c_int64)), self.tf_n, C.byref(ns))
        return counts, ns.value

    def density_reset(self):
        self._call("adress_density_reset")

    def tf_update(self, alpha: float):
        self._call("adress_tf_update", C.c_double(alpha))

    def set_tf(self, tf):
        tf = np.ascontiguousarray(tf, dtype=np.float64)
        self._call("adress_set_tf", _dptr(tf), len(tf))

    def get_tf(self):
        tf = np.zeros(self.tf_n)
        self._call("adress_get_tf", _dptr(tf), self.tf_n)
        return tf

    def set_centers(self, centers):
        """Move the resolution centres (n, 3) of the self-adjusting geometry."""
        c = np.ascontiguousarray(np.asarray(centers, dtype=np.float64).reshape(-1))
        self._call("adress_set_centers", _dptr(c), C.c_int32(len(c) // 3))

    def set_uniform_lambda(self, lam):
        """Every molecule at resolution lam (None: the geometry decides again); rebuild the
        lists (build_lists / compute_forces) before stepping."""
        self._call("adress_set_uniform_lambda", C.c_int32(0 if lam is None else 1), C.c_double(0.0 if lam is None else lam))

    def kirkwood(self, lambdas, n_equil: int, n_samples: int, every: int):
        """Kirkwood thermodynamic integration: mean dH/dl per molecule at each uniform l."""
        lam = np.ascontiguousarray(np.asarray(lambdas, dtype=np.float64).reshape(-1))
        out = np.zeros(len(lam))
        self._call("adress_kirkwood", _dptr(lam), C.c_int32(len(lam)), C.c_int32(n_equil), C.c_int32(n_samples),
                   C.c_int32(every), _dptr(out))
        return out

    def set_tuning(self, force_block: int, skin: float):
        self._call("adress_set_tuning", C.c_int32(int(force_block)), C.c_double(float(skin)))

    def get_tuning(self):
        b, sk = C.c_int32(), C.c_double()
        self._call("adress_get_tuning", C.byref(b), C.byref(sk))
        return b.value, sk.value

    def autotune(self, nsteps: int = 20):
        """Pick threads per block and list skin by timing nsteps-step runs (5 timed runs per
        trial, the state restored); returns the trial table as rows (force_block, skin, median
        ms per step, fastest, slowest)."""
        rows = np.zeros((32, 5))
        n = C.c_int32()
        self._call("adress_autotune", C.c_int32(int(nsteps)), _dptr(rows), 32, C.byref(n))
        return [(int(r[0]), float(r[1]), float(r[2]), float(r[3]), float(r[4])) for r in rows[:n.value]]

    LIMIT_PAIR_CAPACITY, LIMIT_MMA_WAIT_POLLS = 0, 1

    def set_limit(self, which: int, value: int):
        """Run-time limit of the handle (adress_set_limit): LIMIT_PAIR_CAPACITY (pairs the
        learned force's buffers may hold, <= 0: the allocation) or LIMIT_MMA_WAIT_POLLS (polls
        of the tcgen05 evaluation's bounded waits, < 0: the default)."""
        self._call("adress_set_limit", C.c_int32(int(which)), C.c_int64(int(value)))

    def list_stats(self):
        out = np.zeros(8, dtype=np.int64)
        self._call("adress_list_stats", out.ctypes.data_as(C.POINTER(C.c_int64)))
        keys = ["n_hr", "n_cg", "rebuilds", "max_nn", "capacity", "n_cells"]
        return {k: int(out[i]) for i, k in enumerate(keys)}

    def neighbour_lists(self):
        """(items, nn, nbr[M, capacity]) of the current lists, on the host."""
        cap = self.list_stats()["capacity"]
        items = np.zeros(self.M, dtype=np.int32)
        nn = np.zeros(self.M, dtype=np.int32)
        nbr = np.zeros(self.M * cap, dtype=np.int32)
        p32 = lambda a: a.ctypes.data_as(C.POINTER(C.c_int32))
        self._call("adress_list_export", p32(items), p32(nn), p32(nbr))
        return items, nn, nbr.reshape(self.M, cap)

    def neighbour_pairs(self):
        items, nn, nbr = self.neighbour_lists()
        return {(int(items[t]), int(nbr[t, q])) for t in range(self.M) for q in range(nn[t])}

    def time_kernels(self, reps: int = 20):
        """ms per launch of the step kernels (advances the state by reps + 1 steps)."""
        out = (C.c_float * 4)()
        self._call("adress_time_kernels", C.c_int32(int(reps)), out)
        return dict(prologue=out[0], rebuild=out[1], step=out[2], last=out[3])

    # -- learned CG force ---------------------------------------------------------------
    MLP_NPAR, MLP_NNORM = 4865, 19

    @staticmethod
    def mlp_flatten(p):
        """dict (W1 [64,9], b1, W2 [64,64], b2, w3, b3) -> flat float32 [4865]."""
        return np.concatenate([np.asarray(p[k], dtype=np.float32).reshape(-1)
                               for k in ("W1", "b1", "W2", "b2", "w3")] + [np.float32([p["b3"]])])

    @staticmethod
    def mlp_unflatten(v):
        v = np.asarray(v, dtype=np.float64)
        o = 0
        out = {}
        for k, shape in (("W1", (64, 9)), ("b1", (64,)), ("W2", (64, 64)), ("b2", (64,)), ("w3", (64,))):
            n = int(np.prod(shape))
            out[k] = v[o:o + n].reshape(shape)
            o += n
        out["b3"] = float(v[o])
        return out

    def mlp_set(self, params, in_mean, in_std, out_scale):
        flat = np.ascontiguousarray(self.mlp_flatten(params))
        norm = np.ascontiguousarray(np.concatenate([in_mean, in_std, [out_scale]]).astype(np.float32))
        f32 = lambda a: a.ctypes.data_as(C.POINTER(C.c_float))
        self._call("adress_mlp_set", f32(flat), f32(norm))

    def mlp_get(self):
        flat = np.zeros(self.MLP_NPAR, dtype=np.float32)
        norm = np.zeros(self.MLP_NNORM, dtype=np.float32)
        f32 = lambda a: a.ctypes.data_as(C.POINTER(C.c_float))
        self._call("adress_mlp_get", f32(flat), f32(norm))
        p = self.mlp_unflatten(flat)
        p.update(in_mean=norm[:9].astype(np.float64), in_std=norm[9:18].astype(np.float64),
                 out_scale=float(norm[18]))
        return p

    def set_cg_mode(self, mode: int):
        self._call("adress_set_cg_mode", C.c_int32(int(mode)))

    def mlp_collect(self, cap: int) -> int:
        n = C.c_int64()
        self._call("adress_mlp_collect", C.c_int64(int(cap)), C.byref(n))
        return n.value

    def mlp_samples(self, n: int):
        feat = np.zeros((n, 9), dtype=np.float32)
        t = np.zeros(n, dtype=np.float32)
        ids = np.zeros((n, 2), dtype=np.int32)
        self._call("adress_mlp_samples", feat.ctypes.data_as(C.POINTER(C.c_float)),
                   t.ctypes.data_as(C.POINTER(C.c_float)), ids.ctypes.data_as(C.POINTER(C.c_int32)), C.c_int64(n))
        return feat, t, ids

    def mlp_load_samples(self, feat, target):
        feat = np.ascontiguousarray(feat, dtype=np.float32)
        target = np.ascontiguousarray(target, dtype=np.float32)
        self._call("adress_mlp_load_samples", feat.ctypes.data_as(C.POINTER(C.c_float)),
                   target.ctypes.data_as(C.POINTER(C.c_float)), C.c_int64(len(target)))

    def mlp_forward(self, feat):
        t = self.torch
        fd = t.from_numpy(np.ascontiguousarray(feat, dtype=np.float32)).to(self.device)
        y = t.zeros(len(fd), dtype=t.float32, device=self.device)
        self._call("adress_mlp_forward", C.c_void_p(fd.data_ptr()), C.c_int64(len(fd)), C.c_void_p(y.data_ptr()))
        self.stream.synchronize()
        return y.cpu().numpy().astype(np.float64)

    def mlp_loss_grad(self, feat, target):
        t = self.torch
        fd = t.from_numpy(np.ascontiguousarray(feat, dtype=np.float32)).to(self.device)
        td = t.from_numpy(np.ascontiguousarray(target, dtype=np.float32)).to(self.device)
        g = np.zeros(self.MLP_NPAR + 1, dtype=np.float32)
        self._call("adress_mlp_loss_grad", C.c_void_p(fd.data_ptr()), C.c_void_p(td.data_ptr()),
                   C.c_int64(len(td)), g.ctypes.data_as(C.POINTER(C.c_float)))
        grads = self.mlp_unflatten(g[:-1])
        return float(g[-1]) / len(td), grads

    def cg_fit(self, fit_dr: float, n_min: int = 1, install: bool = False):
        """Force-matched CG table (F, V on the table's nodes) from the held samples; with
        install=True it becomes the handle's CG table."""
        n = len(self.system[0].cg_F) if isinstance(self.system, (list, tuple)) else len(self.system.cg_F)
        F, V = np.zeros(n), np.zeros(n)
        self._call("adress_cg_fit", C.c_double(float(fit_dr)), C.c_int32(int(n_min)), C.c_int32(1 if install else 0),
                   _dptr(F), _dptr(V))
        return F, V

    def mlp_train(self, epochs: int, batch: int = 1024, lr: float = 1e-3):
        loss = np.zeros(epochs, dtype=np.float32)
        self._call("adress_mlp_train", C.c_int32(int(epochs)), C.c_int32(int(batch)), C.c_float(lr),
                   loss.ctypes.data_as(C.POINTER(C.c_float)))
        return loss

    def check(self):
        self._call("adress_check")
