"""Benchmark of the AdResS force-interpolation step on the 800k-atom tetrahedral fluid.

A bench step is one thermodynamic-force iteration block: 100 Langevin velocity-Verlet
MD steps (list rebuilds on the device as needed), a COM density sample every 10 MD
steps, and one thermodynamic-force update from that profile.  Metric: atom-steps/s =
atoms x MD steps / device seconds.  L2 is flushed (a 512 MB write) between timed
bench steps, outside the timed region.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp32|fp64]
  python bench.py --impl reference ...   # the FP64 CPU oracle on host cores

Under torchrun each rank runs an independent replica (replicas only; no collective on
the data path) and value is the sum over ranks of atoms x steps / max rank time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

MD_PER_BLOCK = 100
SAMPLE_EVERY = 10
TF_ALPHA = 0.5
METRIC = "AdResS atom-steps/s"
RDF_BINS, RDF_DR, RDF_EQ, RDF_SNAPS, RDF_EVERY = 250, 0.02, 2000, 50, 400
FIT_DR, FIT_NMIN = 0.01, 20  # force-matched table: bin width (sigma) and samples a bin needs
CONFIG_NAME = "tetrahedral AdResS fluid, 200k molecules / 800k atoms, 200x100x100 sigma, AT 40 + 2x10 hybrid"


def profiled_traffic(profile, sources):
    """DRAM bytes (read + write) per launch from an ncu summary under profiles/, or None when
    the kernel's sources changed since the capture (the summary records their hash)."""
    import hashlib
    import re

    path = os.path.join(ROOT, "profiles", profile)
    if not os.path.exists(path):
        return None
    txt = open(path).read()
    m = re.search(r"sha256\[:16\] = `([0-9a-f]+)`", txt)
    h = hashlib.sha256()
    for name in sources:
        h.update(open(os.path.join(ROOT, "paper_1806_10841_gb300", "csrc", name), "rb").read())
    if not m or m.group(1) != h.hexdigest()[:16]:
        return None
    scale = {"byte": 1.0, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9}
    total = 0.0
    for metric in ("dram__bytes_read.sum", "dram__bytes_write.sum"):
        r = re.search(r"`" + re.escape(metric) + r"` \| ([0-9.]+) \| (\w+) \|", txt)
        if not r:
            return None
        total += float(r.group(1)) * scale.get(r.group(2), float("nan"))
    return total


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            return json.load(open(p)), "measured"
        except Exception:
            pass
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class Clocks:
    """nvidia-smi sampling (every 50 ms) started before the warm-up, so that it runs during the
    timed region; the summary keeps the samples taken inside that region (the one nearest to
    its middle when the region is shorter than the sampling interval)."""

    Q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        import tempfile

        try:
            fd, self.path = tempfile.mkstemp(prefix=f"adress_clocks_{self.index}_", suffix=".csv")
            self.fh = os.fdopen(fd, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()
        if self.path and os.path.exists(self.path):
            with open(self.path) as fh:
                self.lines = fh.readlines()
            os.unlink(self.path)

    def summary(self, t0=None, t1=None):
        if self.proc is None or not getattr(self, "lines", None):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        import datetime

        rows = []
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 10:
                continue
            try:
                ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                rows.append((ts, float(parts[2]), float(parts[3]), parts[6:10]))
            except ValueError:
                continue
        if t0 is not None and rows:
            inside = [r for r in rows if t0 <= r[0] <= t1]
            if not inside:
                mid = 0.5 * (t0 + t1)
                inside = [min(rows, key=lambda r: abs(r[0] - mid))]
            rows = inside
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            for n, v in zip(names, r[3]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        sm = [r[1] for r in rows]
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(r[2] for r in rows) if rows else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def pair_statistics(s, x):
    """Unique interactions of the force evaluation (algorithmic work per launch), counted
    on the host from the positions with numpy (cell grid over molecule centres)."""
    L = np.array(s.box)
    M, na = s.M, s.na
    xm = x.reshape(M, na, 3)
    d0 = xm - xm[:, :1]
    d0 -= L * np.rint(d0 / L)
    R = np.mod(xm[:, 0] + (s.mass[None, :, None] * d0).sum(1) / s.mass.sum(), L)
    dxc = R[:, 0] - s.xc
    dxc -= L[0] * np.rint(dxc / L[0])
    d = np.abs(dxc)
    w = np.where(d < s.d_at, 1.0, np.where(d >= s.d_at + s.d_hy, 0.0,
                                           np.cos(0.5 * np.pi * (d - s.d_at) / max(s.d_hy, 1e-30)) ** 2))
    reach = max(s.rc_cg, s.rc_at + 2 * 0.75)
    nc = np.maximum(1, np.floor(L / reach)).astype(int)
    cell = np.minimum((R / L * nc).astype(int), nc - 1)
    lin = (cell[:, 0] * nc[1] + cell[:, 1]) * nc[2] + cell[:, 2]
    order = np.argsort(lin, kind="stable")
    lin_s = lin[order]
    starts = np.searchsorted(lin_s, np.arange(nc.prod() + 1))
    n_at = n_cg = 0
    offs = [(i, j, k) for i in (-1, 0, 1) for j in (-1, 0, 1) for k in (-1, 0, 1)]
    for o in offs:
        nb = (cell + np.array(o)) % nc
        nl = (nb[:, 0] * nc[1] + nb[:, 1]) * nc[2] + nb[:, 2]
        cnt = starts[nl + 1] - starts[nl]
        mx = cnt.max()
        for q in range(mx):
            has = cnt > q
            a = np.nonzero(has)[0]
            b = order[starts[nl[a]] + q]
            keep = b > a
            a, b = a[keep], b[keep]
            dR = R[a] - R[b]
            dR -= L * np.rint(dR / L)
            r2 = (dR ** 2).sum(1)
            wab = w[a] * w[b]
            n_cg += int(((r2 < s.rc_cg ** 2) & (wab < 1)).sum())
            sel = wab > 0
            a2, b2 = a[sel], b[sel]
            for i in range(na):
                for j in range(na):
                    dd = xm[a2, i] - xm[b2, j]
                    dd -= L * np.rint(dd / L)
                    n_at += int(((dd ** 2).sum(1) < s.rc_at ** 2).sum())
    return {"at_pairs": n_at, "cg_pairs": n_cg, "bonds": M * len(s.bonds), "atoms": M * na,
            "hr_molecules": int((w > 0).sum())}


FLOPS = {"at_pair": 35, "cg_pair": 55, "bond": 40}  # FP32 flops per interaction
ALGO_BYTES_PER_ATOM = 110  # HBM bytes per atom-step of the fused step kernel (see main)


def job_throughput(seconds, atom_steps, dist=None, device=None):
    """Whole-job throughput: every rank runs its own replica; the job's time is the slowest
    rank's, its work the sum over ranks.  Returns (atom-steps/s, max seconds)."""
    if dist is not None and dist.is_initialized():
        import torch

        t = torch.tensor([seconds, float(atom_steps)], dtype=torch.float64, device=device)
        tmax, tsum = t.clone(), t.clone()
        dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
        dist.all_reduce(tsum, op=dist.ReduceOp.SUM)
        seconds, atom_steps = float(tmax[0]), float(tsum[1])
    return atom_steps / seconds, seconds


def oracle_all_cores():
    """Path of the oracle's all-core (OpenMP) build and the threads it runs with."""
    import ctypes

    import oracle

    path = oracle.build(extra_flags=("-fopenmp",))
    return path, int(ctypes.CDLL(path).omp_get_max_threads())


def reference_arm(args, world, rank):
    """The FP64 CPU oracle on all host cores (its OpenMP build; a bounded sample of the same
    workload: one MD step of the full 800k-atom system per bench step)."""
    if rank != 0:
        return 0
    import oracle
    from paper_1806_10841_gb300 import inputs

    path, cores = oracle_all_cores()
    s = inputs.c2_800k()
    x, v = inputs.tetra_state(s)
    o = oracle.Oracle(s, lib_path=path)
    f, _ = o.forces(x)
    for k in range(args.warmup):
        x, v, f = o.run(x, v, f, k, 1)
    t0 = time.perf_counter()
    for k in range(args.steps):
        x, v, f = o.run(x, v, f, args.warmup + k, 1)
    dt = time.perf_counter() - t0
    value = s.N * args.steps / dt
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "atom-steps/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": CONFIG_NAME, "md_steps_per_bench_step": 1, "atoms": s.N},
            "cpu_baseline": {"value": value, "unit": "atom-steps/s", "cores": cores, "kind": "oracle",
                             "sample": f"{args.steps} MD steps of the full 800k-atom system (1 per bench step), "
                                       f"OpenMP build on {cores} host threads"},
            "e2e": {"value": value, "unit": "atom-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def cpu_baseline_sample(s, x, v):
    """The oracle as it stands on the host: its all-core OpenMP build on a bounded sample of
    the benchmark workload (value), the plain single-thread build on the same, and config 1
    (1000 molecules, 4000 atoms) for its full 100 steps, single thread."""
    import oracle
    from paper_1806_10841_gb300 import inputs

    def sample(o, budget_s, max_steps):
        xx, vv = x, v
        f, _ = o.forces(xx)
        n = 0
        t0 = time.perf_counter()
        while True:
            xx, vv, f = o.run(xx, vv, f, n, 1)
            n += 1
            if time.perf_counter() - t0 > budget_s or n >= max_steps:
                break
        return n, time.perf_counter() - t0

    path, cores = oracle_all_cores()
    n_omp, t_omp = sample(oracle.Oracle(s, lib_path=path), 12.0, 200)
    n_one, t_one = sample(oracle.Oracle(s), 8.0, 8)
    c1 = inputs.c1_stable()
    x1, v1 = inputs.tetra_state(c1)
    o1 = oracle.Oracle(c1)
    f1, _ = o1.forces(x1)
    t0 = time.perf_counter()
    o1.run(x1, v1, f1, 0, 100)
    t_c1 = time.perf_counter() - t0
    return {"value": s.N * n_omp / t_omp, "unit": "atom-steps/s", "cores": cores, "kind": "oracle",
            "sample": f"{n_omp} MD steps (force, bonded, thermostat, integration) of the full 800k-atom system, "
                      f"OpenMP build of the oracle on {cores} host threads",
            "single_thread": {"value": s.N * n_one / t_one, "cores": 1,
                              "sample": f"{n_one} MD steps of the full 800k-atom system, plain build"},
            "c1_full": {"value": c1.N * 100 / t_c1, "cores": 1, "seconds": t_c1,
                        "sample": "config 1 (1000 tetrahedra, 4000 atoms, density 0.1 reading), all 100 MD steps, "
                                  "plain build"}}


def run_block(sim, nsteps=MD_PER_BLOCK):
    """One bench step: a thermodynamic-force iteration block as a single captured graph."""
    sim.run(nsteps, sample_every=SAMPLE_EVERY, tf_update=True, alpha=TF_ALPHA)


def atomistic_samples(s, x0, v0, device="cuda:0", cap=1_000_000):
    """Force-matching samples from an all-atomistic FP64 run of the same fluid: after 500
    equilibration steps, every pair with COM distance < rc_cg in snapshots 100 steps apart
    until `cap` samples are held.  Returns (feat, target, sim)."""
    import copy

    from paper_1806_10841_gb300 import adress

    s_at = copy.copy(s)
    s_at.d_at = 1e4  # every molecule atomistic
    at = adress.AdResS(s_at, precision="fp64", device=device)
    at.set_state(x0, v0)
    at.compute_forces(energies=False)
    at.step(500)
    n = 0
    while n < cap:
        at.step(100)
        n = at.mlp_collect(cap=cap)
    feat, t, _ = at.mlp_samples(n)
    return feat, t, at


def held_out_rms(sim, feat, t, scale):
    """RMS error of the symmetrised network pair force on held-out samples."""
    sw = feat.copy()
    sw[:, 1:5], sw[:, 5:9] = feat[:, 5:9], feat[:, 1:5]
    pred = 0.5 * scale * (sim.mlp_forward(feat) + sim.mlp_forward(sw))
    return float(math.sqrt(np.mean((pred - t) ** 2)))


def train_network(sim, feat, t, seed=20180628, max_epochs=300, check_every=5, patience=4, radial=False):
    """Standardise, initialise and train the 9-64-64-1 network on 90% of the samples (on the
    GPU, in `sim`), checking the held-out 10% every `check_every` epochs: the learning rate
    halves when the held-out error stops improving, training stops after `patience` checks
    without improvement (or max_epochs), and the best parameters are kept.  radial=True
    switches the eight orientation inputs off (their standardisation divides by 1e30, so the
    network sees zeros there): a network of the COM distance alone."""
    n = len(t)
    rng = np.random.default_rng(seed)
    idx = rng.permutation(n)
    ntr = int(0.9 * n)
    tr, te = idx[:ntr], idx[ntr:]
    mean, std = feat[tr].mean(0), feat[tr].std(0) + 1e-3
    if radial:
        std[1:] = 1e30
    scale = float(t[tr].std())
    params = dict(W1=rng.normal(0, 1 / 3, (64, 9)), b1=np.zeros(64), W2=rng.normal(0, 1 / 8, (64, 64)),
                  b2=np.zeros(64), w3=rng.normal(0, 1 / 8, 64), b3=float(t[tr].mean() / scale))
    sim.mlp_set(params, mean, std, scale)
    sim.mlp_load_samples(feat[tr], t[tr])
    t1 = time.perf_counter()
    lr, epochs, best, best_p, best_epoch, bad, losses, curve = 2e-3, 0, float("inf"), None, 0, 0, [], []
    while epochs < max_epochs:
        losses += [float(v) for v in sim.mlp_train(epochs=check_every, batch=4096, lr=lr)]
        epochs += check_every
        err = held_out_rms(sim, feat[te], t[te], scale)
        curve.append((epochs, err))
        if err < best * (1 - 1e-3):
            best, best_p, best_epoch, bad = err, sim.mlp_get(), epochs, 0
        else:
            bad += 1
            lr *= 0.5
            if bad >= patience:
                break
    sim.mlp_set(best_p, best_p["in_mean"], best_p["in_std"], best_p["out_scale"])
    return {"tr": tr, "te": te, "scale": scale, "losses": losses, "train_s": time.perf_counter() - t1,
            "epochs": epochs, "best_epoch": best_epoch, "held_out_rms": best, "curve": curve}


def learned_arm(s, x0, v0, make, timed, steps, device):
    """FP32 path with the learned CG force: samples from an all-atomistic FP64 run of the
    same fluid, the force-matched CG table from the same samples (the tabulated run the
    network is judged against), GPU training to convergence, then the same timed blocks in
    network mode; structure (COM g(r)) of the network, force-matched-table, LJ-like-table
    and all-atomistic runs."""
    import copy

    from paper_1806_10841_gb300 import adress

    t0 = time.perf_counter()
    feat, t, at = atomistic_samples(s, x0, v0, device=device)
    n = len(t)
    nb, dr = RDF_BINS, RDF_DR

    def rdf_of(sim, eq):
        sim.step(eq)
        c = np.zeros(nb, dtype=np.int64)
        for _ in range(RDF_SNAPS):
            sim.step(RDF_EVERY)
            c += sim.rdf_counts(nb, dr)[0]
        sim.check()
        return adress.AdResS.rdf_normalise(c, s.M, float(np.prod(s.box)), dr, RDF_SNAPS)

    g_at = rdf_of(at, RDF_EQ - 800)  # the sampling run is 800+ steps in already
    # force-matched table from the same samples (GPU), then its own handle
    F_fm, V_fm = at.cg_fit(FIT_DR, FIT_NMIN)
    at.close()
    s_fm = copy.copy(s)
    s_fm.cg_F, s_fm.cg_V = F_fm, V_fm
    sim = make("fp32")
    tn = train_network(sim, feat, t)
    tr, te, scale = tn["tr"], tn["te"], tn["scale"]
    rms = lambda a: float(math.sqrt(np.mean(np.square(a))))
    grid = np.arange(len(s.cg_F)) * s.cg_dr
    d_te = feat[te][:, 0].astype(np.float64)
    err_fm = rms(np.interp(d_te, grid, F_fm) - t[te])
    err_lj = rms(np.interp(d_te, grid, s.cg_F) - t[te])
    prep_s = time.perf_counter() - t0
    sim.set_cg_mode(1)
    sim.set_state(x0, v0)
    sim.compute_forces(energies=False)
    tot, _, _ = timed(sim, steps, 2)
    value = s.N * MD_PER_BLOCK * steps / tot
    # the same network as a slow force of multiple time stepping (evaluated every 4th step)
    p = sim.mlp_get()
    s4 = copy.copy(s)
    s4.respa_n = 4
    sim4 = adress.AdResS(s4, precision="fp32", device=device)
    sim4.mlp_set(p, p["in_mean"], p["in_std"], p["out_scale"])
    sim4.set_cg_mode(1)
    sim4.set_state(x0, v0)
    sim4.compute_forces(energies=False)
    tot4, _, _ = timed(sim4, steps, 2)
    sim4.check()
    sim4.close()
    value_respa4 = s.N * MD_PER_BLOCK * steps / tot4
    # structure: COM g(r) of each run from the initial state after RDF_EQ steps
    sim.set_state(x0, v0)
    sim.compute_forces(energies=False)
    g_net = rdf_of(sim, RDF_EQ)
    sim.close()
    fm = adress.AdResS(s_fm, precision="fp32", device=device)
    fm.set_state(x0, v0)
    fm.compute_forces(energies=False)
    g_fm = rdf_of(fm, RDF_EQ)
    fm.close()
    lj = make("fp32")
    g_lj = rdf_of(lj, RDF_EQ)
    lj.close()
    # the same network on the COM distance alone (orientation inputs off)
    rad = make("fp32")
    tn_r = train_network(rad, feat, t, radial=True)
    rad.set_cg_mode(1)
    rad.set_state(x0, v0)
    rad.compute_forces(energies=False)
    g_rad = rdf_of(rad, RDF_EQ)
    rad.close()
    l2 = lambda a, b: float(math.sqrt(((a - b) ** 2).sum() * dr))
    return {"value": value, "unit": "atom-steps/s", "value_respa4": value_respa4,
            "samples": int(n), "training_samples": int(len(tr)), "held_out": int(len(te)),
            "epochs": tn["epochs"], "best_epoch": tn["best_epoch"], "train_s": tn["train_s"], "prep_s": prep_s,
            "held_out_force_rms": {"target": rms(t[te]), "network": tn["held_out_rms"],
                                   "force_matched_table": err_fm, "lj_table": err_lj,
                                   "network_relative": tn["held_out_rms"] / rms(t[te]),
                                   "radial_network": tn_r["held_out_rms"]},
            "rdf_l2": {"network_vs_force_matched_table": l2(g_net, g_fm), "network_vs_all_atomistic": l2(g_net, g_at),
                       "force_matched_table_vs_all_atomistic": l2(g_fm, g_at),
                       "lj_table_vs_all_atomistic": l2(g_lj, g_at), "network_vs_lj_table": l2(g_net, g_lj),
                       "radial_network_vs_force_matched_table": l2(g_rad, g_fm),
                       "radial_network_vs_all_atomistic": l2(g_rad, g_at),
                       "target": 1e-2,
                       "recipe": f"COM g(r) 0..{nb * dr:g} sigma, dr {dr}, {RDF_SNAPS} snapshots every "
                                 f"{RDF_EVERY} steps after {RDF_EQ} steps from the initial state (AdResS geometry "
                                 "of the benchmark, FP32); L2 = sqrt(sum (g1 - g2)^2 dr)"},
            "source": f"pairs with COM distance < rc_cg from snapshots 100 steps apart of an all-atomistic FP64 run "
                      f"after 500 steps; force-matched table: bins of {FIT_DR} sigma with >= {FIT_NMIN} samples"}


def water_arm(timed, steps, local):
    """The water-like fluid (64,000 flexible three-site molecules, 192,000 atoms; Lennard-Jones
    + reaction-field Coulomb, harmonic bonds and angle; AT 3 nm + 2 x 1.5 nm hybrid), FP32
    mixed and FP64 paths timed on the same bench step, force error of both against the
    oracle on the initial state."""
    import oracle
    from paper_1806_10841_gb300 import adress, inputs

    s = inputs.c3_water()
    x, v = inputs.water_state(s)
    out = {"atoms": s.N, "molecules": s.M, "box_nm": list(s.box), "dt_ps": s.dt}
    f_ref, _ = oracle.Oracle(s).forces(x)
    for prec in ("fp32", "fp64"):
        sim = adress.AdResS(s, precision=prec, device=f"cuda:{local}")
        sim.set_state(x, v)
        fg, _ = sim.forces()
        err = math.sqrt(((fg - f_ref) ** 2).sum() / (f_ref ** 2).sum())
        sim.set_state(x, v)
        sim.compute_forces(energies=False)
        tot, _, _ = timed(sim, steps, 2)
        out[prec] = {"value": s.N * MD_PER_BLOCK * steps / tot, "unit": "atom-steps/s",
                     "force_rel_rms_vs_fp64_oracle": err, "lists": sim.list_stats()}
        sim.close()
    return out


def spheres_arm(timed, steps, local):
    """Self-adjusting geometry on the 800k-atom fluid: the AT region is the union of 16
    spheres (radius 10, hybrid shell 5) around centres drawn in the box, which move by a
    random displacement of 0.1 sigma between bench steps (adress_set_centers; the next step
    rebuilds the lists), FP32 mixed.  A moved region changes the resolution of a molecule in
    the shell at once, by up to (pi / (2 d_hy)) times the displacement; kept that small, two
    overlapping coarse-grained molecules that find themselves at the shell's outer edge get an
    atomistic weight of order 1e-6."""
    import torch

    from paper_1806_10841_gb300 import adress, inputs

    s = inputs.c2_800k()
    s.d_at, s.d_hy = 10.0, 5.0
    s.tf = np.zeros(int(math.ceil((s.d_at + s.d_hy) / s.tf_dx)) + 2)
    rng = np.random.default_rng(20180628)
    L = np.array(s.box)
    s.centers = rng.uniform(0, 1, (16, 3)) * L
    x, v = inputs.tetra_state(s)
    sim = adress.AdResS(s, precision="fp32", device=f"cuda:{local}")
    sim.set_state(x, v)
    sim.compute_forces(energies=False)
    for _ in range(2):
        run_block(sim)
    sim.check()
    c = s.centers.copy()
    ms = []
    for _ in range(steps):
        c = c + rng.normal(0, 0.1 / math.sqrt(3.0), c.shape)
        sim.set_centers(c)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(sim.stream)
        run_block(sim)
        e1.record(sim.stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    sim.check()
    st = sim.list_stats()
    sim.close()
    return {"value": s.N * MD_PER_BLOCK * steps / (sum(ms) / 1e3), "unit": "atom-steps/s", "centers": 16,
            "radius": s.d_at, "hybrid_shell": s.d_hy, "hr_molecules": st["n_hr"],
            "ms_per_bench_step_median": statistics.median(ms)}


def hadress_arm(timed, steps, local):
    """Energy interpolation (H-AdResS) on the 800k-atom fluid: pair weight (l_a + l_b)/2,
    drift force on hybrid molecules, high-resolution band widened by r_list; FP32 mixed,
    the same bench step (thermodynamic-force iteration block), force error against the
    oracle on the initial state."""
    import oracle
    from paper_1806_10841_gb300 import adress, inputs

    s = inputs.c2_800k()
    s.scheme = 1
    x, v = inputs.tetra_state(s)
    f_ref, _ = oracle.Oracle(s).forces(x)
    sim = adress.AdResS(s, precision="fp32", device=f"cuda:{local}")
    sim.set_state(x, v)
    fg, _ = sim.forces()
    err = math.sqrt(((fg - f_ref) ** 2).sum() / (f_ref ** 2).sum())
    sim.set_state(x, v)
    sim.compute_forces(energies=False)
    tot, _, _ = timed(sim, steps, 2)
    st = sim.list_stats()
    sim.close()
    return {"value": s.N * MD_PER_BLOCK * steps / tot, "unit": "atom-steps/s", "precision": "fp32",
            "force_rel_rms_vs_fp64_oracle": err, "hr_molecules": st["n_hr"], "cg_molecules": st["n_cg"]}


def respa_arm(timed, steps, local):
    """Multiple time stepping on the 800k-atom fluid (force interpolation, FP32 mixed): the
    CG pair forces and the thermodynamic force every n-th step with weight n, n = 2 and 4,
    the same bench step; throughput counts inner (atomistic) steps."""
    from paper_1806_10841_gb300 import adress, inputs

    out = {}
    for n in (2, 4):
        s = inputs.c2_800k()
        s.respa_n = n
        x, v = inputs.tetra_state(s)
        sim = adress.AdResS(s, precision="fp32", device=f"cuda:{local}")
        sim.set_state(x, v)
        sim.compute_forces(energies=False)
        tot, _, _ = timed(sim, steps, 2)
        sim.check()
        sim.close()
        out[f"n{n}"] = {"value": s.N * MD_PER_BLOCK * steps / tot, "unit": "atom-steps/s"}
    return out


def replicas_arm(timed, steps, local):
    """64 independent replicas (log-uniform 500..20000 molecules, AT width U(3, 15), hybrid
    U(1, 5)) in one handle: every MD step is one launch over all replicas' molecules, the
    bench step one captured graph.  Timed with the default launch configuration, then after
    the autotuner, and against the same replicas stepped one handle after another."""
    import torch

    from paper_1806_10841_gb300 import adress, inputs

    systems = inputs.replica_batch(64)
    x, v = inputs.replica_states(systems)
    sim = adress.AdResS(systems, precision="fp32", device=f"cuda:{local}")
    sim.set_state(x, v)
    sim.compute_forces(energies=False)
    sim.check()
    n_atoms = sim.N
    t_def, ms_def, _ = timed(sim, steps, 2)
    tuning0 = sim.get_tuning()
    rows = sim.autotune(nsteps=50)
    tuning = sim.get_tuning()
    t_tuned, ms_tuned, clocks = timed(sim, steps, 2)
    sim.close()
    # the same replicas one handle at a time (one graph launch per replica per bench step)
    sims = []
    a0 = np.concatenate([[0], np.cumsum([q.N for q in systems])])
    for r, s in enumerate(systems):
        one = adress.AdResS(s, precision="fp32", device=f"cuda:{local}", replica=r)
        one.set_state(x[a0[r]:a0[r + 1]], v[a0[r]:a0[r + 1]])
        one.compute_forces(energies=False)
        run_block(one)
        sims.append(one)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stream = sims[0].stream
    e0.record(stream)
    for _ in range(steps):
        for one in sims:
            run_block(one)
    e1.record(stream)
    torch.cuda.synchronize()
    t_seq = e0.elapsed_time(e1) / 1e3
    for one in sims:
        one.check()
        one.close()
    per = lambda t: n_atoms * MD_PER_BLOCK * steps / t
    return {"value": per(t_tuned), "unit": "atom-steps/s", "replicas": len(systems), "atoms": n_atoms,
            "molecules_min_median_max": [int(min(q.M for q in systems)), int(statistics.median(q.M for q in systems)),
                                         int(max(q.M for q in systems))],
            "value_default_tuning": per(t_def),
            "tuned_gain": t_def / t_tuned - 1.0,
            "bench_step_ms_default": {"min": min(ms_def), "median": statistics.median(ms_def), "max": max(ms_def)},
            "bench_step_ms_tuned": {"min": min(ms_tuned), "median": statistics.median(ms_tuned), "max": max(ms_tuned)},
            "autotune_default_row": [r for r in rows if (r[0], r[1]) == tuple(tuning0)][:1],
            "autotune_chosen_row": [r for r in rows if (r[0], r[1]) == tuple(tuning)][:1],
            "value_one_handle_per_replica": per(t_seq), "tuning": {"force_block": tuning[0], "skin": tuning[1]},
            "autotune_trials": len(rows), "ms_per_bench_step": t_tuned / steps * 1e3}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-compare", action="store_true", help="skip the FP64 GPU comparison arm")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned-CG-force arm")
    ap.add_argument("--no-replicas", action="store_true", help="skip the 64-replica batch arm")
    ap.add_argument("--no-water", action="store_true", help="skip the water-like fluid arm")
    ap.add_argument("--no-spheres", action="store_true", help="skip the self-adjusting-geometry arm")
    ap.add_argument("--no-hadress", action="store_true", help="skip the energy-interpolation arm")
    ap.add_argument("--no-respa", action="store_true", help="skip the multiple-time-stepping arm")
    ap.add_argument("--profile", type=int, default=0,
                    help="profiling driver: set up, run this many MD steps, exit (no timing output)")
    ap.add_argument("--cg-mode", type=int, default=0, choices=[0, 1],
                    help="for --profile: 1 = learned CG force (network trained on atomistic samples first)")
    ap.add_argument("--water", action="store_true",
                    help="for --profile: the water-like fluid (64k molecules, or --molecules at its density)")
    ap.add_argument("--molecules", type=int, default=200_000,
                    help="system size for --profile (same density, shape and slab proportions)")
    ap.add_argument("--save-state", default=None,
                    help="for --profile: run --equilibrate MD steps from the initial state, save x, v and the "
                         "thermodynamic-force table to this .npz and exit (so that a profiled process can start "
                         "from the equilibrated fluid without hundreds of launches before the captured ones)")
    ap.add_argument("--load-state", default=None, help="for --profile: start from a state saved by --save-state")
    ap.add_argument("--equilibrate", type=int, default=600, help="for --save-state: MD steps (multiple of 100)")
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return reference_arm(args, world, rank)

    import torch

    from paper_1806_10841_gb300 import adress, inputs

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)

    if args.profile:
        if args.water:
            s = inputs.c3_water() if args.molecules == 200_000 else inputs.scaled_c3(args.molecules)
            x0, v0 = inputs.water_state(s)
        else:
            s = inputs.c2_800k() if args.molecules == 200_000 else inputs.scaled_c2(args.molecules)
            x0, v0 = inputs.tetra_state(s)
        sim = adress.AdResS(s, precision=args.precision, device=f"cuda:{local}")
        if args.save_state:
            sim.set_state(x0, v0)
            sim.compute_forces(energies=False)
            for _ in range(max(1, args.equilibrate // MD_PER_BLOCK)):
                sim.run(MD_PER_BLOCK, sample_every=SAMPLE_EVERY, tf_update=True, alpha=TF_ALPHA)
            sim.check()
            xe, ve, _ = sim.get_state()
            np.savez(args.save_state, x=xe, v=ve, tf=sim.get_tf())
            print(json.dumps({"saved": args.save_state, "steps": sim.get_step(), "lists": sim.list_stats()}))
            sim.close()
            return 0
        xi, vi = x0, v0  # the initial state (atomistic samples start from it)
        if args.load_state:
            saved = np.load(args.load_state)
            x0, v0 = saved["x"], saved["v"]
            sim.set_tf(saved["tf"])
        sim.set_state(x0, v0)
        if args.cg_mode:
            # the production network: trained on samples of an all-atomistic run from the
            # initial state (an AdResS state has overlapping atoms in its CG region)
            feat, t, at = atomistic_samples(s, xi, vi, device=f"cuda:{local}")
            at.close()
            train_network(sim, feat, t)
            sim.set_cg_mode(1)
        sim.compute_forces(energies=False)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("md_steps")  # ncu --nvtx --nvtx-include md_steps/ selects these launches
        sim.run(args.profile, sample_every=SAMPLE_EVERY, tf_update=True, alpha=TF_ALPHA)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        sim.check()
        print(json.dumps({"profile_steps": args.profile, "atoms": s.N, "lists": sim.list_stats()}))
        sim.close()
        return 0

    s = inputs.c2_800k(seed=20180628 + rank)
    x0, v0 = inputs.tetra_state(s)

    def make(prec):
        sim = adress.AdResS(s, precision=prec, device=f"cuda:{local}", replica=rank)
        sim.set_state(x0, v0)
        sim.compute_forces(energies=False)
        sim.check()
        return sim

    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def timed(sim, k, w):
        stream = sim.stream
        with Clocks(local) as clk:  # sampling runs from the warm-up on
            for _ in range(w):
                run_block(sim)
            sim.check()
            evs = []
            timed.rebuilds0 = sim.list_stats()["rebuilds"]
            if dist:
                dist.barrier()
            torch.cuda.synchronize()
            t0 = time.time()
            for _ in range(k):
                with torch.cuda.stream(stream):
                    flush.zero_()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                run_block(sim)
                e1.record(stream)
                evs.append((e0, e1))
            torch.cuda.synchronize()
            t1 = time.time()
        if dist:
            dist.barrier()
        sim.check()
        timed.rebuilds = sim.list_stats()["rebuilds"] - timed.rebuilds0  # inside the timed steps
        ms = [a.elapsed_time(b) for a, b in evs]
        return sum(ms) / 1e3, ms, clk.summary(t0, t1)

    sim = make(args.precision)
    total_s, ms, clocks = timed(sim, args.steps, args.warmup)
    rebuilds = timed.rebuilds
    # kernels per bench step (one graph): 1 prologue + 99 fused + 1 last + 100 decide
    # + 10 density samples + 2 for the TF update (update, sample-count reset); 9 kernels
    # per list rebuild (count, 2 scan, fill, sort, 2 scan, lists, dense-cell lists)
    per_block = 1 + (MD_PER_BLOCK - 1) + 1 + MD_PER_BLOCK + MD_PER_BLOCK // SAMPLE_EVERY + 2
    launches = args.steps * per_block + 9 * rebuilds
    value, total_s = job_throughput(total_s, s.N * MD_PER_BLOCK * args.steps, dist, dev)

    # ---- live kernel timing (CUDA events on the library's stream) + roofline ----
    kt = sim.time_kernels(reps=20)
    stats = pair_statistics(s, sim.get_state()[0]) if rank == 0 else None
    # ---- e2e through the public API: pinned host state in, state + KE out, every step ----
    hx = torch.from_numpy(np.ascontiguousarray(x0.T)).pin_memory()
    hv = torch.from_numpy(np.ascontiguousarray(v0.T)).pin_memory()
    hf = torch.empty(sim.f.shape, dtype=sim.f.dtype).pin_memory()
    hf.copy_(sim.f.cpu())
    ox = torch.empty_like(hx).pin_memory()
    ov = torch.empty_like(hv).pin_memory()
    e2e_steps = max(2, min(args.steps, 5))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        with torch.cuda.stream(sim.stream):
            sim.x.copy_(hx, non_blocking=True)
            sim.v.copy_(hv, non_blocking=True)
            sim.f.copy_(hf, non_blocking=True)
        sim.build_lists()
        run_block(sim)
        with torch.cuda.stream(sim.stream):
            ox.copy_(sim.x, non_blocking=True)
            ov.copy_(sim.v, non_blocking=True)
        ke, _ = sim.kinetic()
    sim.check()
    e2e_s = time.perf_counter() - t0
    h2d = hx.numel() * 8 + hv.numel() * 8 + hf.numel() * hf.element_size()
    d2h = ox.numel() * 8 + ov.numel() * 8 + 4 * 8

    compare = None
    if not args.no_compare and rank == 0:
        other = "fp64" if args.precision == "fp32" else "fp32"
        sim.close()
        sim2 = make(other)
        t2, _, _ = timed(sim2, max(2, args.steps // 2), 2)
        compare = {"precision": other,
                   "value": s.N * MD_PER_BLOCK * max(2, args.steps // 2) / t2,
                   "unit": "atom-steps/s"}
        # force error of both GPU paths against the FP64 oracle on the initial state
        import oracle

        f_ref, _ = oracle.Oracle(s).forces(x0)
        errs = {}
        for prec, sm in ((other, sim2),):
            sm.set_tf(np.zeros(sm.tf_n))
            sm.set_state(x0, v0)
            fg, _ = sm.forces()
            errs[prec] = math.sqrt(((fg - f_ref) ** 2).sum() / (f_ref ** 2).sum())
        sim2.close()
        sim3 = make(args.precision)
        fg, _ = sim3.forces()
        errs[args.precision] = math.sqrt(((fg - f_ref) ** 2).sum() / (f_ref ** 2).sum())
        sim3.close()
        compare["force_rel_rms_vs_fp64_oracle"] = errs
    else:
        sim.close()

    learned = None
    if not args.no_learned and rank == 0:
        learned = learned_arm(s, x0, v0, make, timed, max(2, args.steps // 2), f"cuda:{local}")

    replicas = None
    if not args.no_replicas and rank == 0:
        replicas = replicas_arm(timed, max(2, args.steps // 2), local)
    water = None
    if not args.no_water and rank == 0:
        water = water_arm(timed, max(2, args.steps // 2), local)
    spheres = None
    if not args.no_spheres and rank == 0:
        spheres = spheres_arm(timed, max(2, args.steps // 2), local)
    hadress = None
    if not args.no_hadress and rank == 0:
        hadress = hadress_arm(timed, max(2, args.steps // 2), local)
    respa = None
    if not args.no_respa and rank == 0:
        respa = respa_arm(timed, max(2, args.steps // 2), local)

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return 0

    pk, src = peaks()
    sm_mhz = clocks.get("sm_mhz") or 2070.0
    # Dominant kernel: the fused step kernel (forces of Eq. 1 + bonded + TF + thermostat +
    # both half kicks + drift + next mapping).  Algorithmic work per launch, per atom: the
    # state crosses HBM once (x, v read and written in FP64, 96 B, and the FP32 force,
    # 12 B, plus ~2 B of molecule records): 110 B per atom-step.
    flops32 = (stats["at_pairs"] * FLOPS["at_pair"] + stats["cg_pairs"] * FLOPS["cg_pair"]
               + stats["bonds"] * FLOPS["bond"])
    fp64_per_atom = 12  # v += 2h f and x += dt v: 6 FMA = 12 flops
    f64_flops = s.N * fp64_per_atom
    step_bytes = s.N * ALGO_BYTES_PER_ATOM
    # this implementation's own layout moves more: double-buffered float4 offsets (read +
    # write) and molecule records (int4 centre + float2 region data, read + write)
    off_b = 16 if args.precision == "fp32" else 32
    mol_b = 24 if args.precision == "fp32" else 56
    layout_bytes = s.N * (4 * 24 + 2 * off_b) + s.M * 2 * mol_b
    t_step = kt["step"] * 1e-3
    fp32_peak = 152 * 128 * 2 * sm_mhz * 1e6 / 1e12   # TFLOP/s, unit counts x sampled clock
    fp64_peak = 152 * 4 * sm_mhz * 1e6 / 1e12          # 2 DFMA/clk/SM, unit counts x sampled clock
    hbm_peak = float(pk.get("hbm_gbs", 6800.0))
    achieved = step_bytes / t_step / 1e9
    traffic = (profiled_traffic("k_step_fused_c2_800k_fp32.md", ("step_impl.cuh", "step.cu", "internal.cuh"))
               if args.precision == "fp32" else None)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s", "frac": achieved / hbm_peak,
                "traffic": traffic,
                "kernel": "k_step fused (forces + bonded + TF + Langevin + kicks + drift + mapping)",
                "algorithmic_bytes_per_launch": step_bytes, "bytes_per_atom": ALGO_BYTES_PER_ATOM,
                "ms_per_launch": kt["step"], "peak_source": f"{src} HBM copy bandwidth (MEASURED_PEAKS.json)",
                "layout_bytes_per_launch": layout_bytes, "layout_frac": layout_bytes / t_step / 1e9 / hbm_peak,
                "fp32_alu": {"achieved_tflops": flops32 / t_step / 1e12, "peak_tflops": fp32_peak,
                             "frac": flops32 / t_step / 1e12 / fp32_peak,
                             "peak_source": f"152 SMs x 128 lanes x 2 x {sm_mhz:.0f} MHz (sampled)"},
                "fp64_alu": {"achieved_tflops": f64_flops / t_step / 1e12, "peak_tflops": fp64_peak,
                             "frac": f64_flops / t_step / 1e12 / fp64_peak,
                             "peak_source": f"152 SMs x 2 DFMA/clk x 2 x {sm_mhz:.0f} MHz (sampled)"},
                "traffic_source": "profiles/k_step_fused_c2_800k_fp32.md (one ncu capture, cold cache; "
                                  "null when the kernel's sources changed since)"}
    line = {
        "metric": METRIC, "value": value, "unit": "atom-steps/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_s / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 forces / f64 state" if args.precision == "fp32" else "f64",
        "data": "synthetic (seeded lattice + jitter, random orientations, Maxwell-Boltzmann)",
        "config": {"workload": CONFIG_NAME, "atoms": s.N, "molecules": s.M,
                   "md_steps_per_bench_step": MD_PER_BLOCK, "density_samples_per_bench_step": MD_PER_BLOCK // SAMPLE_EVERY,
                   "tf_updates_per_bench_step": 1, "l2": "flushed (512 MB write) between timed bench steps",
                   "parallelism": f"replicas x{world}"},
        "e2e": {"value": s.N * MD_PER_BLOCK * e2e_steps / e2e_s, "unit": "atom-steps/s",
                "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": launches,
        "roofline": roofline,
        "clocks": clocks,
        "bench_step_ms": {"min": min(ms), "median": statistics.median(ms), "max": max(ms)},
        "kernel_ms": kt,
        "pair_stats": stats,
        "replicas_64": replicas,
        "water_64k": water,
        "spheres_16": spheres,
        "energy_interpolation": hadress,
        "multiple_time_stepping": respa,
    }
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_sample(s, x0, v0)
    # the metric's comparison (the plain FP64 GPU path) and the learned arm last, so that a
    # reader of the line's tail has them
    line["learned_cg"] = learned
    line["compare"] = compare
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
