"""Slab decomposition with the library as the local force engine: two ranks (processes with
a gloo group for their messages) share one GPU, each computing its molecules' forces with
its own handle; the assembled forces equal the oracle's for the whole box (FP64 1e-10,
FP32 2e-5).  The ranks' kernels never wait on each other: every exchange goes through host
messages between force evaluations."""
import os
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, mode, precision, q):
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import torch.distributed as dist

    from paper_1806_10841_gb300 import slabs
    from test_slabs import _case

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        s, x, _ = _case()
        L = float(s.box[0])
        cx = slabs.com_x(x, s.na, s.mass, L)
        cls = slabs.resolution_class(cx, L, s.xc, s.d_at, s.d_hy)
        halo = slabs.halo_width(s)
        bounds = slabs.balance_bounds(cx, cls, L, world, slabs.cost_per_class(8.0, 1.0), halo)
        dec = slabs.SlabDecomposition(s, bounds, halo, mode=mode)
        mine = np.nonzero(slabs.owner_of(cx, bounds) == rank)[0]
        eng = slabs.LibraryEngine(s, mode=mode, precision=precision)
        f, _ = dec.forces(mine, x.reshape(s.M, s.na, 3)[mine].reshape(-1, 3), eng)
        eng.close()
        out = [None] * world
        dist.all_gather_object(out, dict(owned=mine, f=f))
        if rank == 0:
            q.put(out)
    finally:
        dist.barrier()
        dist.destroy_process_group()


@pytest.mark.parametrize("mode,precision", [("half_shell", "fp64"), ("full_shell", "fp32"), ("half_shell", "fp32")])
def test_library_engine_decomposition_matches_the_oracle(mode, precision):
    import torch.multiprocessing as mp

    import oracle
    from test_slabs import _case, _free_port

    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, mode, precision, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = q.get(timeout=600)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    s, x, _ = _case()
    f_ref, _ = oracle.Oracle(s).forces(x)
    f = np.zeros_like(f_ref)
    for o in out:
        f.reshape(s.M, s.na, 3)[o["owned"]] = o["f"].reshape(-1, s.na, 3)
    rel = np.sqrt(((f - f_ref) ** 2).sum() / (f_ref ** 2).sum())
    assert rel < (1e-10 if precision == "fp64" else 2e-5), rel


def test_measured_class_costs():
    from paper_1806_10841_gb300 import inputs, slabs

    c = slabs.measure_class_costs(inputs.c2_800k(), molecules=20000)
    assert c[0] == c[1] and c[0] > c[2] > 0
