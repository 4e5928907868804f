"""Slab domain decomposition (Sec. 5.5) with the library's kernels as the local operations.

Two ranks (gloo, host-staged halo exchange) share cuda:0: each sets up a
context on its slab plus ghost elements and runs paper_1808_03595_gb300.slab
with LibraryLocalOps.  The ranks synchronise on the host only (no kernel
waits on another rank), and their solve must equal the library's
single-domain solve: the same iteration count and the same solution to 1e-10.
"""
import os
import socket

import numpy as np
import pytest

import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _local(x, slab, q):
    idx = [slice(None)] * 3
    idx[slab.dim] = slice(slab.e0 * q, slab.e1 * q + 1)
    return np.ascontiguousarray(x[tuple(idx)])


def _owned(x, slab, q):
    lo, hi = slab.own_planes(q)
    idx = [slice(None)] * 3
    idx[slab.dim] = slice(lo, hi)
    return np.asarray(x)[tuple(idx)]


def _rank_main(rank, world, port, axis, p, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist

    from paper_1808_03595_gb300 import Context
    from paper_1808_03595_gb300.slab import DistributedMG, LibraryLocalOps, Slab, level_degrees
    torch.cuda.set_device(0)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        h = workloads.stretched_widths(4, 23)
        lam, p0 = 1.0, 2
        f = workloads.random_nodal(h, p, 9, "uniform")
        slab = Slab(h, axis, world, rank)
        with Context(h, p, lam, p0=p0) as g:  # the single-domain reference and the global coarse solve
            fd = torch.as_tensor(f, device="cuda")
            u_ref, info = g.solve(fd)
            Fh = g.unpack(g.L, g.condense_rhs(fd), out=torch.zeros(g.nodal_shape(), dtype=torch.float64,
                                                                      device="cuda"))
            with Context(h, p0, lam, p0=p0) as c0, Context(slab.local_h, p, lam, p0=p0, bc=slab.local_bc) as c:
                dm = DistributedMG(slab, LibraryLocalOps(c, c0), level_degrees(p, p0), c0.nodal_shape(0))
                F_loc = torch.as_tensor(_local(Fh.cpu().numpy(), slab, p), device="cuda")
                uu, it, hist = dm.solve(F_loc)
                assert it == info.iters, (it, info.iters)
                assert hist[-1] <= 1e-10 * hist[0]
                # the skeleton of the single-domain solution, at the owned nodes
                uref_hat = g.unpack(g.L, g.pack(g.L, u_ref), out=torch.zeros_like(u_ref)).cpu().numpy()
                a = _owned(uu.cpu().numpy(), slab, p)
                b = _owned(_local(uref_hat, slab, p), slab, p)
                err = np.abs(a - b).max() / np.abs(b).max()
                assert err < 1e-10, err
        open(os.path.join(out_dir, f"ok{rank}"), "w").write(f"{it} {err:.2e}\n")
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("axis", [0, 2])
def test_slab_decomposition_with_the_library(axis, tmp_path):
    import torch.multiprocessing as mp
    mp.spawn(_rank_main, args=(2, _free_port(), axis, 8, str(tmp_path)), nprocs=2, join=True)
    assert sorted(os.listdir(tmp_path)) == ["ok0", "ok1"]
