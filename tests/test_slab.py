"""Slab domain decomposition (Sec. 5.5) over gloo ranks on the CPU.

Each rank holds its slab of elements plus one ghost element per shared side
and runs paper_1808_03595_gb300.slab with the oracle's matrix-free operations
as its local operations.  Checked against the oracle on the whole mesh:
  - the condensed operator and the star smoother at the owned nodes (halo
    exchange of the ghost element, then the local operation): 1e-12;
  - Algorithms 3 and 4 over the ranks: the same iteration count as the
    single-domain solve, the same solution to 1e-10.
For 2 and 3 ranks, split along x1 (as the paper's decomposition) and along x3.
"""
import os
import socket

import numpy as np
import pytest

import workloads
from oracle import dense, matfree

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


class OracleOps:
    """The oracle's matrix-free operations on a slab's local mesh (LocalOps of slab.DistributedMG)."""

    def __init__(self, slab, p, lam, p0, global_h, bc):
        from paper_1808_03595_gb300.slab import level_degrees
        self.degs = level_degrees(p, p0)
        self.meshes = [dense.Mesh(slab.local_h, q, lam, slab.local_bc) for q in self.degs]
        self.tables = [matfree.StarTables(m) if l > 0 else None for l, m in enumerate(self.meshes)]
        self.coarse_solver = matfree.CoarseSolver(dense.Mesh(global_h, p0, lam, bc))

    def apply(self, l, u):
        return torch.from_numpy(matfree.apply_condensed(self.meshes[l], u.numpy()))

    def smooth(self, l, r):
        return torch.from_numpy(matfree.smooth(self.meshes[l], r.numpy(), self.tables[l]))

    def restrict(self, l, r):
        return torch.from_numpy(matfree.restrict(self.meshes[l], self.meshes[l - 1], r.numpy()))

    def prolong(self, l, uc):
        return torch.from_numpy(matfree.prolong(self.meshes[l - 1], self.meshes[l], uc.numpy()))

    def mask(self, l):
        return torch.from_numpy(matfree.condensed_mask(self.meshes[l]))

    def coarse(self, F0):
        return torch.from_numpy(self.coarse_solver.solve(F0.numpy()))


def _local(x, slab, q):
    """The local planes (own + ghost elements) of a global nodal array at degree q."""
    idx = [slice(None)] * 3
    idx[slab.dim] = slice(slab.e0 * q, slab.e1 * q + 1)
    return np.ascontiguousarray(x[tuple(idx)])


def _owned(x, slab, q):
    lo, hi = slab.own_planes(q)
    idx = [slice(None)] * 3
    idx[slab.dim] = slice(lo, hi)
    return np.asarray(x)[tuple(idx)]


def _rank_main(rank, world, port, axis, case):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist

    from paper_1808_03595_gb300.slab import DistributedMG, Slab, level_degrees
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        h, p, lam, bc, p0 = case
        mesh = dense.Mesh(h, p, lam, bc)
        slab = Slab(h, axis, world, rank, bc)
        ops = OracleOps(slab, p, lam, p0, h, bc)
        degs = level_degrees(p, p0)
        dm = DistributedMG(slab, ops, degs, dense.Mesh(h, p0, lam, bc).shape)
        L = len(degs) - 1
        mask = matfree.condensed_mask(mesh)
        u = np.where(mask, workloads.random_nodal(h, p, 7), 0.0)
        # operator and smoother at the owned nodes
        y = dm.apply(L, torch.from_numpy(_local(u, slab, p))).numpy()
        y_ref = matfree.apply_condensed(mesh, u)
        scale = np.abs(y_ref).max()
        assert np.abs(_owned(y, slab, p) - _owned(_local(y_ref, slab, p), slab, p)).max() <= 1e-12 * scale
        d = dm.smooth(L, torch.from_numpy(_local(u, slab, p))).numpy()
        d_ref = matfree.smooth(mesh, u)
        scale = np.abs(d_ref).max()
        assert np.abs(_owned(d, slab, p) - _owned(_local(d_ref, slab, p), slab, p)).max() <= 1e-12 * scale
        # Algorithm 4 over the ranks against the single-domain oracle
        f = workloads.random_nodal(h, p, 8, "uniform")
        Fh = matfree.condense_rhs(mesh, f)
        u_ref, it_ref, _ = matfree.mg_solve(matfree.MG(mesh, p0), Fh)
        uu, it, hist = dm.solve(torch.from_numpy(_local(Fh, slab, p)))
        assert it == it_ref, (it, it_ref)
        assert hist[-1] <= 1e-10 * hist[0]
        scale = np.abs(u_ref).max()
        err = np.abs(_owned(uu.numpy(), slab, p) - _owned(_local(u_ref, slab, p), slab, p)).max()
        assert err <= 1e-10 * scale, err
    finally:
        dist.destroy_process_group()


CASES = {
    "uniform_4x3x3_p4": ([np.full(4, 0.25), np.full(3, 1 / 3), np.full(3, 1 / 3)], 4, 1.0, ("D",) * 6, 2),
    "stretched_neumann_p6": (workloads.stretched_widths(4, 17), 6, 2.0, ("D", "D", "N", "D", "D", "N"), 2),
}


@pytest.mark.parametrize("world", [2, 3])
@pytest.mark.parametrize("axis", [0, 2])
@pytest.mark.parametrize("case", sorted(CASES))
def test_slab_decomposition_matches_single_domain(world, axis, case):
    import torch.multiprocessing as mp
    h, p, lam, bc, p0 = CASES[case]
    if len(h[axis]) < world:
        pytest.skip("fewer elements than ranks along the split axis")
    mp.spawn(_rank_main, args=(world, _free_port(), axis, CASES[case]), nprocs=world, join=True)


def test_slab_partition_and_halo_plan():
    from paper_1808_03595_gb300.slab import Slab
    h = [np.full(7, 1 / 7), np.full(2, 0.5), np.full(2, 0.5)]
    p = 4
    owned = []
    for rank in range(3):
        s = Slab(h, 0, 3, rank)
        assert s.a1 - s.a0 in (2, 3) and len(s.local_h[0]) == s.a1 - s.a0 + s.gl + s.gr
        assert s.local_bc[0] == ("D" if rank == 0 else "N") and s.local_bc[1] == ("D" if rank == 2 else "N")
        lo, hi = s.own_planes(p)
        owned += [s.global_plane(p, i) for i in range(lo, hi)]
        for nb, (slo, shi), (rlo, rhi) in s.halo_plan(p):
            # what I send is what the neighbour receives, plane for plane (global indices)
            t = Slab(h, 0, 3, nb)
            back = [(a, b) for n2, a, b in t.halo_plan(p) if n2 == rank][0]
            assert [s.global_plane(p, i) for i in range(slo, shi)] == \
                [t.global_plane(p, i) for i in range(back[1][0], back[1][1])]
            # the received planes fill every local plane that is not owned
            assert (rlo < lo) == (nb < rank)
    assert owned == list(range(7 * p + 1))  # every global plane has exactly one owner
