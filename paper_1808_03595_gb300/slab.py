"""Slab domain decomposition of the p-multigrid solver over ranks (Sec. 5.5).

The elements are split along one axis into contiguous slabs, one per rank,
and every rank keeps one ghost element beyond each side it shares with a
neighbour.  Rank s owns the node planes g (global index along the axis) with
a0 p < g <= a1 p of its elements a0..a1-1 (rank 0 also owns g = 0), at every
level of the hierarchy; the interface plane belongs to the rank on its left.

With the ghost layer in place, the condensed operator and the star smoother of
a rank's local mesh are exact at the nodes it owns: every element touching an
owned node, and every star whose weight reaches one, lies inside own + ghost
elements (a star centred on vertex plane c spans the elements c-1 and c, and
its weights vanish one element away from c).  So each application is
  1. a halo exchange that copies the neighbours' owned planes into the ghost
     element (p + 1 planes from the left neighbour, p from the right one);
  2. the local operation (the library's kernels on the local mesh, or any
     other implementation of LocalOps);
  3. its result kept on the owned planes only.
Restriction and prolongation interpolate face by face, and a face's values
depend on the edges and vertices that bound it, which may lie on a
neighbour's plane; so they take the same halo exchange first (the fine
residual before restricting, the coarse correction before prolonging), and
are then exact at the owned nodes too.  The coarse problem is summed from the owned parts
(all-reduce) and solved on every rank.  The local mesh has the global boundary
conditions, except on a face beyond a ghost element, which is Neumann: the
nodes there stay unknowns whose (exchanged) values enter the local operator.

Algorithms 3 and 4 then run unchanged on the owned parts; norms and dot
products are sums of the owned parts (all-reduce).  The exchange uses
torch.distributed point-to-point messages of contiguous host or device
buffers; nothing here reads another rank's memory directly.
"""
import numpy as np
import torch
import torch.distributed as dist


def level_degrees(p, p0):
    """Degrees of the hierarchy (Sec. 4.1): p0 2^l while below p, then p."""
    degs = [p0]
    while degs[-1] * 2 < p:
        degs.append(degs[-1] * 2)
    if degs[-1] != p:
        degs.append(p)
    return degs


class Slab:
    """The part of a tensor-product mesh that rank `rank` of `world` holds (split along `axis`).

    h: per-axis element widths (global); bc: the six global face conditions ("D", "N"; a periodic
    split axis is not supported).  local_h / local_bc describe the local mesh (own elements plus
    ghosts); own_planes(q) and the exchange plan are in local node-plane indices along the axis.
    """

    def __init__(self, h, axis, world, rank, bc=None):
        self.axis = int(axis)
        self.world, self.rank = int(world), int(rank)
        self.bc = tuple(bc) if bc is not None else ("D",) * 6
        if self.bc[2 * self.axis] == "P":
            raise ValueError("slab decomposition: the split axis cannot be periodic")
        n = len(h[self.axis])
        counts = [n // world + (1 if r < n % world else 0) for r in range(world)]
        if min(counts) < 1:
            raise ValueError(f"slab decomposition: {n} elements along axis {axis} for {world} ranks")
        self.a0 = sum(counts[:rank])
        self.a1 = self.a0 + counts[rank]
        self.gl = 1 if rank > 0 else 0
        self.gr = 1 if rank < world - 1 else 0
        self.e0, self.e1 = self.a0 - self.gl, self.a1 + self.gr  # local elements (with ghosts)
        self.global_h = [np.asarray(x, dtype=float) for x in h]
        self.local_h = [x.copy() for x in self.global_h]
        self.local_h[self.axis] = self.global_h[self.axis][self.e0:self.e1].copy()
        lb = list(self.bc)
        if self.gl:
            lb[2 * self.axis] = "N"
        if self.gr:
            lb[2 * self.axis + 1] = "N"
        self.local_bc = tuple(lb)

    # array dimension of the split axis in a nodal array [g3][g2][g1]
    @property
    def dim(self):
        return 2 - self.axis

    def own_planes(self, q):
        """Local plane indices [lo, hi) owned at degree q."""
        lo = (self.a0 - self.e0) * q + (0 if self.rank == 0 else 1)
        hi = (self.a1 - self.e0) * q + 1
        return lo, hi

    def global_plane(self, q, local_index):
        return self.e0 * q + local_index

    def halo_plan(self, q):
        """[(neighbour, send [lo, hi), receive [lo, hi))] in local plane indices at degree q."""
        plan = []
        if self.gl:  # left neighbour: it needs my planes (a0 q, (a0 + 1) q]; I need its [(a0 - 1) q, a0 q]
            base = (self.a0 - self.e0) * q
            plan.append((self.rank - 1, (base + 1, base + q + 1), (base - q, base + 1)))
        if self.gr:  # right neighbour: it needs my [(a1 - 1) q, a1 q]; I need its (a1 q, (a1 + 1) q]
            base = (self.a1 - self.e0) * q
            plan.append((self.rank + 1, (base - q, base + 1), (base + 1, base + q + 1)))
        return plan


def _planes(x, dim, lo, hi):
    idx = [slice(None)] * 3
    idx[dim] = slice(lo, hi)
    return x[tuple(idx)]


class DistributedMG:
    """Algorithms 3 and 4 on a slab of the mesh, with halo exchanges over a process group.

    ops: the local operations on the slab's local mesh, per level l (0 = coarsest), on nodal
    condensed arrays (torch tensors shaped like the local nodal grid at that level):
      ops.apply(l, u)        Hhat_l u
      ops.smooth(l, r)       Smoother_l(r) (Algorithm 2 on the local mesh)
      ops.restrict(l, r)     J^T r from level l to level l - 1
      ops.prolong(l, uc)     J uc from level l - 1 to level l
      ops.mask(l)            condensed-unknown mask of the local mesh (bool tensor)
      ops.coarse(F0)         exact solve of the GLOBAL coarse problem; F0, result: global nodal arrays
    degs: the level degrees; global_shape0: the global nodal shape at level 0.
    """

    def __init__(self, slab, ops, degs, global_shape0, group=None):
        self.s, self.ops, self.degs = slab, ops, list(degs)
        self.group = group
        self.global_shape0 = tuple(global_shape0)
        self.L = len(self.degs) - 1
        # gloo moves host buffers: device data is staged through host copies
        self.stage = dist.get_backend(group) == "gloo"

    def _out(self, t):
        return t.cpu() if self.stage else t

    def _back(self, t, like):
        return t.to(like.device) if self.stage else t

    # ---- communication
    def halo(self, l, x):
        """Copy the neighbours' owned planes into this rank's ghost planes (in place), level l."""
        q, d = self.degs[l], self.s.dim
        reqs, recv = [], []
        for nb, (slo, shi), (rlo, rhi) in self.s.halo_plan(q):
            buf = self._out(_planes(x, d, slo, shi).contiguous())
            rbuf = torch.empty_like(self._out(_planes(x, d, rlo, rhi).contiguous()))
            reqs.append(dist.isend(buf, nb, group=self.group))
            reqs.append(dist.irecv(rbuf, nb, group=self.group))
            recv.append((rlo, rhi, rbuf))
        for r in reqs:
            r.wait()
        for rlo, rhi, rbuf in recv:
            _planes(x, d, rlo, rhi).copy_(self._back(rbuf, x))
        return x

    def own(self, l, x):
        """x on the owned planes, zero elsewhere (and off the condensed unknowns)."""
        lo, hi = self.s.own_planes(self.degs[l])
        out = torch.zeros_like(x)
        _planes(out, self.s.dim, lo, hi).copy_(_planes(x, self.s.dim, lo, hi))
        return torch.where(self.ops.mask(l), out, torch.zeros_like(out))

    def dot(self, l, x, y):
        v = self._out(torch.sum(self.own(l, x) * y).reshape(1).to(torch.float64))
        dist.all_reduce(v, group=self.group)
        return float(v.item())

    def norm(self, l, x):
        return self.dot(l, x, x) ** 0.5

    # ---- distributed operations (owned results)
    def apply(self, l, u):
        return self.own(l, self.ops.apply(l, self.halo(l, u.clone())))

    def smooth(self, l, r):
        return self.own(l, self.ops.smooth(l, self.halo(l, r.clone())))

    def coarse(self, F0):
        """Owned coarse right-hand sides summed into the global array, solved on every rank."""
        g = torch.zeros(self.global_shape0, dtype=F0.dtype, device=F0.device)
        lo, hi = self.s.own_planes(self.degs[0])
        q0 = self.degs[0]
        glo, ghi = self.s.global_plane(q0, lo), self.s.global_plane(q0, hi)
        _planes(g, self.s.dim, glo, ghi).copy_(_planes(self.own(0, F0), self.s.dim, lo, hi))
        gs = self._out(g)
        dist.all_reduce(gs, group=self.group)
        U = self.ops.coarse(self._back(gs, g))
        n_local = F0.shape[self.s.dim]
        g0 = self.s.global_plane(q0, 0)
        return self.own(0, _planes(U, self.s.dim, g0, g0 + n_local).clone())

    # ---- Algorithms 3 and 4
    def vcycle(self, u, F):
        """Algorithm 3 on the owned parts: u_L, F_L local nodal arrays at the finest level."""
        L = self.L
        ul, Fl = [None] * (L + 1), [None] * (L + 1)
        ul[L], Fl[L] = u.clone(), F
        for l in range(L, 0, -1):
            if l != L:
                ul[l] = torch.zeros_like(Fl[l])
            ul[l] = ul[l] + self.smooth(l, Fl[l] - self.apply(l, ul[l]))
            Fl[l - 1] = self.own(l - 1, self.ops.restrict(l, self.halo(l, Fl[l] - self.apply(l, ul[l]))))
        ul[0] = self.coarse(Fl[0])
        for l in range(1, L + 1):
            ul[l] = ul[l] + self.own(l, self.ops.prolong(l, self.halo(l - 1, ul[l - 1].clone())))
            ul[l] = ul[l] + self.smooth(l, Fl[l] - self.apply(l, ul[l]))
        return ul[L]

    def solve(self, Fhat, rtol=1e-10, maxit=50):
        """Algorithm 4 from u = 0: (owned u, iterations, residual-norm history)."""
        L = self.L
        F = self.own(L, Fhat)
        u = torch.zeros_like(F)
        r = F - self.apply(L, u)
        hist = [self.norm(L, r)]
        it = 0
        while hist[-1] > rtol * hist[0] and it < maxit:
            u = self.vcycle(u, F)
            r = F - self.apply(L, u)
            hist.append(self.norm(L, r))
            it += 1
        return u, it, hist


class LibraryLocalOps:
    """LocalOps backed by the semmg library on the slab's local mesh (device nodal arrays, FP64).

    ctx: a Context on the local mesh (slab.local_h, slab.local_bc); coarse_ctx: a Context on the
    global mesh at the coarse degree (only its level-0 coarse solve is used)."""

    def __init__(self, ctx, coarse_ctx):
        self.c, self.c0 = ctx, coarse_ctx
        self._mask = {}

    def _hat(self, l, x):
        return self.c.pack(l, x.contiguous())

    def _nodal(self, l, xh):
        return self.c.unpack(l, xh, out=torch.zeros(self.c.nodal_shape(l), dtype=torch.float64, device=xh.device))

    def apply(self, l, u):
        return self._nodal(l, self.c.apply_condensed(l, self._hat(l, u)))

    def smooth(self, l, r):
        return self._nodal(l, self.c.smooth(l, self._hat(l, r)))

    def restrict(self, l, r):
        return self._nodal(l - 1, self.c.restrict(l, self._hat(l, r)))

    def prolong(self, l, uc):
        fine = torch.zeros(self.c.condensed_size(l), dtype=torch.float64, device=uc.device)
        return self._nodal(l, self.c.prolong_add(l, self._hat(l - 1, uc), fine))

    def mask(self, l):
        if l not in self._mask:
            one = torch.ones(self.c.nodal_shape(l), dtype=torch.float64, device="cuda")
            self._mask[l] = self._nodal(l, self._hat(l, one)) != 0.0
        return self._mask[l]

    def coarse(self, F0):
        g = self.c0.coarse_solve(self.c0.pack(0, F0.contiguous()))
        return self.c0.unpack(0, g, out=torch.zeros(self.c0.nodal_shape(0), dtype=torch.float64, device=F0.device))
