"""Neumann and periodic boundaries (Sec. 3.3) on the CUDA path, against the FP64 oracle.

Every face of the domain is Dirichlet or Neumann on its own, or an axis is
periodic; at a Neumann face the boundary nodes are unknowns, the ghost element
beyond it is decoupled (identity padding of the star tables) and the operator
loses the missing element's contributions; on a periodic axis the ghost element
is the element at the other end and the last node plane repeats the first.
Same tolerances as the Dirichlet parity tests.
"""
import numpy as np
import pytest

import workloads
from oracle import dense, matfree

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 2e-5

MIXED_BC = ("N", "D", "D", "N", "N", "N")
NEUMANN = ("N",) * 6
BCS = {"mixed": MIXED_BC, "neumann": NEUMANN, "alt": ("D", "N", "N", "D", "N", "D"),
       "per": ("P", "P", "N", "D", "P", "P"), "perall": ("P",) * 6, "perd": ("D", "D", "P", "P", "D", "N")}
MESHES = {
    "stretched_3x2x2": [np.array([0.2, 0.5, 0.3]), np.array([0.7, 0.3]), np.array([0.4, 0.6])],
    "uniform_3": workloads.uniform_widths(3),
    "thin_2x1x2": [np.array([0.6, 0.4]), np.array([0.5]), np.array([1.0, 1.0])],
}


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1808_03595_gb300 import build
    build.build()


def ctx(h, p, lam, bc, **kw):
    from paper_1808_03595_gb300 import Context
    return Context(h, p, lam, bc=bc, **kw)


def cuda(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def rel(a, b):
    b = np.asarray(b)
    return float(np.abs(np.asarray(a) - b).max() / max(np.abs(b).max(), 1e-300))


def skel_random(m, seed):
    h = m.h
    return np.where(matfree.condensed_mask(m), workloads.random_nodal(h, m.p, seed), 0.0)


def to_nodal(c, level, hat):
    torch.cuda.synchronize()
    return c.unpack(level, hat).cpu().numpy()


@pytest.mark.parametrize("mesh_name,bc,p,lam", [("stretched_3x2x2", "mixed", 4, 0.0), ("uniform_3", "neumann", 5, 1.0),
                                                ("thin_2x1x2", "alt", 8, 2.0), ("uniform_3", "mixed", 16, 0.5),
                                                ("stretched_3x2x2", "per", 4, 0.0), ("uniform_3", "perall", 8, 1.0),
                                                ("uniform_3", "perd", 16, 0.0), ("uniform_3", "perall", 12, 1.0),
                                                ("thin_2x1x2", "alt", 13, 2.0), ("stretched_3x2x2", "per", 14, 0.0)])
def test_apply_condensed_and_pack(mesh_name, bc, p, lam):
    h = MESHES[mesh_name]
    m = dense.Mesh(h, p, lam, BCS[bc])
    u = skel_random(m, 11)
    ref = matfree.apply_condensed(m, u)
    mask = matfree.condensed_mask(m)
    with ctx(h, p, lam, BCS[bc]) as c:
        uh = c.pack(c.L, cuda(u))
        back = to_nodal(c, c.L, uh)
        y = to_nodal(c, c.L, c.apply_condensed(c.L, uh))
    assert np.array_equal(back[mask], u[mask])  # Neumann boundary nodes are stored unknowns
    assert rel(y[mask], ref[mask]) < TOL64
    if p <= 5:
        cond = dense.Condensed(m)
        assert rel(y.ravel()[cond.B], cond.Hhat @ u.ravel()[cond.B]) < TOL64


@pytest.mark.parametrize("mesh_name,bc,p,lam", [("stretched_3x2x2", "mixed", 3, 0.0), ("uniform_3", "neumann", 4, 1.0),
                                                ("thin_2x1x2", "alt", 8, 2.0), ("uniform_3", "mixed", 16, 0.5),
                                                ("stretched_3x2x2", "neumann", 11, 3.0), ("stretched_3x2x2", "per", 3, 0.0),
                                                ("uniform_3", "perall", 8, 1.0), ("stretched_3x2x2", "perd", 11, 0.5)])
def test_smoother(mesh_name, bc, p, lam):
    h = MESHES[mesh_name]
    m = dense.Mesh(h, p, lam, BCS[bc])
    r = skel_random(m, 21)
    ref = matfree.smooth(m, r, chunk=16)
    mask = matfree.condensed_mask(m)
    with ctx(h, p, lam, BCS[bc], p0=1) as c:
        rh = c.pack(c.L, cuda(r))
        du = to_nodal(c, c.L, c.smooth(c.L, rh))
        du32 = to_nodal(c, c.L, c.smooth(c.L, rh.float()).double())
    assert rel(du[mask], ref[mask]) < TOL64
    assert rel(du32[mask], ref[mask]) < TOL32
    # zero on Dirichlet faces; a periodic image plane repeats its unknowns
    skel, _ = matfree.masks(m)
    assert rel(du[skel], dense.sync_images(m, np.where(mask, ref, 0.0))[skel]) < TOL64
    if p <= 4:
        cond = dense.Condensed(m)
        assert rel(du.ravel()[cond.B], dense.smoother_dense(m, cond, r.ravel()[cond.B])) < TOL64


def test_tensor_core_smoother():
    h = MESHES["uniform_3"]
    m = dense.Mesh(h, 16, 1.0, MIXED_BC)
    r = skel_random(m, 23)
    ref = matfree.smooth(m, r, chunk=16)
    mask = matfree.condensed_mask(m)
    with ctx(h, 16, 1.0, MIXED_BC, precision="mixed_tc") as c:
        du = to_nodal(c, c.L, c.smooth(c.L, c.pack(c.L, cuda(r)).float()).double())
    assert rel(du[mask], ref[mask]) < 5e-3


@pytest.mark.parametrize("mesh_name,bc,pc,pf", [("stretched_3x2x2", "mixed", 1, 2), ("uniform_3", "neumann", 2, 4),
                                                ("thin_2x1x2", "alt", 8, 13), ("stretched_3x2x2", "per", 1, 2),
                                                ("uniform_3", "perall", 4, 8), ("stretched_3x2x2", "per", 2, 3)])
def test_transfers(mesh_name, bc, pc, pf):
    h = MESHES[mesh_name]
    mc, mf = dense.Mesh(h, pc, 0.0, BCS[bc]), dense.Mesh(h, pf, 0.0, BCS[bc])
    uc = skel_random(mc, 31)
    rf = skel_random(mf, 32)
    uf0 = skel_random(mf, 33)
    ref_p = uf0 + matfree.prolong(mc, mf, uc)
    ref_r = matfree.restrict(mf, mc, rf)
    with ctx(h, pf, 1.0, BCS[bc], p0=pc) as c:
        assert c.degrees[-2:] == [pc, pf]
        lf, lc = c.L, c.L - 1
        fine = c.pack(lf, cuda(uf0))
        c.prolong_add(lf, c.pack(lc, cuda(uc)), fine)
        got_p = to_nodal(c, lf, fine)
        got_r = to_nodal(c, lc, c.restrict(lf, c.pack(lf, cuda(rf))))
    mkf, mkc = matfree.condensed_mask(mf), matfree.condensed_mask(mc)
    assert rel(got_p[mkf], ref_p[mkf]) < TOL64
    assert rel(got_r[mkc], ref_r[mkc]) < TOL64


@pytest.mark.parametrize("mesh_name,bc,p0,lam", [("stretched_3x2x2", "mixed", 1, 0.0), ("uniform_3", "neumann", 2, 1.0),
                                                 ("thin_2x1x2", "alt", 2, 0.5), ("stretched_3x2x2", "per", 1, 0.0),
                                                 ("uniform_3", "perall", 2, 1.0)])
def test_coarse_solve_and_vcycle(mesh_name, bc, p0, lam):
    h = MESHES[mesh_name]
    m0 = dense.Mesh(h, p0, lam, BCS[bc])
    cond = dense.Condensed(m0)
    f0 = skel_random(m0, 41)
    ref0 = np.linalg.solve(cond.Hhat, f0.ravel()[cond.B])
    p = 4 * p0
    m = dense.Mesh(h, p, lam, BCS[bc])
    mg = matfree.MG(m, p0=p0)
    u = skel_random(m, 42)
    F = skel_random(m, 43)
    ref = matfree.vcycle(mg, u, F)
    with ctx(h, p0, lam, BCS[bc], p0=p0) as c:
        got0 = to_nodal(c, 0, c.coarse_solve(c.pack(0, cuda(f0))))
    with ctx(h, p, lam, BCS[bc], p0=p0) as c:
        uh = c.pack(c.L, cuda(u))
        c.vcycle(uh, c.pack(c.L, cuda(F)))
        got = to_nodal(c, c.L, uh)
    mask = matfree.condensed_mask(m)
    assert rel(got0.ravel()[cond.B], ref0) < 1e-11
    assert rel(got[mask], ref[mask]) < 1e-11


@pytest.mark.parametrize("bc,kind,solver,precision,p", [(NEUMANN, "ccc", "mg", "fp64", 8), (NEUMANN, "ccc", "kmg", "mixed", 8),
                                                        (("D", "D", "N", "N", "N", "N"), "scc", "mg", "mixed", 8),
                                                        (("N", "D", "N", "D", "D", "N"), "mixed", "kmg", "fp64", 8),
                                                        (NEUMANN, "ccc", "kmg", "fp64", 12),
                                                        (("N", "D", "N", "D", "D", "N"), "mixed", "mg", "mixed_fp32", 13),
                                                        (("N", "D", "N", "D", "D", "N"), "mixed", "kmg", "mixed_ff", 13),
                                                        (NEUMANN, "ccc", "mg", "mixed_ff_tc", 16)])
def test_solve_manufactured(bc, kind, solver, precision, p):
    # solutions with zero normal derivative on the Neumann faces (see the oracle pins);
    # p >= 12 runs the face-parallel operator
    h = workloads.uniform_widths(3)
    m = dense.Mesh(h, p, 1.0, bc)
    x = workloads.node_coords(h, p)
    X3, X2, X1 = np.meshgrid(x[2], x[1], x[0], indexing="ij")
    pi = np.pi
    if kind == "ccc":
        ue, k2 = np.cos(pi * X1) * np.cos(pi * X2) * np.cos(pi * X3), 3 * pi**2
    elif kind == "scc":
        ue, k2 = np.sin(pi * X1) * np.cos(pi * X2) * np.cos(pi * X3), 3 * pi**2
    else:
        ue, k2 = np.cos(pi * X1 / 2) * np.cos(pi * X2 / 2) * np.sin(pi * X3 / 2), 3 * (pi / 2) ** 2
    f = (1.0 + k2) * ue
    mg = matfree.MG(m, p0=2)
    Fh = matfree.condense_rhs(m, f)
    _, it_ref, _ = (matfree.mg_solve if solver == "mg" else matfree.kmg_solve)(mg, Fh)
    with ctx(h, p, 1.0, bc, p0=2, solver=solver, precision=precision) as c:
        u, info = c.solve(cuda(f))
        u = u.cpu().numpy()
    assert info.status == 0 and info.res_final <= 1e-10 * info.res0
    if precision == "fp64":
        assert info.iters == it_ref
    else:
        assert abs(info.iters - it_ref) <= 1
    assert np.abs(u - ue).max() < 1e-8


def test_pure_neumann_needs_positive_lambda():
    from paper_1808_03595_gb300.solver import SemmgError
    with pytest.raises(SemmgError):
        ctx(workloads.uniform_widths(2), 4, 0.0, NEUMANN)


@pytest.mark.parametrize("bc,kind,solver,precision", [(("P",) * 6, "ccc2", "mg", "fp64"),
                                                      (("P", "P", "D", "D", "D", "D"), "css", "kmg", "mixed"),
                                                      (("P", "P", "N", "N", "D", "D"), "scs", "mg", "mixed_tc"),
                                                      (("P", "P", "N", "N", "D", "D"), "scs", "kmg", "mixed_ff_tc")])
def test_solve_manufactured_periodic(bc, kind, solver, precision):
    # period-1 trigonometric solutions (see the oracle pins); the nodal result repeats plane 0
    p = 16 if precision in ("mixed_tc", "mixed_ff_tc") else 8
    h = workloads.uniform_widths(3)
    m = dense.Mesh(h, p, 1.0, bc)
    x = workloads.node_coords(h, p)
    X3, X2, X1 = np.meshgrid(x[2], x[1], x[0], indexing="ij")
    pi = np.pi
    if kind == "ccc2":
        ue, k2 = np.cos(2 * pi * X1) * np.cos(2 * pi * X2) * np.cos(2 * pi * X3), 12 * pi**2
    elif kind == "css":
        ue, k2 = np.cos(2 * pi * X1) * np.sin(pi * X2) * np.sin(pi * X3), 6 * pi**2
    else:
        ue, k2 = np.sin(2 * pi * X1) * np.cos(pi * X2) * np.sin(pi * X3), 6 * pi**2
    f = (1.0 + k2) * ue
    mg = matfree.MG(m, p0=2)
    Fh = matfree.condense_rhs(m, f)
    _, it_ref, _ = (matfree.mg_solve if solver == "mg" else matfree.kmg_solve)(mg, Fh)
    with ctx(h, p, 1.0, bc, p0=2, solver=solver, precision=precision) as c:
        u, info = c.solve(cuda(f))
        u = u.cpu().numpy()
    assert info.status == 0 and info.res_final <= 1e-10 * info.res0
    if precision == "fp64":
        assert info.iters == it_ref
    else:
        assert abs(info.iters - it_ref) <= 1
    assert np.abs(u - ue).max() < 1e-8
    assert np.array_equal(u[:, :, 0], u[:, :, -1])


def test_periodic_setup_checks():
    from paper_1808_03595_gb300.solver import SemmgError
    with pytest.raises(SemmgError):  # one periodic face without its partner
        ctx(workloads.uniform_widths(3), 4, 1.0, ("P", "D", "D", "D", "D", "D"))
    with pytest.raises(SemmgError):  # a single element along a periodic axis
        ctx([np.array([1.0]), np.full(2, 0.5), np.full(2, 0.5)], 4, 1.0, ("P", "P", "D", "D", "D", "D"))
