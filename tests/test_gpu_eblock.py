"""Element-centred block smoother (Sec. 3.4) on the CUDA path, against the FP64 oracle.

The kernel inverts each 3x3x3-element block on its six condensed planes (73 n_E^3
operations, n_E = 3p - 1); the oracle applies the definition (the full block's fast
diagonalisation read on the block's skeleton, pinned against dense restricted
inverses).  Same tolerances as the star smoother: 1e-12 in FP64, 2e-5 in FP32.
"""
import numpy as np
import pytest

import workloads
from oracle import dense, matfree

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 2e-5

BCS = {"dir": ("D",) * 6, "mixed": ("N", "D", "D", "N", "N", "N"), "neumann": ("N",) * 6,
       "per": ("P", "P", "N", "D", "P", "P"), "perall": ("P",) * 6}
MESHES = {
    "stretched_3": [np.full(3, 1 / 3), np.array([0.2, 0.5, 0.3]), np.array([0.7, 0.3, 0.4])],
    "uniform_3": workloads.uniform_widths(3),
    "thin_2x1x4": [np.array([0.6, 0.4]), np.array([0.5]), np.array([0.3, 0.2, 0.25, 0.25])],
    "uniform_2": workloads.uniform_widths(2),
}


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1808_03595_gb300 import build
    build.build()


def ctx(h, p, lam, bc, smoother="element", **kw):
    from paper_1808_03595_gb300 import Context
    return Context(h, p, lam, bc=bc, smoother=smoother, **kw)


KIND = {"element": "element", "element_mult": "multiplicity"}


def cuda(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def rel(a, b):
    b = np.asarray(b)
    return float(np.abs(np.asarray(a) - b).max() / max(np.abs(b).max(), 1e-300))


def skel_random(m, seed):
    return np.where(matfree.condensed_mask(m), workloads.random_nodal(m.h, m.p, seed), 0.0)


def to_nodal(c, level, hat):
    torch.cuda.synchronize()
    return c.unpack(level, hat).cpu().numpy()


@pytest.mark.parametrize("smoother", ["element", "element_mult"])
@pytest.mark.parametrize("mesh_name,bc,p,lam", [("stretched_3", "dir", 2, 0.0), ("stretched_3", "dir", 3, 0.8),
                                                ("uniform_3", "mixed", 4, 1.0), ("thin_2x1x4", "neumann", 5, 2.0),
                                                ("stretched_3", "per", 3, 0.0), ("uniform_3", "perall", 8, 1.0),
                                                ("uniform_3", "dir", 16, 0.5), ("uniform_2", "dir", 32, 1.0)])
def test_smoother(mesh_name, bc, p, lam, smoother):
    h = MESHES[mesh_name]
    m = dense.Mesh(h, p, lam, BCS[bc])
    r = skel_random(m, 51)
    ref = matfree.smooth_eblock(m, r, matfree.EBlockTables(m, KIND[smoother]))
    mask = matfree.condensed_mask(m)
    with ctx(h, p, lam, BCS[bc], smoother, p0=1) as c:
        rh = c.pack(c.L, cuda(r))
        du = to_nodal(c, c.L, c.smooth(c.L, rh))
        du32 = to_nodal(c, c.L, c.smooth(c.L, rh.float()).double())
    assert rel(du[mask], ref[mask]) < TOL64
    assert rel(du32[mask], ref[mask]) < TOL32
    skel, _ = matfree.masks(m)
    assert rel(du[skel], dense.sync_images(m, np.where(mask, ref, 0.0))[skel]) < TOL64
    if p <= 3:
        cond = dense.Condensed(m)
        assert rel(du.ravel()[cond.B], dense.smoother_eblock_dense(m, cond, r.ravel()[cond.B], KIND[smoother])) < TOL64


@pytest.mark.parametrize("mesh_name,bc,p0,lam", [("stretched_3", "mixed", 1, 0.0), ("uniform_3", "dir", 2, 1.0),
                                                 ("stretched_3", "per", 1, 0.5)])
def test_vcycle(mesh_name, bc, p0, lam):
    h = MESHES[mesh_name]
    p = 4 * p0
    m = dense.Mesh(h, p, lam, BCS[bc])
    mg = matfree.MG(m, p0=p0, smoother="element")
    u = skel_random(m, 52)
    F = skel_random(m, 53)
    ref = matfree.vcycle(mg, u, F)
    with ctx(h, p, lam, BCS[bc], p0=p0) as c:
        uh = c.pack(c.L, cuda(u))
        c.vcycle(uh, c.pack(c.L, cuda(F)))
        got = to_nodal(c, c.L, uh)
    mask = matfree.condensed_mask(m)
    assert rel(got[mask], ref[mask]) < 1e-11


@pytest.mark.parametrize("mesh_name,bc,p,solver,precision,smoother",
                         [("stretched_3", "dir", 6, "mg", "fp64", "element"),
                          ("uniform_3", "mixed", 8, "kmg", "fp64", "element_mult"),
                          ("stretched_3", "per", 5, "mg", "mixed", "element"),
                          ("uniform_3", "dir", 16, "kmg", "mixed", "element"),
                          ("uniform_3", "dir", 16, "mg", "fp64", "element_mult")])
def test_solve_matches_oracle(mesh_name, bc, p, solver, precision, smoother):
    h = MESHES[mesh_name]
    lam = 0.0 if bc == "dir" else 1.0
    m = dense.Mesh(h, p, lam, BCS[bc])
    f = workloads.random_nodal(h, p, 54, "uniform")
    mg = matfree.MG(m, p0=2, smoother=smoother)
    Fh = matfree.condense_rhs(m, f)
    uh, it_ref, _ = (matfree.mg_solve if solver == "mg" else matfree.kmg_solve)(mg, Fh)
    ref = matfree.recover(m, f, uh)
    with ctx(h, p, lam, BCS[bc], smoother, p0=2, solver=solver, precision=precision) as c:
        u, info = c.solve(cuda(f))
        u = u.cpu().numpy()
    assert info.status == 0 and info.res_final <= 1e-10 * info.res0
    assert abs(info.iters - it_ref) <= (0 if precision == "fp64" else 1)
    assert rel(u, ref) < 1e-8


def test_element_smoother_setup_checks():
    from paper_1808_03595_gb300.solver import SemmgError
    with pytest.raises(SemmgError):
        ctx([np.full(2, 0.5), np.full(3, 1 / 3), np.full(3, 1 / 3)], 4, 1.0, ("P", "P", "D", "D", "D", "D"))
    with pytest.raises(KeyError):
        from paper_1808_03595_gb300 import Context
        Context(MESHES["uniform_3"], 4, 1.0, smoother="vertex")
