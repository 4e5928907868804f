"""Inhomogeneous Dirichlet data (the test problem of Sec. 5.2) on the CUDA path, against the FP64 oracle.

The library lifts the data: the condensed vector's boundary slots hold g, so the
residual, the operator and the recovery read it as prescribed values, while the
V-cycle corrections vanish there.  The oracle lifts the textbook way (F = M f -
H E g, a homogeneous solve, u = u_0 + E g); the two meet in r_0, the iterates and u.
"""
import numpy as np
import pytest

import workloads
from oracle import dense, matfree

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL64 = 1e-12

BCS = {"dir": ("D",) * 6, "mixed": ("N", "D", "D", "N", "D", "N"), "nd": ("N", "N", "D", "D", "D", "D"),
       "perd": ("P", "P", "P", "P", "D", "D"), "perx": ("P", "P", "D", "N", "D", "D")}
MESHES = {
    "stretched_3x2x2": [np.array([0.2, 0.5, 0.3]), np.array([0.7, 0.3]), np.array([0.4, 0.6])],
    "uniform_3": workloads.uniform_widths(3),
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


def periodic_data(m, a):
    """Nodal data that repeats across periodic axes (image planes equal to the first)."""
    return dense.sync_images(m, a)


@pytest.mark.parametrize("mesh_name,bc,p,lam", [("stretched_3x2x2", "dir", 3, 0.0), ("uniform_3", "mixed", 8, 1.0),
                                                ("stretched_3x2x2", "nd", 5, 2.0), ("uniform_3", "perd", 16, 0.5),
                                                ("stretched_3x2x2", "perx", 4, 0.0), ("uniform_3", "dir", 32, 1.0)])
def test_pack_dirichlet_and_lifted_residual(mesh_name, bc, p, lam):
    h = MESHES[mesh_name]
    m = dense.Mesh(h, p, lam, BCS[bc])
    rng = np.random.default_rng(41)
    f = rng.uniform(-1, 1, m.shape)
    g = periodic_data(m, rng.uniform(-1, 1, m.shape))
    dm = m.dirichlet_mask()
    skel, _ = matfree.masks(m)
    mask = matfree.condensed_mask(m)
    ref = matfree.condense_load(m, matfree.lifted_load(m, f, g))
    with ctx(h, p, lam, BCS[bc]) as c:
        gh = c.pack_dirichlet(c.L, cuda(g))
        eg = c.unpack(c.L, gh).cpu().numpy()
        fh = c.condense_rhs(cuda(f))
        r = c.residual(c.L, fh, gh)
        torch.cuda.synchronize()
        rn = c.unpack(c.L, r).cpu().numpy()
    assert np.array_equal(eg[dm], g[dm])
    assert np.all(eg[skel & ~dm] == 0.0)
    # r_0 = Fhat - Hhat E g equals the oracle's condensed lifted load at the unknowns, 0 on the boundary
    assert rel(rn[mask], ref[mask]) < TOL64
    assert np.all(rn[dm] == 0.0)


@pytest.mark.parametrize("mesh_name,bc,p,lam,solver,precision",
                         [("stretched_3x2x2", "dir", 4, 0.0, "mg", "fp64"), ("uniform_3", "mixed", 8, 1.0, "kmg", "fp64"),
                          ("stretched_3x2x2", "nd", 6, 2.0, "mg", "mixed"), ("uniform_3", "perd", 8, 0.5, "kmg", "mixed"),
                          ("stretched_3x2x2", "perx", 5, 0.0, "mg", "fp64"), ("uniform_3", "dir", 16, 0.0, "mg", "mixed_fp32"),
                          ("uniform_3", "dir", 16, 1.0, "kmg", "fp64")])
def test_solve_dirichlet_matches_oracle(mesh_name, bc, p, lam, solver, precision):
    h = MESHES[mesh_name]
    m = dense.Mesh(h, p, lam, BCS[bc])
    rng = np.random.default_rng(42)
    f = rng.uniform(-1, 1, m.shape)
    g = periodic_data(m, rng.uniform(-1, 1, m.shape))
    mg = matfree.MG(m, p0=2)
    ref, it_ref, hist = matfree.solve_dirichlet(m, f, g, krylov=(solver == "kmg"), mg=mg)
    with ctx(h, p, lam, BCS[bc], p0=2, solver=solver, precision=precision) as c:
        u, info = c.solve(cuda(f), g=cuda(g))
        u = u.cpu().numpy()
    assert info.status == 0 and info.res_final <= 1e-10 * info.res0
    assert abs(info.res0 - hist[0]) <= 1e-12 * hist[0]  # r_0 = Fhat - Hhat E g
    assert abs(info.iters - it_ref) <= (0 if precision == "fp64" else 1)
    assert rel(u, ref) < 1e-8
    dm = m.dirichlet_mask()
    assert np.array_equal(u[dm], g[dm])


@pytest.mark.parametrize("kind,bc,lam,p", [("D", "dir", 0.7, 3), ("ND", "nd", 0.0, 4), ("PD", "perd", 0.3, 3),
                                           ("D", "dir", 0.0, 8)])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_solve_dirichlet_reproduces_polynomials(kind, bc, lam, p, precision):
    # degree <= 3 per variable lies in the discrete space and is integrated exactly (see the oracle pins):
    # the discrete solution equals it at every node
    h = MESHES["stretched_3x2x2"]
    m = dense.Mesh(h, p, lam, BCS[bc])
    x = m.node_coords()
    X3, X2, X1 = np.meshgrid(x[2], x[1], x[0], indexing="ij")
    if kind == "D":
        ue, lap = 1 + X1 - 2 * X2**2 + X3**3 + X1 * X2 * X3 + X1**2 * X2, 2 * X2 - 4 + 6 * X3
    elif kind == "ND":
        L1 = m.X[0][-1]
        q, q2 = X1**2 * (3 * L1 - 2 * X1), 6 * L1 - 12 * X1
        r = 1 + X2 - X3**2 + X2 * X3
        ue, lap = q * r, q2 * r - 2 * q
    else:
        ue, lap = X3**3 - 2 * X3 + 1, 6 * X3
    f = lam * ue - lap
    with ctx(h, p, lam, BCS[bc], p0=1, precision=precision, max_iter=60) as c:
        u, info = c.solve(cuda(f), rtol=1e-12 if precision == "fp64" else 1e-11, g=cuda(ue))
        u = u.cpu().numpy()
    assert info.status == 0
    assert rel(u, ue) < (1e-9 if precision == "fp64" else 1e-8)


def test_zero_data_equals_homogeneous_solve_and_aliasing():
    h, p, lam = MESHES["stretched_3x2x2"], 8, 1.0
    rng = np.random.default_rng(43)
    m = dense.Mesh(h, p, lam)
    f = rng.uniform(-1, 1, m.shape)
    g = rng.uniform(-1, 1, m.shape)
    with ctx(h, p, lam, BCS["dir"]) as c:
        u0, i0 = c.solve(cuda(f))
        u1, i1 = c.solve(cuda(f), g=torch.zeros_like(u0))
        assert torch.equal(u0, u1) and i0.iters == i1.iters and i0.res0 == i1.res0
        # g may alias the output: the data is read before the solution is written
        ug, _ = c.solve(cuda(f), g=cuda(g))
        ua = cuda(g)
        ua, _ = c.solve(cuda(f), g=ua, out=ua)
        assert torch.equal(ug, ua)


@pytest.mark.parametrize("p,bound", [(6, 3e-3), (10, 2e-6)])
def test_paper_solution(p, bound):
    # Sec. 5.2's manufactured solution on (0, 2 pi)^3, lambda = 0, inhomogeneous Dirichlet data at all faces
    # (k = 1/2 so that 3^3 elements resolve it; the oracle pins the same bounds)
    h = [np.full(3, 2 * np.pi / 3)] * 3
    ue, f = workloads.paper_solution(h, p, k=0.5, lam=0.0)
    m = dense.Mesh(h, p, 0.0)
    ref, it_ref, _ = matfree.solve_dirichlet(m, f, ue, mg=matfree.MG(m, p0=2))
    with ctx(h, p, 0.0, BCS["dir"], p0=2) as c:
        u, info = c.solve(cuda(f), g=cuda(ue))
        u = u.cpu().numpy()
    assert info.iters == it_ref
    assert rel(u, ref) < 1e-8
    assert np.abs(u - ue).max() < bound
