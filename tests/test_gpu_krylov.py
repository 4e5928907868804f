"""Algorithm 5 (Krylov-accelerated multigrid) and the varied smoothing counts on the GPU.

The GPU iteration is compared with the oracle's ipCG (oracle.matfree.kmg_solve)
on the paper's stretched grids (8^3 elements on (0, 2 pi)^3, widths growing by a
constant factor alpha): same iteration count in FP64, the solution within the
1e-10 residual bound, and the oracle's own condensed residual of the GPU
solution below 1e-10 of the initial one.
"""
import numpy as np
import pytest

import workloads
from oracle import dense, matfree

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1808_03595_gb300 import build
    build.build()


def _stretched(alpha, p, seed=1808):
    h = workloads.expansion_widths(8, alpha)
    mesh = dense.Mesh(h, p, 0.0)
    f = np.random.default_rng(seed).uniform(-1, 1, mesh.shape)
    return h, mesh, f


def _oracle_reduction(mesh, f, u_nodal):
    mask = matfree.condensed_mask(mesh)
    Fh = matfree.condense_rhs(mesh, f)
    r = Fh - matfree.apply_condensed(mesh, np.where(mask, u_nodal, 0.0))
    return np.linalg.norm(r[mask]) / np.linalg.norm(Fh[mask])


@pytest.mark.parametrize("alpha,p,nu_vary", [(1.5, 4, False), (1.5, 4, True), (2.0, 4, False), (1.5, 8, False),
                                             (1.0, 8, True)])
def test_kmg_fp64_matches_oracle(alpha, p, nu_vary):
    from paper_1808_03595_gb300 import Context
    h, mesh, f = _stretched(alpha, p)
    mg = matfree.MG(mesh, p0=2, nu_vary=nu_vary)
    uh_ref, it_ref, _ = matfree.kmg_solve(mg, matfree.condense_rhs(mesh, f), maxit=60)
    u_ref = matfree.recover(mesh, f, uh_ref)
    with Context(h, p, 0.0, p0=2, solver="kmg", nu_vary=nu_vary, max_iter=60) as c:
        u, info = c.solve(torch.as_tensor(f, device="cuda"))
        u = u.cpu().numpy()
    assert info.status == 0 and info.res_final <= 1e-10 * info.res0
    assert info.iters == it_ref
    assert _oracle_reduction(mesh, f, u) < 2e-10
    assert np.abs(u - u_ref).max() <= 1e-8 * np.abs(u_ref).max()


@pytest.mark.parametrize("alpha,p", [(1.5, 4), (2.0, 8)])
def test_kmg_mixed_precision(alpha, p):
    # FP32 V-cycle as the preconditioner of the FP64 ipCG iteration
    from paper_1808_03595_gb300 import Context
    h, mesh, f = _stretched(alpha, p)
    fd = torch.as_tensor(f, device="cuda")
    with Context(h, p, 0.0, p0=2, solver="kmg", max_iter=60) as c:
        _, info64 = c.solve(fd)
    with Context(h, p, 0.0, p0=2, solver="kmg", precision="mixed", max_iter=60) as c:
        u, info = c.solve(fd)
        u = u.cpu().numpy()
    assert info.status == 0 and info.res_final <= 1e-10 * info.res0
    assert abs(info.iters - info64.iters) <= 1
    assert _oracle_reduction(mesh, f, u) < 2e-10


def test_kmg_fewer_iterations_than_mg_on_stretched_grid():
    # Sec. 5.4: Krylov acceleration cuts the iterations on stretched grids (MG 21 -> kMG 11 at alpha 1.5, p 4)
    from paper_1808_03595_gb300 import Context
    h, mesh, f = _stretched(1.5, 4)
    fd = torch.as_tensor(f, device="cuda")
    with Context(h, 4, 0.0, p0=2, max_iter=60) as c:
        _, info_mg = c.solve(fd)
    with Context(h, 4, 0.0, p0=2, solver="kmg", max_iter=60) as c:
        _, info_k = c.solve(fd)
    assert info_mg.status == 0 and info_k.status == 0
    assert abs(info_mg.iters - 21) <= 1 and abs(info_k.iters - 11) <= 1


def test_kmg_batch_equals_individual_solves():
    from paper_1808_03595_gb300 import Batch, Context
    cases = [(workloads.expansion_widths(3, 1.5), 5, 0.0, "fp64", False),
             (workloads.uniform_widths(2), 9, 2.0, "mixed", True),
             (workloads.stretched_widths(3, 7), 6, 50.0, "fp64", True)]
    ctxs, fs, us, refs = [], [], [], []
    for i, (h, p, lam, prec, vary) in enumerate(cases):
        c = Context(h, p, lam, p0=2, precision=prec, solver="kmg", nu_vary=vary)
        fd = torch.as_tensor(workloads.random_nodal(h, p, 40 + i, "uniform"), device="cuda")
        u_ref, info = c.solve(fd)
        refs.append((u_ref.cpu().numpy(), info.iters))
        ctxs.append(c)
        fs.append(fd)
        us.append(torch.full_like(fd, float("nan")))
    b = Batch(ctxs, fs, us)
    rc, infos = b.solve()
    assert rc == 0
    for (u_ref, it_ref), u, info in zip(refs, us, infos):
        assert info.status == 0 and info.iters == it_ref
        assert info.res_final <= 1e-10 * info.res0
        assert np.abs(u.cpu().numpy() - u_ref).max() <= 1e-12 * np.abs(u_ref).max()
    b.close()
    for c in ctxs:
        c.close()
