"""Parity of the CUDA path (through the C ABI) with the FP64 oracle, element by element.

Tolerances: FP64 operator / smoother / transfer applications 1e-12 relative
(max-norm error over max-norm reference); FP32 smoother and transfers 2e-5
relative (a few hundred FP32 roundings on O(1) data); solves reach a 1e-10
relative residual reduction and match the oracle's solution to
cond-limited accuracy.  Comparisons are made on nodal arrays at the
skeleton nodes, using the library's own pack/unpack (checked bit-exact here).
"""
import numpy as np
import pytest

import workloads
from oracle import dense, matfree

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 2e-5


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1808_03595_gb300 import build
    build.build()


def ctx_for(h, p, lam, **kw):
    from paper_1808_03595_gb300 import Context
    return Context(h, p, lam, **kw)


def cuda(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def rel(a, b):
    b = np.asarray(b)
    return float(np.abs(np.asarray(a) - b).max() / max(np.abs(b).max(), 1e-300))


MESHES = {
    # ragged: three axes with different element counts and widths
    "stretched_3x2x2": [np.array([0.2, 0.5, 0.3]), np.array([0.7, 0.3]), np.array([0.4, 0.6])],
    "uniform_3": workloads.uniform_widths(3),
    "thin_2x1x2": [np.array([0.6, 0.4]), np.array([0.5]), np.array([1.0, 1.0])],
    "uniform_5x4x3": [np.full(5, 0.2), np.full(4, 0.25), np.full(3, 1 / 3)],
}


def omesh(h, p, lam):
    return dense.Mesh(h, p, lam)


def skel_random(h, p, seed, level_mesh=None):
    m = omesh(h, p, 0.0)
    u = workloads.random_nodal(h, p, seed)
    return np.where(matfree.condensed_mask(m), u, 0.0)


def to_hat(ctx, level, nodal):
    return ctx.pack(level, cuda(nodal))


def to_nodal(ctx, level, hat):
    torch.cuda.synchronize()
    return ctx.unpack(level, hat).cpu().numpy()


# ------------------------------------------------------------------ layout

@pytest.mark.parametrize("p", [1, 2, 5, 8])
def test_pack_unpack_roundtrip(p):
    h = MESHES["stretched_3x2x2"]
    with ctx_for(h, p, 1.0, p0=1) as c:
        m = omesh(h, p, 0.0)
        u = workloads.random_nodal(h, p, 3)
        hat = to_hat(c, c.L, u)
        assert hat.numel() == c.condensed_size()
        back = to_nodal(c, c.L, hat)
        mask = matfree.condensed_mask(m)
        skel, free = matfree.masks(m)
        assert np.array_equal(back[mask], u[mask])          # bit-exact on free skeleton nodes
        assert np.all(back[skel & ~free] == 0.0)             # Dirichlet slots hold zero
        assert np.all(back[~skel] == 0.0)                    # interiors untouched
        # every free skeleton node has exactly one slot
        n_free_skel = int(mask.sum())
        assert int((hat != 0).sum().item()) == n_free_skel


# ------------------------------------------------------------------ condensed operator (Sec. 2.2)

@pytest.mark.parametrize("mesh_name,p,lam", [("stretched_3x2x2", 2, 0.0), ("stretched_3x2x2", 4, 1.5),
                                             ("uniform_3", 5, 100.0), ("thin_2x1x2", 6, 0.3),
                                             ("stretched_3x2x2", 7, 2.0)])
def test_apply_condensed_vs_dense_schur(mesh_name, p, lam):
    h = MESHES[mesh_name]
    m = omesh(h, p, lam)
    cond = dense.Condensed(m)
    u = skel_random(h, p, 11)
    ref = cond.Hhat @ u.ravel()[cond.B]
    with ctx_for(h, p, lam) as c:
        y = to_nodal(c, c.L, c.apply_condensed(c.L, to_hat(c, c.L, u)))
    assert rel(y.ravel()[cond.B], ref) < TOL64


@pytest.mark.parametrize("mesh_name,p,lam", [("uniform_5x4x3", 8, 1.0), ("stretched_3x2x2", 12, 0.0),
                                             ("uniform_3", 16, 100.0), ("thin_2x1x2", 24, 1.0),
                                             ("thin_2x1x2", 32, 0.5), ("thin_2x1x2", 47, 0.0),
                                             ("thin_2x1x2", 48, 2.0)])
def test_apply_condensed_vs_matrix_free_oracle(mesh_name, p, lam):
    h = MESHES[mesh_name]
    m = omesh(h, p, lam)
    u = skel_random(h, p, 12)
    ref = matfree.apply_condensed(m, u)
    with ctx_for(h, p, lam) as c:
        y = to_nodal(c, c.L, c.apply_condensed(c.L, to_hat(c, c.L, u)))
        f = skel_random(h, p, 13)
        r = to_nodal(c, c.L, c.residual(c.L, to_hat(c, c.L, f), to_hat(c, c.L, u)))
    mask = matfree.condensed_mask(m)
    assert rel(y[mask], ref[mask]) < TOL64
    assert rel(r[mask], (f - ref)[mask]) < TOL64


# ------------------------------------------------------------------ smoother (Algorithms 1, 2)

@pytest.mark.parametrize("mesh_name,p,lam", [("stretched_3x2x2", 2, 0.0), ("stretched_3x2x2", 4, 1.5),
                                             ("uniform_3", 3, 100.0), ("thin_2x1x2", 5, 0.3)])
def test_smooth_vs_dense_star_inverses(mesh_name, p, lam):
    h = MESHES[mesh_name]
    m = omesh(h, p, lam)
    cond = dense.Condensed(m)
    r = skel_random(h, p, 21)
    ref = dense.smoother_dense(m, cond, r.ravel()[cond.B])
    with ctx_for(h, p, lam, p0=1) as c:
        du = to_nodal(c, c.L, c.smooth(c.L, to_hat(c, c.L, r)))
    assert rel(du.ravel()[cond.B], ref) < TOL64


@pytest.mark.parametrize("mesh_name,p,lam", [("uniform_5x4x3", 8, 1.0), ("stretched_3x2x2", 11, 0.0),
                                             ("uniform_3", 16, 100.0), ("thin_2x1x2", 24, 1.0),
                                             ("thin_2x1x2", 47, 0.5), ("thin_2x1x2", 48, 0.0)])
def test_smooth_vs_matrix_free_oracle(mesh_name, p, lam):
    h = MESHES[mesh_name]
    m = omesh(h, p, lam)
    r = skel_random(h, p, 22)
    ref = matfree.smooth(m, r)
    mask = matfree.condensed_mask(m)
    with ctx_for(h, p, lam, p0=1) as c:
        rh = to_hat(c, c.L, r)
        du = to_nodal(c, c.L, c.smooth(c.L, rh))
        du32 = c.smooth(c.L, rh.float())
        du32n = to_nodal(c, c.L, du32.double())
    assert rel(du[mask], ref[mask]) < TOL64
    assert rel(du32n[mask], ref[mask]) < TOL32


# ------------------------------------------------------------------ transfers and coarse solve (Sec. 4.1)

@pytest.mark.parametrize("mesh_name,pc,pf", [("stretched_3x2x2", 1, 2), ("stretched_3x2x2", 2, 4),
                                             ("uniform_3", 4, 8), ("uniform_5x4x3", 8, 13),
                                             ("thin_2x1x2", 16, 24)])
def test_transfers_vs_oracle(mesh_name, pc, pf):
    h = MESHES[mesh_name]
    mc, mf = omesh(h, pc, 0.0), omesh(h, pf, 0.0)
    uc = skel_random(h, pc, 31)
    rf = skel_random(h, pf, 32)
    uf0 = skel_random(h, pf, 33)
    ref_p = uf0 + matfree.prolong(mc, mf, uc)
    ref_r = matfree.restrict(mf, mc, rf)
    # a context whose two finest levels are (pc, pf)
    with ctx_for(h, pf, 0.0, p0=pc) as c:
        assert c.degrees[-2:] == [pc, pf]
        lf, lc = c.L, c.L - 1
        fine = to_hat(c, lf, uf0)
        c.prolong_add(lf, to_hat(c, lc, uc), fine)
        got_p = to_nodal(c, lf, fine)
        got_r = to_nodal(c, lc, c.restrict(lf, to_hat(c, lf, rf)))
        fine32 = to_hat(c, lf, uf0).float()
        c.prolong_add(lf, to_hat(c, lc, uc).float(), fine32)
        got_p32 = to_nodal(c, lf, fine32.double())
        got_r32 = to_nodal(c, lc, c.restrict(lf, to_hat(c, lf, rf).float()).double())
    mkf, mkc = matfree.condensed_mask(mf), matfree.condensed_mask(mc)
    assert rel(got_p[mkf], ref_p[mkf]) < TOL64
    assert rel(got_r[mkc], ref_r[mkc]) < TOL64
    assert rel(got_p32[mkf], ref_p[mkf]) < TOL32
    assert rel(got_r32[mkc], ref_r[mkc]) < TOL32


@pytest.mark.parametrize("mesh_name,p0,lam", [("stretched_3x2x2", 1, 0.0), ("uniform_5x4x3", 1, 3.0),
                                              ("stretched_3x2x2", 2, 1.0), ("thin_2x1x2", 2, 0.0)])
def test_coarse_solve_exact(mesh_name, p0, lam):
    h = MESHES[mesh_name]
    m = omesh(h, p0, lam)
    cond = dense.Condensed(m)
    f = skel_random(h, p0, 41)
    ref = np.linalg.solve(cond.Hhat, f.ravel()[cond.B]) if len(cond.B) else np.zeros(0)
    with ctx_for(h, p0, lam, p0=p0) as c:
        got = to_nodal(c, 0, c.coarse_solve(to_hat(c, 0, f)))
    if len(cond.B):
        assert rel(got.ravel()[cond.B], ref) < 1e-11


# ------------------------------------------------------------------ condensation, recovery (Algorithm 4)

@pytest.mark.parametrize("mesh_name,p,lam", [("stretched_3x2x2", 4, 1.0), ("uniform_5x4x3", 9, 0.0),
                                             ("thin_2x1x2", 20, 2.0), ("thin_2x1x2", 48, 0.5)])
def test_condense_and_recover_vs_oracle(mesh_name, p, lam):
    h = MESHES[mesh_name]
    m = omesh(h, p, lam)
    f = workloads.random_nodal(h, p, 51)
    uh = skel_random(h, p, 52)
    ref_F = matfree.condense_rhs(m, f)
    ref_u = matfree.recover(m, f, uh)
    with ctx_for(h, p, lam) as c:
        F = to_nodal(c, c.L, c.condense_rhs(cuda(f)))
        u = c.recover(cuda(f), to_hat(c, c.L, uh)).cpu().numpy()
    mask = matfree.condensed_mask(m)
    assert rel(F[mask], ref_F[mask]) < TOL64
    assert rel(u, ref_u) < TOL64


# ------------------------------------------------------------------ V-cycle and solver (Algorithms 3, 4)

@pytest.mark.parametrize("mesh_name,p,p0", [("stretched_3x2x2", 4, 1), ("uniform_3", 6, 2), ("thin_2x1x2", 9, 2)])
def test_vcycle_vs_oracle(mesh_name, p, p0):
    h = MESHES[mesh_name]
    m = omesh(h, p, 1.0)
    mg = matfree.MG(m, p0=p0)
    u = skel_random(h, p, 61)
    F = skel_random(h, p, 62)
    ref = matfree.vcycle(mg, u, F)
    with ctx_for(h, p, 1.0, p0=p0) as c:
        uh = to_hat(c, c.L, u)
        c.vcycle(uh, to_hat(c, c.L, F))
        got = to_nodal(c, c.L, uh)
    mask = matfree.condensed_mask(m)
    assert rel(got[mask], ref[mask]) < 1e-11


@pytest.mark.parametrize("precision", ["fp64", "mixed", "mixed_fp32"])
def test_solve_config1_poisson_4x4x4_p4(precision):
    h, p, lam, f, p0 = workloads.config("poisson_4x4x4_p4")
    m = omesh(h, p, lam)
    ref, it_ref, _ = matfree.solve(m, f, p0=p0)
    with ctx_for(h, p, lam, p0=p0, precision=precision) as c:
        u, info = c.solve(cuda(f), rtol=1e-10)
        u = u.cpu().numpy()
    assert info.res_final <= 1e-10 * info.res0
    if precision == "fp64":
        assert info.iters == it_ref
    else:
        assert abs(info.iters - it_ref) <= 1
    assert rel(u, ref) < 1e-8
    # the discrete solution approximates sin(pi x) sin(pi y) sin(pi z) spectrally
    ue = workloads.sinsinsin(h, p)
    assert np.abs(u - ue).max() < 2e-3


@pytest.mark.parametrize("p", [4, 8])
def test_solve_helmholtz_8x8x8(p):
    h, p, lam, f, p0 = workloads.config(f"helmholtz_8x8x8_p{p}")
    m = omesh(h, p, lam)
    ref, it_ref, hist = matfree.solve(m, f, p0=p0)
    for precision in ("fp64", "mixed", "mixed_fp32"):
        with ctx_for(h, p, lam, p0=p0, precision=precision) as c:
            u, info = c.solve(cuda(f), rtol=1e-10)
            u = u.cpu().numpy()
        assert info.res_final <= 1e-10 * info.res0
        assert abs(info.iters - it_ref) <= (0 if precision == "fp64" else 1)
        assert rel(u, ref) < 1e-8


@pytest.mark.parametrize("p,precision", [(4, "fp64"), (16, "fp64"), (16, "mixed_ff_tc")])
def test_solve_host_matches_device(p, precision):
    # page-locked u is written through its device mapping, pageable u gets a copy: both as on the device
    h, p, lam, f, p0 = workloads.config(f"helmholtz_8x8x8_p{p}")
    with ctx_for(h, p, lam, p0=p0, precision=precision) as c:
        ud, info_d = c.solve(cuda(f))
        fh = torch.as_tensor(f).pin_memory()
        uh = torch.empty_like(fh).pin_memory()
        c.solve_host(fh, uh)
        fp = torch.as_tensor(f).clone()
        up = torch.full_like(fp, float("nan"))
        c.solve_host(fp, up)
    assert np.array_equal(ud.cpu().numpy(), uh.numpy())
    assert np.array_equal(ud.cpu().numpy(), up.numpy())


def test_not_converged_and_nonfinite_status():
    from paper_1808_03595_gb300.solver import SemmgError
    h, p, lam, f, p0 = workloads.config("helmholtz_8x8x8_p4")
    with ctx_for(h, p, lam, p0=p0, max_iter=1) as c:
        u, info = c.solve(cuda(f), allow_not_converged=True)
        assert info.status == -4 and info.iters == 1
        with pytest.raises(SemmgError):
            c.solve(cuda(f))
        fbad = f.copy()
        fbad[3, 3, 3] = np.nan
        with pytest.raises(SemmgError) as e:
            c.solve(cuda(fbad))
        assert e.value.code == -5


def test_single_element_mesh_has_empty_condensed_system():
    # n = (1, 1, 1): every skeleton node is on the Dirichlet boundary; the solve
    # is condensation plus interior recovery only
    h = [np.array([1.0]), np.array([0.5]), np.array([2.0])]
    p, lam = 6, 1.0
    m = omesh(h, p, lam)
    cond = dense.Condensed(m, dense=False)
    f = workloads.random_nodal(h, p, 71)
    uex = cond.full_solve(cond.load(f))
    with ctx_for(h, p, lam) as c:
        u, info = c.solve(cuda(f))
        u = u.cpu().numpy()
    assert info.iters == 0 and info.res0 == 0.0
    assert rel(u, uex) < 1e-12
