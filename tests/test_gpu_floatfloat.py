"""Float-float level residuals of the V-cycle (SEMMG_MIXED_FF, SEMMG_MIXED_FF_TC).

On the levels with p >= 12 (the face-parallel form of the condensed operator)
these forms evaluate the V-cycle's residual F - Hhat u in float-float
arithmetic (every value the unevaluated sum of two FP32 numbers) instead of
FP64; F, u and the result are FP32 vectors as in every mixed form.

The level residual is checked in the case that decides whether a residual is
good enough for the V-cycle: u smooth and F = Hhat u + a perturbation of 1e-4,
so that the residual is four orders below F and Hhat u, and Hhat u itself is a
small difference of the face block H_BB u and the Schur term.  The reference is
the oracle's FP64 residual of the same FP32 values.  The float-float residual
must be the exact one rounded once to FP32, as the FP64-arithmetic form
SEMMG_MIXED gives it (on the deepest cancellation, p = 40 on stretched 6^3
elements, FP64 arithmetic itself is a few FP32 roundings away, and float-float
must be as close), while the all-FP32 form loses digits in this case (the
contrast shows the case exercises the cancellation).  Solves must reach the
1e-10 reduction, re-checked with the oracle's residual, in the iteration count
of the FP64-residual form with the same smoother.
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


def _round32(c, level, nodal):
    """Condensed FP32 vector of a nodal FP64 array and its values back on the nodal grid (FP64)."""
    x32 = c.pack(level, torch.as_tensor(nodal, device="cuda")).float()
    back = c.unpack(level, x32.double()).cpu().numpy()
    return x32, back


def _case(h, q, lam, seed):
    """(mesh, mask, u, f): u smooth (the manufactured solution), f = Hhat u + 1e-4 perturbation."""
    m = dense.Mesh(h, q, lam)
    mask = matfree.condensed_mask(m)
    u = np.where(mask, workloads.sinsinsin(h, q), 0.0)
    hu = matfree.apply_condensed(m, u)
    rng = np.random.default_rng(seed)
    f = np.where(mask, hu + 1e-4 * np.abs(hu).max() * rng.uniform(-1.0, 1.0, hu.shape), 0.0)
    return m, mask, u, f


def _level_residual_errors(h, p, lam, level_from_top=0):
    from paper_1808_03595_gb300 import Context
    errs = {}
    for precision in ("mixed_ff", "mixed", "mixed_fp32"):
        with Context(h, p, lam, p0=2, precision=precision) as c:
            lv = c.L - level_from_top
            q = c.degrees[lv]
            m, mask, u, f = _case(h, q, lam, 5)
            u32, u_back = _round32(c, lv, u)
            f32, f_back = _round32(c, lv, f)
            ref = f_back - matfree.apply_condensed(m, u_back)  # FP64 residual of the FP32 inputs
            got = c.unpack(lv, c.residual_cycle(lv, f32, u32).double()).cpu().numpy()
            again = c.unpack(lv, c.residual_cycle(lv, f32, u32).double()).cpu().numpy()
            assert np.array_equal(got, again)  # fixed evaluation order: bitwise reproducible
            assert np.all(got[~mask] == 0.0)
            errs[precision] = np.abs(got[mask] - ref[mask]).max() / np.abs(ref[mask]).max()
    return q, errs


@pytest.mark.parametrize("p,n,stretched", [(16, 3, False), (32, 2, False), (20, 2, True), (47, 2, True),
                                           (48, 2, True), (16, 6, True), (40, 6, True)])
def test_ff_level_residual_is_the_rounded_exact_one(p, n, stretched):
    # 6^3 elements: a partial last round on the SMs, so two CTAs share each element
    h = workloads.stretched_widths(n, 23) if stretched else workloads.uniform_widths(n)
    q, errs = _level_residual_errors(h, p, 1.0)
    assert q == p
    # one FP32 rounding of each output entry: at most 2^-24 of the largest entry, with margin;
    # where the cancellation is deep enough that FP64 arithmetic (here and in the oracle's
    # reference) no longer reaches that, the float-float residual is as close as the FP64 one
    fp64_bound = max(2.5e-7, errs["mixed"])
    assert errs["mixed"] < 1e-6, errs
    assert errs["mixed_ff"] < 2.0 * fp64_bound, errs
    # the case is one where FP32 arithmetic loses digits
    assert errs["mixed_fp32"] > 20 * errs["mixed_ff"], errs


def test_ff_levels_below_the_face_form_use_fp64():
    # p = 16: the next level (p = 8) has no face-parallel form, so its residual is the FP64 one
    q, errs = _level_residual_errors(workloads.uniform_widths(3), 16, 1.0, level_from_top=1)
    assert q == 8
    assert errs["mixed_ff"] < 2.5e-7 and errs["mixed"] < 2.5e-7, errs


def test_residual_cycle_rejects_an_fp64_context():
    from paper_1808_03595_gb300 import Context
    from paper_1808_03595_gb300.solver import SemmgError
    h = workloads.uniform_widths(2)
    with Context(h, 16, 1.0, p0=2) as c:
        x = torch.zeros(c.condensed_size(c.L), dtype=torch.float32, device="cuda")
        with pytest.raises(SemmgError):
            c.residual_cycle(c.L, x, x.clone())


@pytest.mark.parametrize("pair", [("mixed_ff", "mixed"), ("mixed_ff_tc", "mixed_tc")])
@pytest.mark.parametrize("p", [16, 32])
def test_ff_solve_matches_the_fp64_residual_form(p, pair):
    from paper_1808_03595_gb300 import Context
    ff_form, ref_form = pair
    h, p, lam, f, p0 = workloads.config(f"helmholtz_8x8x8_p{p}")
    fd = torch.as_tensor(f, device="cuda")
    with Context(h, p, lam, p0=p0, precision=ref_form) as c:
        _, info_ref = c.solve(fd)
    with Context(h, p, lam, p0=p0, precision=ff_form) as c:
        u, info = c.solve(fd)
        u = u.cpu().numpy()
    assert info.status == 0 and info.res_final <= 1e-10 * info.res0
    assert info.iters == info_ref.iters
    m = dense.Mesh(h, p, lam)
    mask = matfree.condensed_mask(m)
    Fh = matfree.condense_rhs(m, f)
    res = Fh - matfree.apply_condensed(m, np.where(mask, u, 0.0))
    assert np.linalg.norm(res[mask]) / np.linalg.norm(Fh[mask]) < 2e-10


def test_ff_tc_p48_full_size_iterations():
    # 6^3 stretched elements, p = 48: FP32 level residuals need one cycle more than FP64 ones
    # here (the reduction after three cycles is just above 1e-10); float-float ones do not
    from paper_1808_03595_gb300 import Context
    h, p, lam, f, p0 = workloads.config("poisson_6x6x6_p48_stretched")
    fd = torch.as_tensor(f, device="cuda")
    iters, red3 = {}, {}
    for precision in ("fp64", "mixed_tc", "mixed_ff_tc"):
        with Context(h, p, lam, p0=p0, precision=precision) as c:
            _, info = c.solve(fd)
            assert info.status == 0 and info.res_final <= 1e-10 * info.res0
            iters[precision] = info.iters
        with Context(h, p, lam, p0=p0, precision=precision, max_iter=3) as c:
            _, info = c.solve(fd, allow_not_converged=True)
            red3[precision] = info.res_final / info.res0
    assert iters["mixed_ff_tc"] == iters["mixed_tc"] == iters["fp64"], iters
    # the float-float form reduces the residual as the FP64-residual form does, cycle for cycle
    assert abs(red3["mixed_ff_tc"] / red3["mixed_tc"] - 1.0) < 0.05, red3


@pytest.mark.parametrize("p,n", [(16, 3), (33, 2), (48, 2), (16, 6), (24, 5)])
def test_ff_condense_and_recover(p, n):
    # 6^3 and 5^3 elements fill the SMs in a partial last round: two CTAs share each element there
    # a solve with no outer iteration condenses f, takes u_hat = 0 and recovers the interiors:
    # u = (0 on the skeleton, H_II^{-1} F_I inside), here in float-float against the FP64 form
    # and the oracle's recovery
    from paper_1808_03595_gb300 import Context
    h = workloads.stretched_widths(n, 29)
    lam = 1.0
    f = workloads.random_nodal(h, p, 31, "uniform")
    fd = torch.as_tensor(f, device="cuda")
    out = {}
    for precision in ("mixed_ff", "fp64"):
        with Context(h, p, lam, p0=2, precision=precision, max_iter=0) as c:
            u, info = c.solve(fd, allow_not_converged=True)
            out[precision] = (u.cpu().numpy(), info.res0)
    u_ff, r_ff = out["mixed_ff"]
    u64, r64 = out["fp64"]
    scale = np.abs(u64).max()
    assert np.abs(u_ff - u64).max() <= 1e-12 * scale
    assert abs(r_ff / r64 - 1.0) < 1e-12  # ||F_hat||: the condensed right-hand side
    m = dense.Mesh(h, p, lam)
    ref = matfree.recover(m, f, np.zeros_like(f))
    assert np.abs(u_ff - ref).max() <= 1e-12 * np.abs(ref).max()
