"""Star smoother with tcgen05 tensor-core transforms (SEMMG_MIXED_TC, _FP32_TC, _BF16).

The four in-plane 1D transforms of Algorithm 1 run as TF32 or BF16 products
with FP32 accumulation; the eigenspace step stays FP32.  The smoother output is
checked against the FP64 oracle at the operand type's tolerance (each of the
four transform stages rounds its operands once: an 11-bit significand for
TF32, 8-bit for BF16), for 16 <= p <= 48, and solves in these forms must still
reach the 1e-10 residual reduction, re-checked with the oracle's own condensed
residual.
"""
import numpy as np
import pytest

import workloads
from oracle import dense, matfree

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_TF32 = 5e-3
TOL_BF16 = 4e-2


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1808_03595_gb300 import build
    build.build()


def _skel(h, p, seed):
    m = dense.Mesh(h, p, 0.0)
    return np.where(matfree.condensed_mask(m), workloads.random_nodal(h, p, seed), 0.0)


@pytest.mark.parametrize("p,n,stretched", [(16, 3, False), (16, 2, True), (32, 2, False), (24, 2, False),
                                           (19, 3, True), (8, 3, False), (33, 2, True), (47, 2, True),
                                           (48, 2, False), (48, 3, True)])
def test_tc_smoother_matches_oracle(p, n, stretched):
    from paper_1808_03595_gb300 import Context
    h = workloads.stretched_widths(n, 11) if stretched else workloads.uniform_widths(n)
    lam = 2.0
    m = dense.Mesh(h, p, lam)
    r = _skel(h, p, 61)
    ref = matfree.smooth(m, r, chunk=16)
    mask = matfree.condensed_mask(m)
    outs = {}
    for precision, tol in (("mixed_tc", TOL_TF32), ("mixed_fp32_tc", TOL_TF32), ("mixed_bf16", TOL_BF16)):
        with Context(h, p, lam, p0=2, precision=precision) as c:
            rh = c.pack(c.L, torch.as_tensor(r, device="cuda")).float()
            got = c.unpack(c.L, c.smooth(c.L, rh).double()).cpu().numpy()
            again = c.unpack(c.L, c.smooth(c.L, rh).double()).cpu().numpy()
        err = np.abs(got[mask] - ref[mask]).max() / np.abs(ref[mask]).max()
        assert err < tol, (precision, err)
        assert np.all(got[~mask] == 0.0)
        assert np.array_equal(got, again)  # fixed summation orders: bitwise reproducible
        outs[precision] = got
    # the TF32 smoother is the same kernel in both cycle forms
    assert np.array_equal(outs["mixed_tc"], outs["mixed_fp32_tc"])


@pytest.mark.parametrize("p", [8, 12, 16, 32, 47, 48])
def test_tc_levels(p):
    # the tensor-core kernel (one 512-thread block per SM at most, 128 registers, no work arrays)
    # takes the FP32 star smoothing on the levels with 16 <= p <= 48
    from paper_1808_03595_gb300 import Context
    h = workloads.uniform_widths(2)
    for precision in ("mixed_tc", "mixed_bf16"):
        with Context(h, p, 1.0, p0=2, precision=precision) as c, Context(h, p, 1.0, p0=2, precision="mixed") as c32:
            for lv in range(1, c.L + 1):
                q = c.degrees[lv]
                tc = c.launch_shape(lv, "star", torch.float32)
                cuda_core = c32.launch_shape(lv, "star", torch.float32)
                if 16 <= q <= 48:
                    assert tc != cuda_core and tc[0] == 512 and tc[3] == 128 and tc[2] <= 152, (q, tc)
                else:
                    assert tc == cuda_core, (q, tc, cuda_core)


@pytest.mark.parametrize("precision", ["mixed_tc", "mixed_fp32_tc", "mixed_bf16"])
@pytest.mark.parametrize("p", [16, 32])
def test_tc_solve_reaches_1e10(p, precision):
    # mixed_fp32_tc: the tensor-core smoother inside the all-FP32 V-cycle (FP32 level residuals)
    from paper_1808_03595_gb300 import Context
    h, p, lam, f, p0 = workloads.config(f"helmholtz_8x8x8_p{p}")
    fd = torch.as_tensor(f, device="cuda")
    with Context(h, p, lam, p0=p0) as c:
        _, info64 = c.solve(fd)
    with Context(h, p, lam, p0=p0, precision=precision) as c:
        u, info = c.solve(fd)
        u = u.cpu().numpy()
    assert info.status == 0 and info.res_final <= 1e-10 * info.res0
    assert info.iters <= info64.iters + (4 if precision == "mixed_bf16" else 2)
    m = dense.Mesh(h, p, lam)
    mask = matfree.condensed_mask(m)
    Fh = matfree.condense_rhs(m, f)
    res = Fh - matfree.apply_condensed(m, np.where(mask, u, 0.0))
    assert np.linalg.norm(res[mask]) / np.linalg.norm(Fh[mask]) < 2e-10


def test_tc_krylov_and_batch():
    from paper_1808_03595_gb300 import Batch, Context
    cases = [(workloads.uniform_widths(3), 16, 1.0), (workloads.stretched_widths(2, 5), 20, 10.0)]
    ctxs, fs, us, refs = [], [], [], []
    for i, (h, p, lam) in enumerate(cases):
        c = Context(h, p, lam, p0=2, precision="mixed_tc", solver="kmg")
        fd = torch.as_tensor(workloads.random_nodal(h, p, 70 + i, "uniform"), device="cuda")
        u_ref, info = c.solve(fd)
        assert info.status == 0 and info.res_final <= 1e-10 * info.res0
        refs.append((u_ref.cpu().numpy(), info.iters))
        ctxs.append(c)
        fs.append(fd)
        us.append(torch.full_like(fd, float("nan")))
    b = Batch(ctxs, fs, us)
    rc, infos = b.solve()
    assert rc == 0
    for (u_ref, it_ref), u, info in zip(refs, us, infos):
        assert info.status == 0 and info.iters == it_ref
        assert np.abs(u.cpu().numpy() - u_ref).max() <= 1e-12 * np.abs(u_ref).max()
    b.close()
    for c in ctxs:
        c.close()


@pytest.mark.parametrize("precision", ["mixed_tc", "mixed_bf16", "mixed_ff_tc"])
def test_tc_solve_stretched_p48_full_size(precision):
    # the 6^3 stretched workload at p = 48: the finest level's smoother on the tensor cores
    from paper_1808_03595_gb300 import Context
    h, p, lam, f, p0 = workloads.config("poisson_6x6x6_p48_stretched")
    fd = torch.as_tensor(f, device="cuda")
    with Context(h, p, lam, p0=p0, precision=precision) as c:
        assert c.launch_shape(c.L, "star", torch.float32)[0] == 512  # the tensor-core kernel at p = 48
        u, info = c.solve(fd)
        u = u.cpu().numpy()
    assert info.status == 0 and info.res_final <= 1e-10 * info.res0
    m = dense.Mesh(h, p, lam)
    mask = matfree.condensed_mask(m)
    Fh = matfree.condense_rhs(m, f)
    res = Fh - matfree.apply_condensed(m, np.where(mask, u, 0.0))
    assert np.linalg.norm(res[mask]) / np.linalg.norm(Fh[mask]) < 2e-10
    assert np.abs(u - workloads.sinsinsin(h, p)).max() < 1e-8
