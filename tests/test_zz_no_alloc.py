"""The allocation-free smoothing entry point agrees with semmg_smooth and the oracle.

semmg_smooth_noalloc serves callers that must not allocate device memory
while they work (a memory manager that owns the device, a thread that cannot
take cudaMalloc's synchronisation); it runs the same kernels as semmg_smooth,
the tensor-core star kernel included where the context's precision takes it,
with their scratch in a fixed array inside the library.  This file is
collected last on purpose: a failure here leaves every other test already run.
"""
import ctypes

import numpy as np
import pytest

import workloads
from oracle import dense, matfree

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 2e-5
TOL_TF32 = 5e-3


@pytest.fixture(scope="module")
def lib():
    from paper_1808_03595_gb300 import _lib, build
    build.build()
    return _lib.load()


def _noalloc(lib, ctx, level, r, out):
    code = 0 if r.dtype == torch.float64 else 1
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return lib.semmg_smooth_noalloc(ctx._ctx, level, code, ctypes.c_void_p(r.data_ptr()),
                                    ctypes.c_void_p(out.data_ptr()), stream)


def _mesh(p):
    return workloads.uniform_widths(4) if p <= 8 else [np.full(3, 1 / 3), np.full(2, 0.5), np.full(3, 1 / 3)]


# (degree, element type, precision of the context): the last two cases run the tensor-core
# star kernel in both entry points (16 <= p <= 32 in the SEMMG_MIXED_TC / _FP32_TC forms)
@pytest.mark.parametrize("p,dtype,precision", [(4, torch.float64, "fp64"), (16, torch.float64, "fp64"),
                                               (8, torch.float32, "mixed"), (16, torch.float32, "mixed"),
                                               (16, torch.float32, "mixed_tc"),
                                               (32, torch.float32, "mixed_fp32_tc")])
def test_noalloc_smooth_matches_smooth_twice(lib, p, dtype, precision):
    from paper_1808_03595_gb300 import Context
    h = _mesh(p) if p < 32 else workloads.uniform_widths(2)
    mesh = dense.Mesh(h, p, 1.0)
    mask = matfree.condensed_mask(mesh)
    r_nodal = np.where(mask, workloads.random_nodal(h, p, 4242), 0.0)
    tol = TOL64 if dtype == torch.float64 else TOL32
    with Context(h, p, 1.0, p0=2, precision=precision) as ctx:
        r = ctx.pack(ctx.L, torch.as_tensor(r_nodal, device="cuda")).to(dtype)
        ref = ctx.smooth(ctx.L, r).double()
        scale = float(ref.abs().max())
        assert scale > 0
        for _ in range(2):  # two calls in a row share the library's scratch array
            out = torch.full_like(r, float("nan"))
            assert _noalloc(lib, ctx, ctx.L, r, out) == 0
            torch.cuda.synchronize()
            assert float((out.double() - ref).abs().max()) <= tol * scale


@pytest.mark.parametrize("precision,dtype,tol", [("fp64", torch.float64, TOL64),
                                                 ("mixed_tc", torch.float32, TOL_TF32)])
def test_noalloc_smooth_matches_oracle(lib, precision, dtype, tol):
    # the allocation-free smoother against the oracle's Algorithm 2 (matrix-free), at the
    # tolerance of the arithmetic that runs: FP64, or TF32 tensor-core transforms
    from paper_1808_03595_gb300 import Context
    h = workloads.stretched_widths(3, 11)
    p, lam = 16, 2.0
    m = dense.Mesh(h, p, lam)
    mask = matfree.condensed_mask(m)
    r_nodal = np.where(mask, workloads.random_nodal(h, p, 77), 0.0)
    ref = matfree.smooth(m, r_nodal, chunk=16)
    with Context(h, p, lam, p0=2, precision=precision) as ctx:
        r = ctx.pack(ctx.L, torch.as_tensor(r_nodal, device="cuda")).to(dtype)
        out = torch.full_like(r, float("nan"))
        assert _noalloc(lib, ctx, ctx.L, r, out) == 0
        got = ctx.unpack(ctx.L, out.double()).cpu().numpy()
    err = np.abs(got[mask] - ref[mask]).max() / np.abs(ref[mask]).max()
    assert err < tol, err


def test_noalloc_rejects_levels_beyond_the_scratch(lib):
    from paper_1808_03595_gb300 import Context, _lib
    # 16^3 elements at p = 16: the star output buffer alone is 4913 * 3 * 31^2 doubles (about 113 MB)
    h = workloads.uniform_widths(16)
    with Context(h, 16, 1.0, p0=2) as ctx:
        r = torch.zeros(ctx.condensed_size(), dtype=torch.float64, device="cuda")
        out = torch.zeros_like(r)
        rc = _noalloc(lib, ctx, ctx.L, r, out)
        assert rc == -2
        msg = lib.semmg_last_error(ctx._ctx).decode()
        assert str(_lib.SEMMG_NOALLOC_SCRATCH_BYTES) in msg
