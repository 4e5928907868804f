"""The allocation-free smoothing entry point agrees with semmg_smooth.

semmg_smooth_noalloc serves callers that must not allocate device memory
while they work (a memory manager that owns the device, a thread that cannot
take cudaMalloc's synchronisation); it runs the same kernels with their
scratch in a fixed array inside the library.  This file is collected last on
purpose: a failure here leaves every other test already run.
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


@pytest.mark.parametrize("p,dtype", [(4, torch.float64), (16, torch.float64), (8, torch.float32),
                                     (16, torch.float32)])
def test_noalloc_smooth_matches_smooth_twice(lib, p, dtype):
    from paper_1808_03595_gb300 import Context
    h = workloads.uniform_widths(4) if p <= 8 else [np.full(3, 1 / 3), np.full(2, 0.5), np.full(3, 1 / 3)]
    mesh = dense.Mesh(h, p, 1.0)
    mask = matfree.condensed_mask(mesh)
    r_nodal = np.where(mask, workloads.random_nodal(h, p, 4242), 0.0)
    tol = TOL64 if dtype == torch.float64 else TOL32
    with Context(h, p, 1.0, p0=2) as ctx:
        r = ctx.pack(ctx.L, torch.as_tensor(r_nodal, device="cuda")).to(dtype)
        ref = ctx.smooth(ctx.L, r).double()
        scale = float(ref.abs().max())
        assert scale > 0
        for _ in range(2):  # two calls in a row share the library's scratch array
            out = torch.full_like(r, float("nan"))
            assert _noalloc(lib, ctx, ctx.L, r, out) == 0
            torch.cuda.synchronize()
            assert float((out.double() - ref).abs().max()) <= tol * scale


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
