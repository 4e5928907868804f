"""Failure detection without a GPU fault.

The two failure checks of a context are driven to trip on purpose through
their limits (semmg_set_guards), and the context is used again afterwards:
  - the divergence stop of the outer iteration (Algorithm 4 and the batched
    graph) with a factor below the first iteration's residual reduction;
  - the bounded completion waits of the tensor-core star smoother with a
    budget of 0 cycles: every wait whose products are still in flight runs
    out, the kernel drains its products, frees its tensor memory and returns,
    and the solve reports SEMMG_ERR_TIMEOUT.
Nothing here faults, traps or hangs the GPU: every wait stays bounded and the
kernels return normally.
"""
import ctypes

import numpy as np
import pytest

import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_1808_03595_gb300 import _lib, build
    build.build()
    return _lib.load()


def _solve(lib, ctx, f, u):
    from paper_1808_03595_gb300 import _lib as L
    info = L.semmg_info()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.semmg_solve(ctx._ctx, ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(u.data_ptr()), 1e-10,
                         ctypes.byref(info), stream)
    return rc, info


def test_guards_reject_bad_limits(lib):
    from paper_1808_03595_gb300 import Context
    with Context(workloads.uniform_widths(2), 4, 1.0) as ctx:
        assert lib.semmg_set_guards(ctx._ctx, 0.0, 10) == -1
        assert lib.semmg_set_guards(ctx._ctx, float("nan"), 10) == -1
        assert lib.semmg_set_guards(ctx._ctx, 2.0, -1) == -1
        assert lib.semmg_set_guards(ctx._ctx, float("inf"), 0) == 0


@pytest.mark.parametrize("solver", ["mg", "kmg"])
def test_divergence_stop_trips_on_first_iteration(lib, solver):
    from paper_1808_03595_gb300 import Context
    h, p, lam, f, p0 = workloads.config("helmholtz_8x8x8_p8")
    fd = torch.as_tensor(f, device="cuda")
    u = torch.empty_like(fd)
    with Context(h, p, lam, p0=p0, solver=solver) as ctx:
        # one iteration reduces the residual by about 1e-3; a factor of 1e-9 calls that growth
        ctx.set_guards(divergence=1e-9)
        rc, info = _solve(lib, ctx, fd, u)
        assert rc == -8, rc
        assert info.status == -8 and info.iters == 1
        assert 0 < info.res_final < info.res0
        assert b"diverged" in lib.semmg_last_error(ctx._ctx)
        ctx.set_guards(divergence=1e3)  # the context stays usable
        rc, info = _solve(lib, ctx, fd, u)
        assert rc == 0 and info.res_final <= 1e-10 * info.res0


def test_divergence_stop_in_the_batched_graph():
    from paper_1808_03595_gb300 import Batch, Context
    h, p, lam, f, p0 = workloads.config("helmholtz_8x8x8_p4")
    fd = [torch.as_tensor(f, device="cuda") for _ in range(2)]
    ud = [torch.empty_like(x) for x in fd]
    ctxs = [Context(h, p, lam, p0=p0, precision="mixed") for _ in range(2)]
    ctxs[1].set_guards(divergence=1e-9)  # read when the graph is captured
    b = Batch(ctxs, fd, ud)
    rc, infos = b.solve()
    assert rc == -8
    assert infos[0].status == 0 and infos[0].res_final <= 1e-10 * infos[0].res0
    assert infos[1].status == -8 and infos[1].iters == 1
    b.close()
    for c in ctxs:
        c.close()


@pytest.mark.parametrize("precision", ["mixed_tc", "mixed_fp32_tc"])
def test_tensor_core_wait_runs_out_and_the_context_recovers(lib, precision):
    from paper_1808_03595_gb300 import Context
    h, p = workloads.uniform_widths(3), 16  # p = 16: the finest level runs the tensor-core star kernel
    f = workloads.random_nodal(h, p, 5)
    fd = torch.as_tensor(f, device="cuda")
    u = torch.empty_like(fd)
    with Context(h, p, 1.0, p0=2, precision=precision) as ctx:
        ctx.set_guards(tc_wait_cycles=0)
        rc, _ = _solve(lib, ctx, fd, u)
        assert rc == -6, rc
        assert b"tensor-core" in lib.semmg_last_error(ctx._ctx)
        torch.cuda.synchronize()  # the device is healthy: the kernels returned
        ctx.set_guards()  # default budget: the same context solves again
        rc, info = _solve(lib, ctx, fd, u)
        assert rc == 0 and info.res_final <= 1e-10 * info.res0
    with Context(h, p, 1.0, p0=2, precision=precision) as fresh:
        rc2, info2 = _solve(lib, fresh, fd, torch.empty_like(fd))
        assert rc2 == 0 and info2.iters == info.iters
        # a fresh context reproduces the recovered one's solution bitwise
    u2 = torch.empty_like(fd)
    with Context(h, p, 1.0, p0=2, precision=precision) as fresh:
        _solve(lib, fresh, fd, u2)
    assert torch.equal(u, u2)
