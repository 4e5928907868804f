"""The batched, graph-captured form gives the same solves as one-at-a-time solving.

Each solve of the batch is one branch of a single CUDA graph with a device-side
loop; results must equal the stand-alone semmg_solve of the same context
(same kernels, same order of operations), iteration counts included.
"""
import numpy as np
import pytest

import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1808_03595_gb300 import build
    build.build()


def _case(n, p, lam, seed, precision):
    h = workloads.uniform_widths(n) if seed % 2 else workloads.stretched_widths(n, seed)
    f = workloads.random_nodal(h, p, seed, "uniform")
    return h, p, lam, f, precision


CASES = [_case(2, 4, 0.01, 1, "fp64"), _case(3, 7, 5.0, 2, "mixed"), _case(4, 5, 300.0, 3, "fp64"),
         _case(2, 12, 1.0, 5, "mixed_fp32"), _case(3, 9, 0.0, 4, "fp64"), _case(3, 14, 1.0, 6, "mixed_ff_tc"),
         _case(2, 16, 2.0, 7, "mixed_ff")]


def test_batch_equals_individual_solves_and_relaunches():
    from paper_1808_03595_gb300 import Batch, Context
    ctxs, fs, us, refs = [], [], [], []
    for h, p, lam, f, prec in CASES:
        c = Context(h, p, lam, p0=2, precision=prec)
        fd = torch.as_tensor(f, device="cuda")
        u_ref, info = c.solve(fd)
        refs.append((u_ref.cpu().numpy(), info.iters))
        ctxs.append(c)
        fs.append(fd)
        us.append(torch.full_like(fd, float("nan")))
    b = Batch(ctxs, fs, us)
    assert b.graph_nodes() >= 3 * len(CASES)
    for rep in range(2):  # the captured graph is relaunched
        for u in us:
            u.fill_(float("nan"))
        rc, infos = b.solve()
        assert rc == 0
        for (u_ref, it_ref), u, info in zip(refs, us, infos):
            got = u.cpu().numpy()
            assert info.status == 0
            assert info.iters == it_ref
            assert info.res_final <= 1e-10 * info.res0
            assert np.abs(got - u_ref).max() <= 1e-12 * np.abs(u_ref).max()
    b.close()
    for c in ctxs:
        c.close()


def test_batch_device_side_stopping_status():
    from paper_1808_03595_gb300 import Batch, Context
    h, p, lam, f, _ = _case(3, 6, 1.0, 7, "fp64")
    c1 = Context(h, p, lam, p0=2, max_iter=1)
    c2 = Context(h, p, lam, p0=2)
    f1 = torch.as_tensor(f, device="cuda")
    f2 = torch.as_tensor(f, device="cuda").clone()
    f2[2, 2, 2] = float("nan")
    u1, u2 = torch.empty_like(f1), torch.empty_like(f2)
    b = Batch([c1, c2], [f1, f2], [u1, u2])
    rc, infos = b.solve()
    assert infos[0].status == -4 and infos[0].iters == 1   # cycle cap reached on the device
    assert infos[1].status == -5                           # non-finite residual detected on the device
    assert rc == -4
    b.close()
    c1.close()
    c2.close()


def test_batch_rejects_a_context_twice():
    from paper_1808_03595_gb300 import Batch, Context
    from paper_1808_03595_gb300.solver import SemmgError
    h, p, lam, f, _ = _case(2, 4, 1.0, 9, "fp64")
    c = Context(h, p, lam)
    fd = torch.as_tensor(f, device="cuda")
    with pytest.raises(SemmgError):
        Batch([c, c], [fd, fd], [torch.empty_like(fd), torch.empty_like(fd)])
    c.close()


def test_batch_with_dirichlet_data_and_element_smoother():
    # per-solve Dirichlet data (None: homogeneous) and the element-centred smoother inside the graph:
    # each branch equals its stand-alone semmg_solve_dirichlet / semmg_solve
    from paper_1808_03595_gb300 import Batch, Context
    specs = [(workloads.uniform_widths(3), 6, 0.0, "fp64", "star", True),
             (workloads.stretched_widths(3, 8), 5, 1.0, "mixed", "element", True),
             (workloads.uniform_widths(2), 8, 2.0, "fp64", "star", False)]
    ctxs, fs, gs, us, refs = [], [], [], [], []
    for i, (h, p, lam, prec, sm, lifted) in enumerate(specs):
        c = Context(h, p, lam, p0=2, precision=prec, smoother=sm)
        fd = torch.as_tensor(workloads.random_nodal(h, p, 90 + i, "uniform"), device="cuda")
        gd = torch.as_tensor(workloads.random_nodal(h, p, 95 + i, "uniform"), device="cuda") if lifted else None
        u_ref, info = c.solve(fd, g=gd)
        refs.append((u_ref.cpu().numpy(), info.iters))
        ctxs.append(c)
        fs.append(fd)
        gs.append(gd)
        us.append(torch.full_like(fd, float("nan")))
    b = Batch(ctxs, fs, us, g_list=gs)
    rc, infos = b.solve()
    assert rc == 0
    for (u_ref, it_ref), u, info in zip(refs, us, infos):
        assert info.status == 0 and info.iters == it_ref
        assert np.abs(u.cpu().numpy() - u_ref).max() <= 1e-12 * np.abs(u_ref).max()
    b.close()
    for c in ctxs:
        c.close()
