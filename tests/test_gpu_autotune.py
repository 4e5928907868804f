"""Launch autotuning changes only timing: every tuned shape gives bitwise the same results."""
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


@pytest.mark.parametrize("p,precision", [(8, "fp64"), (16, "mixed"), (13, "mixed")])
def test_autotune_is_bitwise_neutral(p, precision):
    from paper_1808_03595_gb300 import Context
    h = workloads.uniform_widths(4)
    f = workloads.random_nodal(h, p, 31, "uniform")
    m = dense.Mesh(h, p, 1.0)
    r = np.where(matfree.condensed_mask(m), workloads.random_nodal(h, p, 32), 0.0)
    out = []
    for tune in (False, True):
        with Context(h, p, 1.0, p0=2, precision=precision) as c:
            if tune:
                c.autotune()
                for lv in range(1, c.nlevels):
                    dt = torch.float32 if precision == "mixed" else torch.float64
                    b, s, g = c.launch_shape(lv, "star", dt)
                    assert b in (256, 512) and g >= 1 and 0 <= s <= 200 * 1024
            rh = c.pack(c.L, torch.as_tensor(r, device="cuda"))
            dt = torch.float32 if precision == "mixed" else torch.float64
            du = c.smooth(c.L, rh.to(dt)).double().cpu().numpy()
            y = c.apply_condensed(c.L, rh).cpu().numpy()
            u, info = c.solve(torch.as_tensor(f, device="cuda"))
            out.append((du, y, u.cpu().numpy(), info.iters))
    (d0, y0, u0, i0), (d1, y1, u1, i1) = out
    assert np.array_equal(d0, d1)
    assert np.array_equal(y0, y1)
    assert np.array_equal(u0, u1) and i0 == i1
