"""The C-ABI library builds for sm_103a, loads, and exports every symbol include/semmg.h declares.

No compute call is made here (no GPU needed).
"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "semmg.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(semmg_\w+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_1808_03595_gb300 import build, _lib
    build.build()
    return _lib.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["semmg_setup", "semmg_apply_condensed", "semmg_smooth", "semmg_vcycle", "semmg_solve",
                     "semmg_restrict", "semmg_prolong_add", "semmg_coarse_solve", "semmg_condense_rhs",
                     "semmg_recover", "semmg_destroy"]:
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    from paper_1808_03595_gb300 import _lib
    names = declared_functions()
    for name in names:
        assert hasattr(lib, name), name
        assert name in _lib.SIGNATURES, name
    assert set(_lib.SIGNATURES) == set(names)


def test_strerror_without_gpu(lib):
    assert lib.semmg_strerror(0) == b"success"
    assert lib.semmg_strerror(-4) == b"not converged"
    assert lib.semmg_strerror(-8) == b"residual diverged"
    from paper_1808_03595_gb300 import _lib as L
    for code in L.ERRORS:
        assert lib.semmg_strerror(code) != lib.semmg_strerror(12345), code
    assert lib.semmg_last_error(None) == b"null context"


def test_setup_rejects_bad_arguments_without_touching_the_gpu(lib):
    from paper_1808_03595_gb300 import _lib as L
    ctx = ctypes.c_void_p()
    assert lib.semmg_setup(None, 4, 1.0, None, None, ctypes.byref(ctx)) == -1
    mesh = L.semmg_mesh()
    for d in range(3):
        mesh.n[d] = 2
    # null width arrays
    assert lib.semmg_setup(ctypes.byref(mesh), 4, 1.0, None, None, ctypes.byref(ctx)) == -1
    import numpy as np
    h = np.full(2, 0.5)
    for d in range(3):
        mesh.h[d] = h.ctypes.data_as(L.P_double)
    assert lib.semmg_setup(ctypes.byref(mesh), 0, 1.0, None, None, ctypes.byref(ctx)) == -2
    assert lib.semmg_setup(ctypes.byref(mesh), 49, 1.0, None, None, ctypes.byref(ctx)) == -2
    assert lib.semmg_setup(ctypes.byref(mesh), 4, -1.0, None, None, ctypes.byref(ctx)) == -1
    opts = L.semmg_opts()
    lib.semmg_default_opts(ctypes.byref(opts))
    assert (opts.p0, opts.nu_pre, opts.nu_post, opts.precision, opts.max_iter) == (2, 1, 1, 0, 50)
    assert (opts.solver, opts.nu_vary, opts.smoother) == (L.SEMMG_SOLVER_MG, 0, L.SEMMG_SMOOTHER_STAR)
    opts.smoother = 5
    assert lib.semmg_setup(ctypes.byref(mesh), 4, 1.0, ctypes.byref(opts), None, ctypes.byref(ctx)) == -1
    # element-centred blocks span three elements: a periodic axis of two is unsupported
    opts.smoother = L.SEMMG_SMOOTHER_ELEMENT
    mesh.bc[0] = mesh.bc[1] = L.SEMMG_BC_PERIODIC
    assert lib.semmg_setup(ctypes.byref(mesh), 4, 1.0, ctypes.byref(opts), None, ctypes.byref(ctx)) == -2
    mesh.bc[0] = mesh.bc[1] = L.SEMMG_BC_DIRICHLET
    opts.smoother = L.SEMMG_SMOOTHER_STAR
    opts.solver = 7
    assert lib.semmg_setup(ctypes.byref(mesh), 4, 1.0, ctypes.byref(opts), None, ctypes.byref(ctx)) == -1
    opts.solver = L.SEMMG_SOLVER_KMG
    opts.nu_vary = 2
    assert lib.semmg_setup(ctypes.byref(mesh), 4, 1.0, ctypes.byref(opts), None, ctypes.byref(ctx)) == -1
    opts.nu_vary = 0
    opts.p0 = 8
    assert lib.semmg_setup(ctypes.byref(mesh), 4, 1.0, ctypes.byref(opts), None, ctypes.byref(ctx)) == -2
    # boundary conditions: unknown kind rejected; pure Neumann needs lambda > 0 (singular otherwise)
    mesh.bc[3] = 7
    assert lib.semmg_setup(ctypes.byref(mesh), 4, 1.0, None, None, ctypes.byref(ctx)) == -1
    for f in range(6):
        mesh.bc[f] = L.SEMMG_BC_NEUMANN
    assert lib.semmg_setup(ctypes.byref(mesh), 4, 0.0, None, None, ctypes.byref(ctx)) == -2
    for f in range(6):
        mesh.bc[f] = L.SEMMG_BC_DIRICHLET
    hbad = np.array([0.5, -0.5])
    mesh.h[0] = hbad.ctypes.data_as(L.P_double)
    assert lib.semmg_setup(ctypes.byref(mesh), 4, 1.0, None, None, ctypes.byref(ctx)) == -1
    assert not ctx.value


def test_guards_and_peak_probe_reject_bad_arguments_without_a_gpu(lib):
    import ctypes as C
    assert lib.semmg_set_guards(None, 1e3, 10) == -1
    out = C.c_double()
    assert lib.semmg_peak_tflops(7, C.byref(out), None) == -1
    assert lib.semmg_peak_tflops(0, None, None) == -1
