"""Python binding of the semmg C ABI: argument marshalling for torch CUDA tensors.

Every computation happens inside libsemmg.so; this module only passes device
pointers, sizes and the current CUDA stream.
"""
import ctypes

import numpy as np
import torch

from . import _lib as L


class SemmgError(RuntimeError):
    def __init__(self, code, msg=""):
        super().__init__(f"{L.ERRORS.get(code, code)}: {msg}")
        self.code = code


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


class Context:
    """A semmg context: mesh (per-axis element widths), degree p, lambda >= 0, options."""

    def __init__(self, h, p, lam, p0=2, nu_pre=1, nu_post=1, precision="fp64", max_iter=50, solver="mg",
                 nu_vary=False, bc=None, stream=None, smoother="star"):
        self._lib = L.load()
        self._ctx = ctypes.c_void_p()
        self.h = [np.ascontiguousarray(np.asarray(hd, dtype=np.float64)) for hd in h]
        self.n = [len(hd) for hd in self.h]
        self.p = int(p)
        self.lam = float(lam)
        mesh = L.semmg_mesh()
        for d in range(3):
            mesh.n[d] = self.n[d]
            mesh.h[d] = self.h[d].ctypes.data_as(L.P_double)
        # faces -x1, +x1, -x2, +x2, -x3, +x3: "D" (Dirichlet, default), "N" (Neumann), "P" (periodic)
        self.bc = tuple(bc) if bc is not None else ("D",) * 6
        if len(self.bc) != 6 or any(b not in ("D", "N", "P") for b in self.bc):
            raise ValueError("bc: six entries, each 'D', 'N' or 'P'")
        kinds = {"D": L.SEMMG_BC_DIRICHLET, "N": L.SEMMG_BC_NEUMANN, "P": L.SEMMG_BC_PERIODIC}
        for f in range(6):
            mesh.bc[f] = kinds[self.bc[f]]
        opts = L.semmg_opts()
        self._lib.semmg_default_opts(ctypes.byref(opts))
        opts.p0 = p0
        opts.nu_pre = nu_pre
        opts.nu_post = nu_post
        opts.precision = {"fp64": L.SEMMG_FP64, "mixed": L.SEMMG_MIXED, "mixed_fp32": L.SEMMG_MIXED_FP32,
                          "mixed_tc": L.SEMMG_MIXED_TC, "mixed_fp32_tc": L.SEMMG_MIXED_FP32_TC,
                          "mixed_bf16": L.SEMMG_MIXED_BF16, "mixed_ff": L.SEMMG_MIXED_FF,
                          "mixed_ff_tc": L.SEMMG_MIXED_FF_TC}[precision]
        opts.max_iter = max_iter
        opts.solver = {"mg": L.SEMMG_SOLVER_MG, "kmg": L.SEMMG_SOLVER_KMG}[solver]
        opts.nu_vary = 1 if nu_vary else 0
        # "star": vertex stars (Algorithms 1 and 2); "element" / "element_mult": element-centred blocks
        # (Sec. 3.4) weighted one on the element / by the inverse multiplicity
        opts.smoother = {"star": L.SEMMG_SMOOTHER_STAR, "element": L.SEMMG_SMOOTHER_ELEMENT,
                         "element_mult": L.SEMMG_SMOOTHER_ELEMENT_MULT}[smoother]
        self.smoother = smoother
        self.precision = precision
        self.solver = solver
        rc = self._lib.semmg_setup(ctypes.byref(mesh), self.p, self.lam, ctypes.byref(opts), _stream(stream),
                                   ctypes.byref(self._ctx))
        if rc != 0:
            raise SemmgError(rc, "setup")
        nl = ctypes.c_int()
        self._check(self._lib.semmg_num_levels(self._ctx, ctypes.byref(nl)))
        self.nlevels = nl.value
        self.degrees = []
        for lv in range(self.nlevels):
            q = ctypes.c_int()
            self._check(self._lib.semmg_level_degree(self._ctx, lv, ctypes.byref(q)))
            self.degrees.append(q.value)

    # ------------------------------------------------------------ helpers
    def _check(self, rc, allow=()):
        if rc != 0 and rc not in allow:
            msg = self._lib.semmg_last_error(self._ctx).decode() if self._ctx else ""
            raise SemmgError(rc, msg)
        return rc

    def close(self):
        if self._ctx:
            self._lib.semmg_destroy(self._ctx)
            self._ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def L(self):
        return self.nlevels - 1

    def condensed_size(self, level=None):
        n = ctypes.c_int64()
        self._check(self._lib.semmg_condensed_size(self._ctx, self.L if level is None else level, ctypes.byref(n)))
        return n.value

    def nodal_size(self, level=None):
        n = ctypes.c_int64()
        self._check(self._lib.semmg_nodal_size(self._ctx, self.L if level is None else level, ctypes.byref(n)))
        return n.value

    def nodal_shape(self, level=None):
        q = self.degrees[self.L if level is None else level]
        return (self.n[2] * q + 1, self.n[1] * q + 1, self.n[0] * q + 1)

    def _hat(self, level, dtype=torch.float64):
        return torch.zeros(self.condensed_size(level), dtype=dtype, device="cuda")

    # ------------------------------------------------------------ entry points
    def pack(self, level, u_nodal, out=None):
        out = self._hat(level) if out is None else out
        self._check(self._lib.semmg_pack(self._ctx, level, _ptr(u_nodal), _ptr(out), _stream()))
        return out

    def pack_dirichlet(self, level, g_nodal, out=None):
        """E g: the Dirichlet-face values of g_nodal in their skeleton slots, zero elsewhere."""
        out = self._hat(level) if out is None else out
        self._check(self._lib.semmg_pack_dirichlet(self._ctx, level, _ptr(g_nodal), _ptr(out), _stream()))
        return out

    def unpack(self, level, u_hat, out=None):
        out = torch.zeros(self.nodal_shape(level), dtype=torch.float64, device="cuda") if out is None else out
        self._check(self._lib.semmg_unpack(self._ctx, level, _ptr(u_hat), _ptr(out), _stream()))
        return out

    def apply_condensed(self, level, u, out=None):
        out = self._hat(level) if out is None else out
        self._check(self._lib.semmg_apply_condensed(self._ctx, level, _ptr(u), _ptr(out), _stream()))
        return out

    def residual(self, level, f, u, out=None):
        out = self._hat(level) if out is None else out
        self._check(self._lib.semmg_residual(self._ctx, level, _ptr(f), _ptr(u), _ptr(out), _stream()))
        return out

    def residual_cycle(self, level, f, u, out=None):
        """The V-cycle's level residual f - Hhat u of a mixed context: FP32 vectors, the context's arithmetic."""
        out = self._hat(level, torch.float32) if out is None else out
        self._check(self._lib.semmg_residual_cycle(self._ctx, level, _ptr(f), _ptr(u), _ptr(out), _stream()))
        return out

    @staticmethod
    def _dtype_code(t):
        if t.dtype == torch.float64:
            return L.SEMMG_F64
        if t.dtype == torch.float32:
            return L.SEMMG_F32
        raise TypeError("float32 or float64 tensors only")

    def smooth(self, level, r, out=None):
        out = self._hat(level, r.dtype) if out is None else out
        self._check(self._lib.semmg_smooth(self._ctx, level, self._dtype_code(r), _ptr(r), _ptr(out), _stream()))
        return out

    def restrict(self, level, fine, out=None):
        out = self._hat(level - 1, fine.dtype) if out is None else out
        self._check(self._lib.semmg_restrict(self._ctx, level, self._dtype_code(fine), _ptr(fine), _ptr(out),
                                             _stream()))
        return out

    def prolong_add(self, level, coarse, fine):
        self._check(self._lib.semmg_prolong_add(self._ctx, level, self._dtype_code(coarse), _ptr(coarse),
                                                _ptr(fine), _stream()))
        return fine

    def coarse_solve(self, f0, out=None):
        out = self._hat(0) if out is None else out
        self._check(self._lib.semmg_coarse_solve(self._ctx, _ptr(f0), _ptr(out), _stream()))
        return out

    def vcycle(self, u, f):
        self._check(self._lib.semmg_vcycle(self._ctx, _ptr(u), _ptr(f), _stream()))
        return u

    def condense_rhs(self, f_nodal, out=None):
        out = self._hat(self.L) if out is None else out
        self._check(self._lib.semmg_condense_rhs(self._ctx, _ptr(f_nodal), _ptr(out), _stream()))
        return out

    def recover(self, f_nodal, u_hat, out=None):
        out = torch.zeros(self.nodal_shape(), dtype=torch.float64, device="cuda") if out is None else out
        self._check(self._lib.semmg_recover(self._ctx, _ptr(f_nodal), _ptr(u_hat), _ptr(out), _stream()))
        return out

    def solve(self, f_nodal, rtol=1e-10, out=None, allow_not_converged=False, g=None):
        """Solve for u; g (nodal, optional): inhomogeneous Dirichlet data, read on the Dirichlet faces."""
        out = torch.empty(self.nodal_shape(), dtype=torch.float64, device="cuda") if out is None else out
        info = L.semmg_info()
        allow = (L.SEMMG_ERR_NOT_CONVERGED,) if allow_not_converged else ()
        if g is None:
            rc = self._lib.semmg_solve(self._ctx, _ptr(f_nodal), _ptr(out), rtol, ctypes.byref(info), _stream())
        else:
            rc = self._lib.semmg_solve_dirichlet(self._ctx, _ptr(f_nodal), _ptr(g), _ptr(out), rtol,
                                                 ctypes.byref(info), _stream())
        self._check(rc, allow)
        return out, info

    def solve_host(self, f_host, u_host, rtol=1e-10, allow_not_converged=False):
        """f_host, u_host: contiguous float64 CPU tensors (pinned for asynchronous copies)."""
        info = L.semmg_info()
        allow = (L.SEMMG_ERR_NOT_CONVERGED,) if allow_not_converged else ()
        self._check(self._lib.semmg_solve_host(self._ctx, _ptr(f_host), _ptr(u_host), rtol, ctypes.byref(info),
                                               _stream()), allow)
        return u_host, info

    # ------------------------------------------------------------ launch tuning
    def autotune(self):
        """Pick the fastest launch shape per level for the star and element kernels (semmg_autotune)."""
        self._check(self._lib.semmg_autotune(self._ctx, _stream()))

    def launch_shape(self, level, kernel, dtype=torch.float64):
        """(block, shared-memory bytes, grid, registers per thread) of kernel 'star' or 'schur' at a level."""
        b, s, g, r = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        self._check(self._lib.semmg_get_launch(self._ctx, level, {"star": 0, "schur": 1}[kernel],
                                               L.SEMMG_F32 if dtype == torch.float32 else L.SEMMG_F64,
                                               ctypes.byref(b), ctypes.byref(s), ctypes.byref(g), ctypes.byref(r)))
        return b.value, s.value, g.value, r.value

    def set_launch(self, level, kernel, dtype, smem_cap, block, max_regs):
        """Pin the launch shape of kernel 'star' or 'schur' at a level (semmg_set_launch)."""
        self._check(self._lib.semmg_set_launch(self._ctx, level, {"star": 0, "schur": 1}[kernel],
                                               L.SEMMG_F32 if dtype == torch.float32 else L.SEMMG_F64,
                                               int(smem_cap), int(block), int(max_regs)))

    # ------------------------------------------------------------ failure detection
    def set_guards(self, divergence=1e3, tc_wait_cycles=4_000_000_000):
        """Divergence factor of the outer iteration and the budget of each tensor-core wait (semmg_set_guards)."""
        self._check(self._lib.semmg_set_guards(self._ctx, float(divergence), int(tc_wait_cycles)))

    # ------------------------------------------------------------ timing
    def set_timing(self, enable=True):
        self._check(self._lib.semmg_set_timing(self._ctx, 1 if enable else 0))

    def reset_kstats(self):
        self._check(self._lib.semmg_reset_kstats(self._ctx))

    def kstats(self):
        """Per kernel class: dict(ms, launches, flops, bytes) accumulated since the last reset."""
        out = {}
        for i, name in enumerate(L.KSTAT_KINDS):
            k = L.semmg_kstat()
            self._check(self._lib.semmg_get_kstat(self._ctx, i, ctypes.byref(k)))
            out[name] = {"ms": k.ms, "launches": k.launches, "flops": k.flops, "bytes": k.bytes, "xflops": k.xflops}
        return out


class Batch:
    """Independent solves of several contexts captured into one CUDA graph (semmg_batch_*).

    f_list / u_list are device nodal tensors that the graph keeps using; refill
    the f tensors in place and call solve() again to solve new right-hand sides.
    """

    def __init__(self, ctxs, f_list, u_list, rtol=1e-10, stream=None, g_list=None):
        """g_list (optional): per solve a device nodal tensor of Dirichlet data, or None."""
        self._lib = L.load()
        self._b = ctypes.c_void_p()
        self.ctxs, self.f, self.u = list(ctxs), list(f_list), list(u_list)
        self.g = list(g_list) if g_list is not None else None
        nb = len(self.ctxs)
        arr = (ctypes.c_void_p * nb)
        ctx_a = arr(*[c._ctx.value for c in self.ctxs])
        f_a, u_a = arr(*[t.data_ptr() for t in self.f]), arr(*[t.data_ptr() for t in self.u])
        if self.g is None:
            rc = self._lib.semmg_batch_create(ctx_a, nb, f_a, u_a, rtol, _stream(stream), ctypes.byref(self._b))
        else:
            g_a = arr(*[(t.data_ptr() if t is not None else None) for t in self.g])
            rc = self._lib.semmg_batch_create_dirichlet(ctx_a, nb, f_a, g_a, u_a, rtol, _stream(stream),
                                                        ctypes.byref(self._b))
        if rc != 0:
            raise SemmgError(rc, "batch_create")

    def solve(self, stream=None):
        """Launch the graph, wait, and return (status, [info per solve])."""
        nb = len(self.ctxs)
        infos = (L.semmg_info * nb)()
        rc = self._lib.semmg_batch_solve(self._b, infos, _stream(stream))
        if rc not in (0, L.SEMMG_ERR_NOT_CONVERGED, L.SEMMG_ERR_NONFINITE, L.SEMMG_ERR_DIVERGED):
            raise SemmgError(rc, "batch_solve")
        return rc, list(infos)

    def graph_nodes(self):
        n = ctypes.c_int64()
        self._lib.semmg_batch_graph_nodes(self._b, ctypes.byref(n))
        return n.value

    def close(self):
        if self._b:
            self._lib.semmg_batch_destroy(self._b)
            self._b = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def peak_tflops(dtype=torch.float64, stream=None):
    """Measured FMA-chain peak of the current device in TFLOP/s (semmg_peak_tflops)."""
    lib = L.load()
    out = ctypes.c_double()
    rc = lib.semmg_peak_tflops(L.SEMMG_F64 if dtype == torch.float64 else L.SEMMG_F32, ctypes.byref(out),
                               _stream(stream))
    if rc != 0:
        raise SemmgError(rc, "peak_tflops")
    return out.value
