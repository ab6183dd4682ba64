"""ctypes binding of libfehom.so (include/fehom.h): argument marshalling only.

Every step of the solve runs in the library's CUDA kernels; this module passes pointers, sizes and
the CUDA stream, and uses torch tensors for device memory.  There is no CPU fallback: loading
fails loudly when the library is missing.

    s = Solver("hex8_3d", "elastic", (128, 128, 128), ids, moduli)
    s.precond_build()
    out = s.solve(loads, tol=1e-6)        # out["C_eff"], out["mean_flux"], out["fields"], out["info"]
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfehom.so")

ELEM = {"p1tri2_2d": 1, "hex8_3d": 2, "q1_2d": 3, "p1tri4_2d": 4}
PHYSICS = {"scalar": 1, "elastic": 2}
PRECISION = {"fp64": 0, "mixed": 1}
STATUS = {0: "FEHOM_OK", 1: "FEHOM_E_INVALID", 2: "FEHOM_E_UNSUPPORTED_SIZE", 3: "FEHOM_E_OOM",
          4: "FEHOM_E_CUDA", 5: "FEHOM_E_NOT_CONVERGED", 6: "FEHOM_E_BREAKDOWN", 7: "FEHOM_E_STATE"}

# every entry point declared in include/fehom.h
EXPORTS = ("fehom_default_options", "fehom_setup", "fehom_precond_build", "fehom_solve", "fehom_destroy",
           "fehom_last_error", "fehom_query", "fehom_apply_stiffness", "fehom_rhs", "fehom_apply_precond",
           "fehom_get_symbol_inverse", "fehom_mean_flux", "fehom_kernel_times", "fehom_launch_count",
           "fehom_fft_plan", "fehom_mean_flux_noalloc", "fehom_pcg_coefficients", "fehom_eig_bounds",
           "fehom_batch_create", "fehom_solve_batch", "fehom_batch_destroy", "fehom_batch_last_error",
           "fehom_effective_energy", "fehom_set_reference", "fehom_newton_solve", "fehom_residual_update",
           "fehom_stencil_plan", "fehom_rhs_df", "fehom_pcg_apply_stiffness", "fehom_pcg_precond_step",
           # include/fehom_unet.h
           "fehom_unet_create", "fehom_unet_destroy", "fehom_unet_last_error", "fehom_unet_param_count",
           "fehom_unet_set_params", "fehom_unet_get_params", "fehom_unet_predict", "fehom_unet_loss_grad",
           "fehom_unet_train_step", "fehom_conv3_bf16", "fehom_conv3_wgrad_bf16", "fehom_unet_set_loss")

KERNEL_CLASSES = ("stiffness", "fft_x_fwd", "fft_y_fwd", "fft_last", "fft_y_inv", "fft_x_inv")


class Options(C.Structure):
    _fields_ = [("precision", C.c_int), ("max_iter", C.c_int), ("inner_tol", C.c_double),
                ("stream", C.c_void_p), ("use_graph", C.c_int), ("profile", C.c_int),
                ("autotune", C.c_int), ("x0_scaling", C.c_int), ("fft_xy", C.c_int), ("residual_df", C.c_int),
                ("stencil_rows", C.c_int)]


class SolveInfo(C.Structure):
    _fields_ = [("iterations", C.c_int), ("refinements", C.c_int), ("converged", C.c_int),
                ("rel_residual_M", C.c_double), ("rel_residual_2", C.c_double), ("solve_ms", C.c_double)]


class NewtonInfo(C.Structure):
    _fields_ = [("newton_iterations", C.c_int), ("pcg_iterations", C.c_int), ("converged", C.c_int),
                ("n_hist", C.c_int), ("residual", C.c_double * 32), ("increment", C.c_double * 32),
                ("pcg_per_step", C.c_int * 32)]


class FehomError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


_lib = None


def load_library(path: str = LIB_PATH):
    """Load libfehom.so (raises when it has not been built) and declare the signatures."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libfehom.so not found at {path}; build it with "
                           "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = C.CDLL(path)
    vp, i, d, i64p = C.c_void_p, C.c_int, C.c_double, C.POINTER(C.c_int64)
    dp = C.POINTER(C.c_double)
    lib.fehom_default_options.argtypes = [C.POINTER(Options)]
    lib.fehom_default_options.restype = None
    lib.fehom_setup.argtypes = [C.POINTER(vp), i, i, i64p, dp, vp, i, i, dp, dp, C.POINTER(Options)]
    lib.fehom_setup.restype = i
    lib.fehom_precond_build.argtypes = [vp]
    lib.fehom_precond_build.restype = i
    lib.fehom_solve.argtypes = [vp, i, dp, d, vp, vp, i, dp, dp, C.POINTER(SolveInfo)]
    lib.fehom_solve.restype = i
    lib.fehom_destroy.argtypes = [vp]
    lib.fehom_destroy.restype = None
    lib.fehom_last_error.argtypes = [vp]
    lib.fehom_last_error.restype = C.c_char_p
    lib.fehom_query.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(C.c_int), i64p, i64p]
    lib.fehom_query.restype = i
    lib.fehom_apply_stiffness.argtypes = [vp, vp, vp, i]
    lib.fehom_apply_stiffness.restype = i
    lib.fehom_rhs.argtypes = [vp, dp, vp]
    lib.fehom_rhs.restype = i
    lib.fehom_residual_update.argtypes = [vp, vp, vp, vp, dp]
    lib.fehom_residual_update.restype = i
    lib.fehom_stencil_plan.argtypes = [vp, i, C.POINTER(C.c_int), C.POINTER(C.c_int), dp]
    lib.fehom_stencil_plan.restype = i
    lib.fehom_rhs_df.argtypes = [vp, dp, vp]
    lib.fehom_rhs_df.restype = i
    lib.fehom_pcg_apply_stiffness.argtypes = [vp, i, i, vp, vp, dp, i, i, dp, dp]
    lib.fehom_pcg_apply_stiffness.restype = i
    lib.fehom_pcg_precond_step.argtypes = [vp, i, i, vp, vp, vp, vp, dp, dp, dp, dp]
    lib.fehom_pcg_precond_step.restype = i
    lib.fehom_apply_precond.argtypes = [vp, vp, vp, i]
    lib.fehom_apply_precond.restype = i
    lib.fehom_get_symbol_inverse.argtypes = [vp, dp]
    lib.fehom_get_symbol_inverse.restype = i
    lib.fehom_mean_flux.argtypes = [vp, dp, vp, dp]
    lib.fehom_mean_flux.restype = i
    lib.fehom_mean_flux_noalloc.argtypes = [vp, dp, vp, dp]
    lib.fehom_mean_flux_noalloc.restype = i
    lib.fehom_pcg_coefficients.argtypes = [vp, i, i, dp, dp, C.POINTER(C.c_int)]
    lib.fehom_pcg_coefficients.restype = i
    lib.fehom_eig_bounds.argtypes = [vp, dp, i64p, C.POINTER(C.c_int), dp, i64p, C.POINTER(C.c_int)]
    lib.fehom_eig_bounds.restype = i
    lib.fehom_batch_create.argtypes = [C.POINTER(vp), i, C.POINTER(vp)]
    lib.fehom_batch_create.restype = i
    lib.fehom_solve_batch.argtypes = [vp, i, dp, d, dp, dp, C.POINTER(SolveInfo)]
    lib.fehom_solve_batch.restype = i
    lib.fehom_batch_destroy.argtypes = [vp]
    lib.fehom_batch_destroy.restype = None
    lib.fehom_batch_last_error.argtypes = [vp]
    lib.fehom_batch_last_error.restype = C.c_char_p
    lib.fehom_kernel_times.argtypes = [vp, i, dp, i64p]
    lib.fehom_kernel_times.restype = i
    lib.fehom_set_reference.argtypes = [vp, dp]
    lib.fehom_set_reference.restype = i
    lib.fehom_newton_solve.argtypes = [vp, dp, dp, d, d, d, i, vp, i, dp, C.POINTER(NewtonInfo)]
    lib.fehom_newton_solve.restype = i
    lib.fehom_effective_energy.argtypes = [vp, dp]
    lib.fehom_effective_energy.restype = i
    lib.fehom_launch_count.argtypes = [vp, i64p]
    lib.fehom_launch_count.restype = i
    ip = C.POINTER(C.c_int)
    lib.fehom_fft_plan.argtypes = [vp, i, ip, ip, ip, dp, ip]
    lib.fehom_fft_plan.restype = i
    fp = C.POINTER(C.c_float)
    lib.fehom_unet_create.argtypes = [C.POINTER(vp), C.c_int64, i, ip, i, i, i, vp]
    lib.fehom_unet_create.restype = i
    lib.fehom_unet_destroy.argtypes = [vp]
    lib.fehom_unet_destroy.restype = None
    lib.fehom_unet_last_error.argtypes = [vp]
    lib.fehom_unet_last_error.restype = C.c_char_p
    lib.fehom_unet_set_loss.argtypes = [vp, i, d]
    lib.fehom_unet_set_loss.restype = i
    lib.fehom_unet_param_count.argtypes = [vp, i64p]
    lib.fehom_unet_param_count.restype = i
    lib.fehom_unet_set_params.argtypes = [vp, fp]
    lib.fehom_unet_set_params.restype = i
    lib.fehom_unet_get_params.argtypes = [vp, fp]
    lib.fehom_unet_get_params.restype = i
    lib.fehom_unet_predict.argtypes = [vp, i, vp, vp, d, vp]
    lib.fehom_unet_predict.restype = i
    lib.fehom_unet_loss_grad.argtypes = [vp, i, vp, vp, vp, d, dp, fp]
    lib.fehom_unet_loss_grad.restype = i
    lib.fehom_unet_train_step.argtypes = [vp, i, vp, vp, vp, d, d, dp]
    lib.fehom_unet_train_step.restype = i
    lib.fehom_conv3_bf16.argtypes = [i, i, i, i, i, i, vp, vp, vp, i, vp, vp]
    lib.fehom_conv3_bf16.restype = i
    lib.fehom_conv3_wgrad_bf16.argtypes = [i, i, i, i, i, i, vp, vp, vp, vp]
    lib.fehom_conv3_wgrad_bf16.restype = i
    _lib = lib
    return lib


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("fehom needs a CUDA GPU")
    return torch


class Solver:
    """One periodic cell: fehom_setup on construction, fehom_destroy on close()."""

    def __init__(self, elem, physics, n, ids, moduli, ref_material=None, precision="fp64", max_iter=10000,
                 inner_tol=1e-3, cell=None, use_graph=True, stream=None, profile=False, autotune=True,
                 x0_scaling=True, fft_xy=-1, residual_df=True, stencil_rows=0):
        torch = _torch()
        self.lib = load_library()
        self.elem, self.physics = elem, physics
        n = tuple(int(v) for v in n) + (1,) * (3 - len(n))
        self.n = n
        self.N = n[0] * n[1] * n[2]
        opt = Options()
        self.lib.fehom_default_options(C.byref(opt))
        opt.precision = PRECISION[precision]
        opt.max_iter = int(max_iter)
        opt.inner_tol = float(inner_tol)
        opt.use_graph = 1 if use_graph else 0
        opt.profile = 1 if profile else 0
        opt.autotune = 1 if autotune else 0
        opt.x0_scaling = 1 if x0_scaling else 0
        opt.fft_xy = int(fft_xy)
        opt.residual_df = 1 if residual_df else 0
        opt.stencil_rows = int(stencil_rows)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        opt.stream = C.c_void_p(self.stream.cuda_stream)
        self._opt = opt
        moduli = np.ascontiguousarray(np.asarray(moduli, dtype=np.float64))
        nn = (C.c_int64 * 3)(*n)
        cellp = _dptr(np.ascontiguousarray(np.asarray(cell, np.float64))) if cell is not None else None
        refp = None
        if ref_material is not None:
            self._ref = np.ascontiguousarray(np.asarray(ref_material, np.float64))
            refp = _dptr(self._ref)
        if isinstance(ids, np.ndarray):
            ids_h = np.ascontiguousarray(ids.astype(np.uint8).ravel())
            ids_ptr, on_dev = ids_h.ctypes.data, 0
        else:  # torch uint8 tensor on the GPU
            ids_t = ids.contiguous().view(-1)
            ids_ptr, on_dev = ids_t.data_ptr(), 1 if ids_t.is_cuda else 0
            if not ids_t.is_cuda:
                ids_h = ids_t.numpy()
        ctx = C.c_void_p()
        st = self.lib.fehom_setup(C.byref(ctx), ELEM[elem], PHYSICS[physics], nn, cellp, C.c_void_p(ids_ptr), on_dev,
                                  int(moduli.shape[0]), _dptr(moduli), refp, C.byref(opt))
        if st != 0:
            raise FehomError(st, self.lib.fehom_last_error(None).decode())
        self.ctx = ctx
        c, m, Nq, nxh = C.c_int(), C.c_int(), C.c_int64(), C.c_int64()
        self.lib.fehom_query(ctx, C.byref(c), C.byref(m), C.byref(Nq), C.byref(nxh))
        self.c, self.m, self.nxh = c.value, m.value, nxh.value
        self.Nh = self.nxh * n[1] * n[2]

    # -- lifetime -------------------------------------------------------------------------------
    def close(self):
        if getattr(self, "ctx", None):
            self.lib.fehom_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st):
        if st != 0:
            raise FehomError(st, self.lib.fehom_last_error(self.ctx).decode())

    # -- the three calls ------------------------------------------------------------------------
    def precond_build(self):
        self._check(self.lib.fehom_precond_build(self.ctx))

    def solve(self, loads, tol, x0=None, fields="device", raise_on_failure=True):
        """Solve for every row of ``loads``; returns mean fluxes, C_eff, fields and per-load info."""
        torch = _torch()
        loads = np.ascontiguousarray(np.atleast_2d(np.asarray(loads, np.float64)))
        L = loads.shape[0]
        flux = np.zeros((L, self.m))
        ceff = np.full((self.m, self.m), np.nan)
        info = (SolveInfo * L)()
        out = None
        out_ptr, on_dev = None, 1
        if fields == "device":
            out = torch.empty((L, self.c, self.N), dtype=torch.float64, device="cuda")
            out_ptr = C.c_void_p(out.data_ptr())
        elif fields == "host":
            out = torch.empty((L, self.c, self.N), dtype=torch.float64).pin_memory()
            out_ptr, on_dev = C.c_void_p(out.data_ptr()), 0
        x0p = C.c_void_p(x0.data_ptr()) if x0 is not None else None
        st = self.lib.fehom_solve(self.ctx, L, _dptr(loads), float(tol), x0p, out_ptr, on_dev, _dptr(flux), _dptr(ceff),
                                  info)
        if st != 0 and raise_on_failure:
            self._check(st)
        infos = [{k: getattr(info[l], k) for k, _ in SolveInfo._fields_} for l in range(L)]
        return dict(status=st, mean_flux=flux, C_eff=ceff if L == self.m else None, fields=out, info=infos)

    # -- operator-level entry points ------------------------------------------------------------
    def apply_stiffness(self, x, precision="fp64"):
        torch = _torch()
        y = torch.empty_like(x)
        self._check(self.lib.fehom_apply_stiffness(self.ctx, C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr()),
                                                   PRECISION[precision]))
        return y

    def rhs(self, e):
        torch = _torch()
        e = np.ascontiguousarray(np.asarray(e, np.float64))
        b = torch.empty((self.c * self.N,), dtype=torch.float64, device="cuda")
        self._check(self.lib.fehom_rhs(self.ctx, _dptr(e), C.c_void_p(b.data_ptr())))
        return b

    def stencil_plan(self, precision="fp64"):
        """(rows, staging, [ms: 8 / 16 rows with cp.async staging, 8 / 16 rows with TMA staging]) of the hex8
        PCG stiffness apply."""
        rows, staging = C.c_int(0), C.c_int(0)
        ms = np.zeros(4)
        self._check(self.lib.fehom_stencil_plan(self.ctx, PRECISION[precision], C.byref(rows), C.byref(staging),
                                                _dptr(ms)))
        return rows.value, staging.value, ms.tolist()

    def residual_update(self, d, r_in, r_out=None):
        """r_out = r_in - K d with K d in double-float arithmetic (d: FP32 field, r_in / r_out: FP64 fields,
        all on the device); returns (r_out, ||r_out||^2, <sigma> of d alone)."""
        torch = _torch()
        if r_out is None:
            r_out = torch.empty_like(r_in)
        sums = np.zeros(1 + self.m)
        self._check(self.lib.fehom_residual_update(self.ctx, C.c_void_p(d.data_ptr()), C.c_void_p(r_in.data_ptr()),
                                                   C.c_void_p(r_out.data_ptr()), _dptr(sums)))
        return r_out, sums[0], sums[1:]

    def rhs_df(self, e):
        """b = -D^T W C e in double-float arithmetic (the mixed solve's right-hand side)."""
        torch = _torch()
        e = np.ascontiguousarray(np.asarray(e, np.float64))
        b = torch.empty((self.c * self.N,), dtype=torch.float64, device="cuda")
        self._check(self.lib.fehom_rhs_df(self.ctx, _dptr(e), C.c_void_p(b.data_ptr())))
        return b

    def apply_precond(self, r, precision="fp64"):
        torch = _torch()
        z = torch.empty_like(r)
        self._check(self.lib.fehom_apply_precond(self.ctx, C.c_void_p(r.data_ptr()), C.c_void_p(z.data_ptr()),
                                                 PRECISION[precision]))
        return z

    def pcg_apply_stiffness(self, p, rz, precision="fp64", rows=0, staging=0):
        """Stiffness launch of a PCG iteration for a batch of loads: p [L, c, N] (device) -> (ap, <p, K p>,
        alpha = rz / <p, K p>), with the solve's fused kernel (fehom_pcg_apply_stiffness)."""
        torch = _torch()
        L = p.shape[0]
        ap = torch.empty_like(p)
        rz = np.ascontiguousarray(np.broadcast_to(np.asarray(rz, np.float64), (L,)))
        pap, alpha = np.zeros(L), np.zeros(L)
        self._check(self.lib.fehom_pcg_apply_stiffness(self.ctx, PRECISION[precision], L, _ptr(p), _ptr(ap), _dptr(rz),
                                                       int(rows), int(staging), _dptr(pap), _dptr(alpha)))
        return ap, pap, alpha

    def pcg_precond_step(self, r, p, precision="fp64", ap=None, x=None, alpha=None, rz=None):
        """Preconditioner passes of a PCG iteration (fehom_pcg_precond_step), in place on r, x, p
        ([L, c, N] device tensors).  Without alpha: the first apply (p = z).  Returns (rz_new, beta)."""
        L = r.shape[0]
        rz_new, beta = np.zeros(L), np.zeros(L)
        al = rzp = None
        if alpha is not None:
            al = np.ascontiguousarray(np.broadcast_to(np.asarray(alpha, np.float64), (L,)))
            rzp = np.ascontiguousarray(np.broadcast_to(np.asarray(rz, np.float64), (L,)))
        self._check(self.lib.fehom_pcg_precond_step(self.ctx, PRECISION[precision], L, _ptr(r), _ptr(ap), _ptr(x),
                                                    _ptr(p), _dptr(al) if al is not None else None,
                                                    _dptr(rzp) if rzp is not None else None, _dptr(rz_new),
                                                    _dptr(beta)))
        return rz_new, beta

    def symbol_inverse(self):
        ne = 4 if self.elem == "p1tri4_2d" else self.c * (self.c + 1) // 2
        out = np.zeros(ne * self.Nh)
        self._check(self.lib.fehom_get_symbol_inverse(self.ctx, _dptr(out)))
        return out.reshape(ne, self.n[2], self.n[1], self.nxh)

    def kernel_times(self, precision="fp64"):
        """{class: (total ms, launches timed)} of the PCG iteration kernels (needs profile=True)."""
        ms = (C.c_double * 6)()
        cnt = (C.c_int64 * 6)()
        self._check(self.lib.fehom_kernel_times(self.ctx, PRECISION[precision], ms, cnt))
        return {k: (ms[i], cnt[i]) for i, k in enumerate(KERNEL_CLASSES)}

    def fft_plan(self, precision="fp64"):
        """Launch plan of the FFT passes: pairs, tc_y, tc_last, the tuner's times (ms), fused x-y passes."""
        p, y, l, xy = C.c_int(), C.c_int(), C.c_int(), C.c_int()
        ms = (C.c_double * 3)()
        self._check(self.lib.fehom_fft_plan(self.ctx, PRECISION[precision], C.byref(p), C.byref(y), C.byref(l), ms,
                                            C.byref(xy)))
        return {"pairs": p.value, "tc_y": y.value, "tc_last": l.value, "ms": list(ms), "xy_fused": xy.value & 1,
                "last_reg": (xy.value >> 1) & 1}

    def set_reference(self, C_ref):
        """Replace the reference material (then call precond_build)."""
        Cr = np.ascontiguousarray(np.asarray(C_ref, np.float64))
        self._check(self.lib.fehom_set_reference(self.ctx, _dptr(Cr)))

    def newton_solve(self, e, power_n, g0, tol_cg=1e-10, eta=1e-10, max_newton=32, raise_on_failure=True):
        """Algorithm 1 for the power-law conductivity (fehom_newton_solve); returns the mean-zero
        fluctuation (device tensor), the mean flux and the Newton history."""
        torch = _torch()
        e = np.ascontiguousarray(np.asarray(e, np.float64))
        pn = np.ascontiguousarray(np.asarray(power_n, np.float64))
        out = torch.empty((self.N,), dtype=torch.float64, device="cuda")
        flux = np.zeros(3)
        info = NewtonInfo()
        st = self.lib.fehom_newton_solve(self.ctx, _dptr(e), _dptr(pn), float(g0), float(tol_cg), float(eta),
                                         int(max_newton), C.c_void_p(out.data_ptr()), 1, _dptr(flux), C.byref(info))
        if st != 0 and raise_on_failure:
            self._check(st)
        n = info.n_hist
        return dict(status=st, fields=out, mean_flux=flux, newton_iterations=info.newton_iterations,
                    pcg_iterations=info.pcg_iterations, converged=bool(info.converged),
                    residual=list(info.residual[:n]), increment=list(info.increment[:n]),
                    pcg_per_step=list(info.pcg_per_step[:n]))

    def effective_energy(self):
        """Energy (Hill-Mandel) form of C_eff from the last solve with m independent loads."""
        out = np.zeros((self.m, self.m))
        self._check(self.lib.fehom_effective_energy(self.ctx, _dptr(out)))
        return out

    def launch_count(self):
        n = C.c_int64()
        self._check(self.lib.fehom_launch_count(self.ctx, C.byref(n)))
        return n.value

    def pcg_coefficients(self, load=0, capacity=2048):
        """alpha_j, beta_j of the last PCG run of a load (numpy arrays)."""
        a = np.zeros(capacity)
        b = np.zeros(capacity)
        n = C.c_int()
        self._check(self.lib.fehom_pcg_coefficients(self.ctx, int(load), int(capacity), _dptr(a), _dptr(b), C.byref(n)))
        return a[: n.value], b[: n.value]

    def eig_bounds(self):
        """Sorted lower and upper bound sequences of the eigenvalues of K_ref^+ K (length c N each)."""
        P = 256
        lv, hv = np.zeros(P), np.zeros(P)
        lc, hc = np.zeros(P, np.int64), np.zeros(P, np.int64)
        nl, nh = C.c_int(), C.c_int()
        i64 = C.POINTER(C.c_int64)
        self._check(self.lib.fehom_eig_bounds(self.ctx, _dptr(lv), lc.ctypes.data_as(i64), C.byref(nl), _dptr(hv),
                                              hc.ctypes.data_as(i64), C.byref(nh)))
        return (np.repeat(lv[: nl.value], lc[: nl.value]), np.repeat(hv[: nh.value], hc[: nh.value]))

    def mean_flux(self, e, u):
        e = np.ascontiguousarray(np.asarray(e, np.float64))
        out = np.zeros(self.m)
        self._check(self.lib.fehom_mean_flux(self.ctx, _dptr(e), C.c_void_p(u.data_ptr()), _dptr(out)))
        return out


class Batch:
    """Several Solver cells solved together (fehom_solve_batch): one CUDA graph, one branch per cell."""

    def __init__(self, solvers):
        self.lib = load_library()
        self.solvers = list(solvers)
        arr = (C.c_void_p * len(self.solvers))(*[sv.ctx.value for sv in self.solvers])
        b = C.c_void_p()
        st = self.lib.fehom_batch_create(C.byref(b), len(self.solvers), arr)
        if st != 0:
            raise FehomError(st, self.lib.fehom_batch_last_error(None).decode())
        self.b = b

    def solve(self, loads, tol, raise_on_failure=True):
        loads = np.ascontiguousarray(np.atleast_2d(np.asarray(loads, np.float64)))
        L, nc = loads.shape[0], len(self.solvers)
        m = self.solvers[0].m
        flux = np.zeros((nc, L, m))
        ceff = np.full((nc, m, m), np.nan)
        info = (SolveInfo * (nc * L))()
        st = self.lib.fehom_solve_batch(self.b, L, _dptr(loads), float(tol), _dptr(flux), _dptr(ceff), info)
        if st != 0 and raise_on_failure:
            raise FehomError(st, self.lib.fehom_batch_last_error(self.b).decode())
        infos = [[{k: getattr(info[c * L + l], k) for k, _ in SolveInfo._fields_} for l in range(L)] for c in range(nc)]
        return dict(status=st, mean_flux=flux, C_eff=ceff if L == m else None, info=infos)

    def close(self):
        if getattr(self, "b", None):
            self.lib.fehom_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


class UNet:
    """The warm-start network of include/fehom_unet.h (fehom_unet_create on construction)."""

    def __init__(self, n, widths=(16, 32, 64, 128), n_phases=2, n_out=3, max_batch=8, stream=None):
        torch = _torch()
        self.lib = load_library()
        self.n, self.widths, self.n_out, self.n_phases = int(n), tuple(int(w) for w in widths), int(n_out), int(n_phases)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        w = (C.c_int * len(self.widths))(*self.widths)
        net = C.c_void_p()
        st = self.lib.fehom_unet_create(C.byref(net), self.n, len(self.widths), w, self.n_phases, self.n_out,
                                        int(max_batch), C.c_void_p(self.stream.cuda_stream))
        if st != 0:
            raise FehomError(st, self.lib.fehom_unet_last_error(None).decode())
        self.net = net
        cnt = C.c_int64()
        self.lib.fehom_unet_param_count(net, C.byref(cnt))
        self.n_params = cnt.value

    def _check(self, st):
        if st != 0:
            raise FehomError(st, self.lib.fehom_unet_last_error(self.net).decode())

    def close(self):
        if getattr(self, "net", None):
            self.lib.fehom_unet_destroy(self.net)
            self.net = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_loss(self, kind="mse", l2_weight=0.0):
        self._check(self.lib.fehom_unet_set_loss(self.net, {"mse": 0, "h1": 1}[kind], float(l2_weight)))

    def set_params(self, theta):
        t = np.ascontiguousarray(np.asarray(theta, np.float32))
        assert t.size == self.n_params
        self._check(self.lib.fehom_unet_set_params(self.net, t.ctypes.data_as(C.POINTER(C.c_float))))

    def get_params(self):
        t = np.zeros(self.n_params, np.float32)
        self._check(self.lib.fehom_unet_get_params(self.net, t.ctypes.data_as(C.POINTER(C.c_float))))
        return t

    def predict(self, ids, features, out_scale, out=None):
        """ids: uint8 [B, N] (device), features: float32 [B, n_phases] (device) -> x0 float64 [B, n_out, N]."""
        torch = _torch()
        B = ids.shape[0]
        if out is None:
            out = torch.empty((B, self.n_out, self.n ** 3), dtype=torch.float64, device=ids.device)
        self._check(self.lib.fehom_unet_predict(self.net, B, _ptr(ids), _ptr(features), float(out_scale), _ptr(out)))
        return out

    def loss_grad(self, ids, features, target, out_scale):
        g = np.zeros(self.n_params, np.float32)
        loss = C.c_double()
        self._check(self.lib.fehom_unet_loss_grad(self.net, ids.shape[0], _ptr(ids), _ptr(features), _ptr(target),
                                                  float(out_scale), C.byref(loss), g.ctypes.data_as(C.POINTER(C.c_float))))
        return loss.value, g

    def train_step(self, ids, features, target, out_scale, lr, want_loss=False):
        loss = C.c_double()
        self._check(self.lib.fehom_unet_train_step(self.net, ids.shape[0], _ptr(ids), _ptr(features), _ptr(target),
                                                   float(out_scale), float(lr), C.byref(loss) if want_loss else None))
        return loss.value if want_loss else None


def conv3_bf16(x, w, bias=None, relu=False):
    """Tensor-core periodic 3x3x3 convolution (fehom_conv3_bf16): x bf16 [B, D, H, W, Cin],
    w bf16 [27, Cout, Cin] -> float32 [B, D, H, W, Cout]."""
    torch = _torch()
    lib = load_library()
    B, D, H, W, Cin = x.shape
    Cout = w.shape[1]
    y = torch.empty((B, D, H, W, Cout), dtype=torch.float32, device=x.device)
    st = lib.fehom_conv3_bf16(B, D, H, W, Cin, Cout, _ptr(x), _ptr(w), _ptr(bias), 1 if relu else 0, _ptr(y),
                              C.c_void_p(torch.cuda.current_stream().cuda_stream))
    if st != 0:
        raise FehomError(st, "fehom_conv3_bf16")
    return y


def conv3_wgrad_bf16(x, dy):
    """Weight gradient of the periodic 3x3x3 convolution (fehom_conv3_wgrad_bf16) -> float32 [27, Cout, Cin]."""
    torch = _torch()
    lib = load_library()
    B, D, H, W, Cin = x.shape
    Cout = dy.shape[-1]
    dw = torch.empty((27, Cout, Cin), dtype=torch.float32, device=x.device)
    st = lib.fehom_conv3_wgrad_bf16(B, D, H, W, Cin, Cout, _ptr(x), _ptr(dy), _ptr(dw),
                                    C.c_void_p(torch.cuda.current_stream().cuda_stream))
    if st != 0:
        raise FehomError(st, "fehom_conv3_wgrad_bf16")
    return dw
