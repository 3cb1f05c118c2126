"""Python binding of libosmodi.so (argument marshalling only).

Every function here forwards to the C entry point of the same name in
``include/osmodi.h``; all computation happens in the library's CUDA kernels.
Tensors are passed as raw device pointers.  The library must have been built
(``paper_2311_16935_gb300.build.build()``); importing this module without it
raises, there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libosmodi.so")

OK, NOT_CONVERGED = 0, 1
E_INVALID, E_UNSUPPORTED, E_NOMEM, E_CUDA, E_DIVERGED, E_TIMEOUT, E_EMPTY, E_NAN_INPUT, E_WORKSPACE = (
    -1, -2, -3, -4, -5, -6, -7, -8, -9)
F32, F64 = 0, 1
FP64, FP32, FP32_REFINE = 0, 1, 2
FPCG, OUTER = 0, 1
DEBUG_BARRIER_SPINS, DEBUG_SKIP_BARRIER_BLOCK, DEBUG_CORRECTION_SCALE, DEBUG_MG_UNFUSED, DEBUG_NET_WMMA = 1, 2, 3, 4, 5
DEBUG_BATCH_BOTTOM_CELLS = 6
DEBUG_CG_FIXED_GRAPH = 7
DEBUG_DEFAULT = -0x7fffffffffffffff
INNER_CG, INNER_JACOBI = 0, 1


class osmodi_options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("scheme", ctypes.c_int), ("inner", ctypes.c_int),
                ("inner_max", ctypes.c_int), ("inner_tol", ctypes.c_double), ("check_every", ctypes.c_int),
                ("sweeps_per_pass", ctypes.c_int), ("max_refine", ctypes.c_int), ("record_history", ctypes.c_int),
                ("threads", ctypes.c_int), ("blocks_per_sm", ctypes.c_int), ("profile", ctypes.c_int),
                ("slab", ctypes.c_int), ("flat_sweeps", ctypes.c_int), ("autotune", ctypes.c_int),
                ("accel", ctypes.c_int), ("precond", ctypes.c_int), ("zero_start", ctypes.c_int),
                ("mg_sweeps", ctypes.c_int), ("mg_scale", ctypes.c_double), ("refine_ff", ctypes.c_int)]


class osmodi_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("outer_iters", ctypes.c_int), ("inner_iters", ctypes.c_int64),
                ("refine_steps", ctypes.c_int), ("eps_R", ctypes.c_double), ("eps_P", ctypes.c_double),
                ("ms", ctypes.c_double), ("point_updates", ctypes.c_double), ("seed_rel_dist", ctypes.c_double),
                ("kernel_launches", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class OsmodiError(RuntimeError):
    def __init__(self, status, what=""):
        self.status = status
        msg = f"{what}: {status_string(status)} ({status})"
        if status == E_CUDA:
            msg += f" [{last_cuda_error()}]"
        super().__init__(msg)


_lib = None

_SIGS = {
    "osmodi_default_options": (None, [ctypes.c_void_p]),
    "osmodi_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.c_void_p, ctypes.c_void_p]),
    "osmodi_workspace_bytes": (ctypes.c_size_t, [ctypes.c_void_p]),
    "osmodi_solve": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int,
                                    ctypes.c_double, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "osmodi_solve_batched": (ctypes.c_int, [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                            ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                            ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "osmodi_batched_workspace_bytes": (ctypes.c_size_t, [ctypes.c_int, ctypes.c_void_p]),
    "osmodi_solve_many": (ctypes.c_int, [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                         ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_void_p, ctypes.c_void_p]),
    "osmodi_source_incompressible": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                                    ctypes.c_void_p, ctypes.c_double, ctypes.c_double,
                                                    ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p]),
    "osmodi_source_rans": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double,
                                          ctypes.c_void_p, ctypes.c_void_p]),
    "osmodi_source_compressible": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                                  ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                                  ctypes.c_double, ctypes.c_double, ctypes.c_void_p,
                                                  ctypes.c_void_p, ctypes.c_void_p]),
    "osmodi_batch_graph_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                                 ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                                 ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "osmodi_batch_graph_launch": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "osmodi_batch_graph_results": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "osmodi_batch_graph_destroy": (None, [ctypes.c_void_p]),
    "osmodi_solve_noalloc": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                            ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_void_p,
                                            ctypes.c_void_p]),
    "osmodi_history": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    "osmodi_history_pressure": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    "osmodi_debug_set": (ctypes.c_longlong, [ctypes.c_int, ctypes.c_longlong]),
    "osmodi_probe_fp64": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "osmodi_probe_convert": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                            ctypes.c_int64, ctypes.c_void_p]),
    "osmodi_net_status": (ctypes.c_int, [ctypes.c_void_p]),
    "osmodi_conv3d": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                     ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                     ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p]),
    "osmodi_tc_gemm": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                      ctypes.c_void_p, ctypes.c_void_p]),
    "osmodi_ray_counts": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "osmodi_source": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]),
    "osmodi_apply": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "osmodi_residual": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int,
                                       ctypes.c_void_p, ctypes.c_void_p]),
    "osmodi_plan_info": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "osmodi_precond_levels": (ctypes.c_int, [ctypes.c_void_p]),
    "osmodi_kernel_stats": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "osmodi_kernel_stats_precond": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "osmodi_plan_constants": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "osmodi_destroy": (None, [ctypes.c_void_p]),
    "osmodi_autotune": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_char_p,
                                       ctypes.c_void_p]),
    "osmodi_autotune_batched": (ctypes.c_int, [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                               ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                               ctypes.c_void_p]),
    "osmodi_net_param_count": (ctypes.c_size_t, []),
    "osmodi_net_create": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]),
    "osmodi_net_set_params": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "osmodi_net_get_params": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "osmodi_net_get_grads": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "osmodi_net_get_output": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "osmodi_net_forward": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                          ctypes.c_double, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]),
    "osmodi_net_backward": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                           ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "osmodi_net_adam": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                       ctypes.c_double, ctypes.c_int, ctypes.c_void_p]),
    "osmodi_net_destroy": (None, [ctypes.c_void_p]),
    "osmodi_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "osmodi_last_cuda_error": (ctypes.c_char_p, []),
}


def lib():
    """Load libosmodi.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with paper_2311_16935_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def exported_symbols():
    return list(_SIGS)


def status_string(st: int) -> str:
    return lib().osmodi_status_string(int(st)).decode()


def last_cuda_error() -> str:
    return lib().osmodi_last_cuda_error().decode()


def _dtype_code(t: torch.Tensor) -> int:
    if t.dtype == torch.float32:
        return F32
    if t.dtype == torch.float64:
        return F64
    raise TypeError(f"unsupported dtype {t.dtype}")


def _stream_ptr(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


def _check_cuda(t: torch.Tensor, name: str):
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous CUDA tensor")


def _check_solve_buffer(t: torch.Tensor, name: str):
    """A contiguous CUDA tensor, or a contiguous page-locked host tensor (the
    kernels then read / write it over the host link; osmodi_solve checks the
    pointer as well)."""
    if not t.is_contiguous() or not (t.is_cuda or (t.device.type == "cpu" and t.is_pinned())):
        raise ValueError(f"{name} must be a contiguous CUDA tensor or a pinned host tensor")


def default_options(**overrides) -> osmodi_options:
    o = osmodi_options()
    lib().osmodi_default_options(ctypes.byref(o))
    names = {f[0] for f in osmodi_options._fields_}
    for k, v in overrides.items():
        if k not in names:
            raise TypeError(f"unknown option {k!r}")
        setattr(o, k, v)
    return o


class Plan:
    """Owns an osmodi_plan and a workspace tensor (device memory from torch)."""

    def __init__(self, ndim, dims, spacing, mask=None, options=None, stream=None, **opt):
        if options is None:
            options = default_options(**opt)
        self.ndim = ndim
        self.dims = tuple(int(d) for d in dims) + (1,) * (3 - len(dims))
        d = (ctypes.c_int64 * 3)(*self.dims)
        sp = (ctypes.c_double * 3)(*(list(spacing) + [1.0] * (3 - len(spacing))))
        mptr = None
        if mask is not None:
            _check_cuda(mask, "mask")
            if mask.dtype != torch.uint8:
                raise TypeError("mask must be uint8")
            mptr = mask.data_ptr()
        h = ctypes.c_void_p()
        st = lib().osmodi_create(ndim, d, sp, mptr, ctypes.byref(options), _stream_ptr(stream), ctypes.byref(h))
        if st != OK:
            raise OsmodiError(st, "osmodi_create")
        self.handle = h
        self.options = options
        self._ws = None

    def workspace_bytes(self) -> int:
        return int(lib().osmodi_workspace_bytes(self.handle))

    def workspace(self) -> torch.Tensor:
        n = self.workspace_bytes()
        if self._ws is None or self._ws.numel() < n:
            self._ws = torch.empty(n + 256, dtype=torch.uint8, device="cuda")
        return self._ws

    def _ws_ptr(self):
        ws = self.workspace()
        p = ws.data_ptr()
        return (p + 255) // 256 * 256

    def info(self):
        out = (ctypes.c_int64 * 8)()
        st = lib().osmodi_plan_info(self.handle, out)
        if st != OK:
            raise OsmodiError(st, "osmodi_plan_info")
        keys = ["nx", "ny", "nz", "n_valid", "n_comp", "px", "n_box", "blocks"]
        d = dict(zip(keys, list(out)))
        d["mg_levels"] = int(lib().osmodi_precond_levels(self.handle))
        return d

    def constants(self):
        c = (ctypes.c_double * 9)()
        F = (ctypes.c_double * 3)()
        a = ctypes.c_double()
        st = lib().osmodi_plan_constants(self.handle, c, F, ctypes.byref(a))
        if st != OK:
            raise OsmodiError(st, "osmodi_plan_constants")
        return list(c), list(F), a.value

    def solve(self, grad: torch.Tensor, p: torch.Tensor, tol: float, max_iter: int = 1 << 30, stream=None,
              check=True) -> osmodi_result:
        """osmodi_solve: p holds P^0 on entry and the pressure on return.
        grad and p may be CUDA tensors or pinned host tensors."""
        _check_solve_buffer(grad, "grad")
        _check_solve_buffer(p, "p")
        res = osmodi_result()
        st = lib().osmodi_solve(self.handle, grad.data_ptr(), _dtype_code(grad), p.data_ptr(), _dtype_code(p),
                                float(tol), int(min(max_iter, 2**31 - 1)), self._ws_ptr(), _stream_ptr(stream),
                                ctypes.byref(res))
        if check and st < 0:
            raise OsmodiError(st, "osmodi_solve")
        return res

    def kernel_stats(self):
        out = (ctypes.c_double * 8)()
        st = lib().osmodi_kernel_stats(self.handle, out)
        if st != OK:
            raise OsmodiError(st, "osmodi_kernel_stats")
        v = list(out)
        return {"cg_apply_ms": v[0], "cg_apply_launches": int(v[1]), "cg_update_ms": v[2],
                "cg_update_launches": int(v[3]), "residual64_ms": v[4], "residual64_launches": int(v[5]),
                "precond_ms": v[6], "precond_applications": int(v[7])}

    def kernel_stats_precond(self):
        out = (ctypes.c_double * 4)()
        st = lib().osmodi_kernel_stats_precond(self.handle, out)
        if st != OK:
            raise OsmodiError(st, "osmodi_kernel_stats_precond")
        v = list(out)
        return {"mg_sweep_ms": v[0], "mg_sweep_launches": int(v[1]), "mg_resid_ms": v[2],
                "mg_resid_launches": int(v[3])}

    def solve_noalloc(self, grad: torch.Tensor, p: torch.Tensor, tol: float, max_iter: int = 1 << 30, stream=None,
                      check=True) -> osmodi_result:
        """osmodi_solve_noalloc: as solve(), with the library's fixed device
        scratch instead of a workspace (nothing is allocated)."""
        _check_cuda(grad, "grad")
        _check_cuda(p, "p")
        res = osmodi_result()
        st = lib().osmodi_solve_noalloc(self.handle, grad.data_ptr(), _dtype_code(grad), p.data_ptr(), _dtype_code(p),
                                        float(tol), int(min(max_iter, 2**31 - 1)), _stream_ptr(stream),
                                        ctypes.byref(res))
        if check and st < 0:
            raise OsmodiError(st, "osmodi_solve_noalloc")
        return res

    def autotune(self, cache_path=None, stream=None):
        """osmodi_autotune; returns the best time per CG iteration (ms)."""
        ms = ctypes.c_double(0.0)
        st = lib().osmodi_autotune(self.handle, self._ws_ptr(), _stream_ptr(stream),
                                   None if cache_path is None else str(cache_path).encode(), ctypes.byref(ms))
        if st != OK:
            raise OsmodiError(st, "osmodi_autotune")
        return ms.value

    def history(self):
        n = lib().osmodi_history(self.handle, None, 0)
        buf = (ctypes.c_double * max(n, 1))()
        lib().osmodi_history(self.handle, buf, n)
        return list(buf)[:n]

    def history_pressure(self):
        n = lib().osmodi_history_pressure(self.handle, None, 0)
        buf = (ctypes.c_double * max(n, 1))()
        lib().osmodi_history_pressure(self.handle, buf, n)
        return list(buf)[:n]

    def ray_counts(self, stream=None) -> torch.Tensor:
        nx, ny, nz = self.dims
        out = torch.empty((nx * ny * nz, 2 + 4 * self.ndim), dtype=torch.float64, device="cuda")
        st = lib().osmodi_ray_counts(self.handle, out.data_ptr(), _stream_ptr(stream))
        if st != OK:
            raise OsmodiError(st, "osmodi_ray_counts")
        return out

    def source(self, grad: torch.Tensor, stream=None) -> torch.Tensor:
        _check_cuda(grad, "grad")
        out = torch.empty(grad.shape[1:], dtype=torch.float64, device="cuda")
        st = lib().osmodi_source(self.handle, grad.data_ptr(), _dtype_code(grad), out.data_ptr(), _stream_ptr(stream))
        if st != OK:
            raise OsmodiError(st, "osmodi_source")
        return out

    def apply(self, which: int, x: torch.Tensor, stream=None) -> torch.Tensor:
        _check_cuda(x, "x")
        if x.dtype != torch.float64:
            raise TypeError("x must be float64")
        y = torch.empty_like(x)
        st = lib().osmodi_apply(self.handle, int(which), x.data_ptr(), y.data_ptr(), _stream_ptr(stream))
        if st != OK:
            raise OsmodiError(st, "osmodi_apply")
        return y

    def residual(self, grad: torch.Tensor, p: torch.Tensor, stream=None) -> float:
        _check_cuda(grad, "grad")
        _check_cuda(p, "p")
        eps = ctypes.c_double()
        st = lib().osmodi_residual(self.handle, grad.data_ptr(), _dtype_code(grad), p.data_ptr(), _dtype_code(p),
                                   ctypes.byref(eps), _stream_ptr(stream))
        if st != OK:
            raise OsmodiError(st, "osmodi_residual")
        return eps.value

    # ---- source-term front ends (FP32 velocity data -> FP32 gradient) ----
    def _vec(self, t, name, planes):
        _check_cuda(t, name)
        if t.dtype != torch.float32 or not t.is_contiguous():
            raise TypeError(f"{name} must be contiguous float32")
        if t.numel() != planes * self.dims[0] * self.dims[1] * self.dims[2]:
            raise ValueError(f"{name} must hold {planes} planes of the plan's grid")
        return t.data_ptr()

    def _grad_out(self, like):
        return torch.empty((self.ndim,) + tuple(like.shape[1:]), dtype=torch.float32, device="cuda")

    def source_incompressible(self, u, u_prev=None, u_next=None, dt=1.0, rho=1.0, mu=0.0, stream=None):
        """osmodi_source_incompressible: f of Eq. 1 from the snapshot u (and
        its neighbours in time, either may be None)."""
        pu = self._vec(u, "u", self.ndim)
        pp = self._vec(u_prev, "u_prev", self.ndim) if u_prev is not None else None
        pn = self._vec(u_next, "u_next", self.ndim) if u_next is not None else None
        out = self._grad_out(u)
        st = lib().osmodi_source_incompressible(self.handle, pu, pp, pn, float(dt), float(rho), float(mu),
                                                out.data_ptr(), _stream_ptr(stream))
        if st != OK:
            raise OsmodiError(st, "osmodi_source_incompressible")
        return out

    def source_rans(self, u_mean, stress, rho=1.0, stream=None):
        """osmodi_source_rans: f of Eq. RANS_f."""
        nst = 3 if self.ndim == 2 else 6
        pu = self._vec(u_mean, "u_mean", self.ndim)
        ps = self._vec(stress, "stress", nst)
        out = self._grad_out(u_mean)
        st = lib().osmodi_source_rans(self.handle, pu, ps, float(rho), out.data_ptr(), _stream_ptr(stream))
        if st != OK:
            raise OsmodiError(st, "osmodi_source_rans")
        return out

    def source_compressible(self, u_mean, stress, gamma, mach_inf, v_inf, t_inf, r_gas, stream=None):
        """osmodi_source_compressible: (grad ln(P/P_inf), T) of Eq.
        compressible-pressure."""
        nst = 3 if self.ndim == 2 else 6
        pu = self._vec(u_mean, "u_mean", self.ndim)
        ps = self._vec(stress, "stress", nst)
        out = self._grad_out(u_mean)
        temp = torch.empty(tuple(u_mean.shape[1:]), dtype=torch.float32, device="cuda")
        st = lib().osmodi_source_compressible(self.handle, pu, ps, float(gamma), float(mach_inf), float(v_inf),
                                              float(t_inf), float(r_gas), out.data_ptr(), temp.data_ptr(),
                                              _stream_ptr(stream))
        if st != OK:
            raise OsmodiError(st, "osmodi_source_compressible")
        return out, temp

    def close(self):
        if getattr(self, "handle", None):
            lib().osmodi_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Workspace holder for osmodi_solve_batched over a fixed list of plans."""

    def __init__(self, plans):
        self.plans = list(plans)
        self._arr = (ctypes.c_void_p * len(self.plans))(*[p.handle.value for p in self.plans])
        n = int(lib().osmodi_batched_workspace_bytes(len(self.plans), self._arr))
        if n == 0:
            raise OsmodiError(E_INVALID, "osmodi_batched_workspace_bytes")
        self.ws = torch.empty(n + 256, dtype=torch.uint8, device="cuda")

    def solve(self, grads, ps, tol, max_iter=1 << 30, stream=None, check=True):
        """osmodi_solve_batched; returns (status, [osmodi_result])"""
        count = len(self.plans)
        if len(grads) != count or len(ps) != count:
            raise ValueError("one gradient and one pressure tensor per plan")
        for g, p in zip(grads, ps):
            _check_cuda(g, "grad")
            _check_cuda(p, "p")
        gdt = {_dtype_code(g) for g in grads}
        pdt = {_dtype_code(p) for p in ps}
        if len(gdt) != 1 or len(pdt) != 1:
            raise TypeError("all gradients (and all pressures) must share one dtype")
        ga = (ctypes.c_void_p * count)(*[g.data_ptr() for g in grads])
        pa = (ctypes.c_void_p * count)(*[p.data_ptr() for p in ps])
        res = (osmodi_result * count)()
        ws = (self.ws.data_ptr() + 255) // 256 * 256
        st = lib().osmodi_solve_batched(count, self._arr, ga, gdt.pop(), pa, pdt.pop(), float(tol),
                                        int(min(max_iter, 2**31 - 1)), ws, _stream_ptr(stream), res)
        if check and st < 0 and st != E_NAN_INPUT:
            raise OsmodiError(st, "osmodi_solve_batched")
        return st, list(res)


    def capture(self, grads, ps, tol, max_iter=1 << 30, stream=None):
        """osmodi_batch_graph_create: one solve of this batch captured as a
        CUDA graph bound to these tensors (keep them alive, refill them in
        place between launches)."""
        return BatchGraph(self, grads, ps, tol, max_iter, stream)

    def autotune(self, grads, ps, stream=None):
        """osmodi_autotune_batched; returns the chosen tile depth."""
        count = len(self.plans)
        ga = (ctypes.c_void_p * count)(*[g.data_ptr() for g in grads])
        pa = (ctypes.c_void_p * count)(*[p.data_ptr() for p in ps])
        depth = ctypes.c_int(0)
        ws = (self.ws.data_ptr() + 255) // 256 * 256
        st = lib().osmodi_autotune_batched(count, self._arr, ga, _dtype_code(grads[0]), pa, _dtype_code(ps[0]), ws,
                                           _stream_ptr(stream), ctypes.byref(depth))
        if st != OK:
            raise OsmodiError(st, "osmodi_autotune_batched")
        return depth.value


class BatchGraph:
    """A captured batched solve (osmodi_batch_graph_*)."""

    def __init__(self, batch, grads, ps, tol, max_iter=1 << 30, stream=None):
        count = len(batch.plans)
        if len(grads) != count or len(ps) != count:
            raise ValueError("one gradient and one pressure tensor per plan")
        for g, p in zip(grads, ps):
            _check_cuda(g, "grad")
            _check_cuda(p, "p")
        gdt = {_dtype_code(g) for g in grads}
        pdt = {_dtype_code(p) for p in ps}
        if len(gdt) != 1 or len(pdt) != 1:
            raise TypeError("all gradients (and all pressures) must share one dtype")
        self.batch, self.grads, self.ps = batch, list(grads), list(ps)  # the graph holds their addresses
        ga = (ctypes.c_void_p * count)(*[g.data_ptr() for g in grads])
        pa = (ctypes.c_void_p * count)(*[p.data_ptr() for p in ps])
        ws = (batch.ws.data_ptr() + 255) // 256 * 256
        h = ctypes.c_void_p()
        st = lib().osmodi_batch_graph_create(count, batch._arr, ga, gdt.pop(), pa, pdt.pop(), float(tol),
                                             int(min(max_iter, 2**31 - 1)), ws, _stream_ptr(stream), ctypes.byref(h))
        if st != OK:
            raise OsmodiError(st, "osmodi_batch_graph_create")
        self.handle = h

    def launch(self, stream=None):
        st = lib().osmodi_batch_graph_launch(self.handle, _stream_ptr(stream))
        if st != OK:
            raise OsmodiError(st, "osmodi_batch_graph_launch")

    def results(self, check=True):
        """Waits for the last launch; returns (status, [osmodi_result])."""
        res = (osmodi_result * len(self.grads))()
        st = lib().osmodi_batch_graph_results(self.handle, res)
        if check and st < 0 and st != E_NAN_INPUT:
            raise OsmodiError(st, "osmodi_batch_graph_results")
        return st, list(res)

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            lib().osmodi_batch_graph_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Many:
    """osmodi_solve_many over a fixed list of plans: one workspace per stream."""

    def __init__(self, plans, streams=8):
        self.plans = list(plans)
        self.streams = max(1, min(int(streams), len(self.plans), 64))
        self._arr = (ctypes.c_void_p * len(self.plans))(*[p.handle.value for p in self.plans])
        self.ws = []
        for w in range(self.streams):
            need = max(p.workspace_bytes() for p in self.plans[w::self.streams])
            self.ws.append(torch.empty(need + 256, dtype=torch.uint8, device="cuda"))
        self._ws_arr = (ctypes.c_void_p * self.streams)(*[(t.data_ptr() + 255) // 256 * 256 for t in self.ws])

    def solve(self, grads, ps, tol, max_iter=1 << 30, check=True):
        """Returns (status, [osmodi_result]); synchronous."""
        count = len(self.plans)
        if len(grads) != count or len(ps) != count:
            raise ValueError("one gradient and one pressure tensor per plan")
        for g, p in zip(grads, ps):
            _check_cuda(g, "grad")
            _check_cuda(p, "p")
        gdt = {_dtype_code(g) for g in grads}
        pdt = {_dtype_code(p) for p in ps}
        if len(gdt) != 1 or len(pdt) != 1:
            raise TypeError("all gradients (and all pressures) must share one dtype")
        ga = (ctypes.c_void_p * count)(*[g.data_ptr() for g in grads])
        pa = (ctypes.c_void_p * count)(*[p.data_ptr() for p in ps])
        res = (osmodi_result * count)()
        torch.cuda.current_stream().synchronize()  # inputs written on torch's stream are complete
        st = lib().osmodi_solve_many(count, self._arr, ga, gdt.pop(), pa, pdt.pop(), float(tol),
                                     int(min(max_iter, 2**31 - 1)), self.streams, self._ws_arr, res)
        if check and st < 0 and st != E_NAN_INPUT:
            raise OsmodiError(st, "osmodi_solve_many")
        return st, list(res)


def osmodi_solve_batched(plans, grads, ps, tol, max_iter=1 << 30, stream=None):
    return Batch(plans).solve(grads, ps, tol, max_iter, stream)


class Net:
    """The seed network (osmodi_net_*): parameters live on the device."""

    def __init__(self, dims, train=False):
        d = (ctypes.c_int64 * 3)(*[int(v) for v in dims])
        h = ctypes.c_void_p()
        st = lib().osmodi_net_create(d, 1 if train else 0, ctypes.byref(h))
        if st != OK:
            raise OsmodiError(st, "osmodi_net_create")
        self.handle = h
        self.dims = tuple(int(v) for v in dims)
        self.train = train

    @staticmethod
    def param_count() -> int:
        return int(lib().osmodi_net_param_count())

    def set_params(self, params):
        import numpy as np

        a = np.ascontiguousarray(np.asarray(params, dtype=np.float32))
        if a.size != self.param_count():
            raise ValueError("wrong parameter count")
        st = lib().osmodi_net_set_params(self.handle, a.ctypes.data)
        if st != OK:
            raise OsmodiError(st, "osmodi_net_set_params")

    def get_params(self):
        import numpy as np

        a = np.empty(self.param_count(), dtype=np.float32)
        st = lib().osmodi_net_get_params(self.handle, a.ctypes.data)
        if st != OK:
            raise OsmodiError(st, "osmodi_net_get_params")
        return a

    def get_grads(self):
        import numpy as np

        a = np.empty(self.param_count(), dtype=np.float32)
        st = lib().osmodi_net_get_grads(self.handle, a.ctypes.data)
        if st != OK:
            raise OsmodiError(st, "osmodi_net_get_grads")
        return a

    def get_output(self):
        import numpy as np

        nx, ny, nz = self.dims
        a = np.empty(nx * ny * nz, dtype=np.float32)
        st = lib().osmodi_net_get_output(self.handle, a.ctypes.data)
        if st != OK:
            raise OsmodiError(st, "osmodi_net_get_output")
        return a.reshape(nz, ny, nx)

    def forward(self, grad, mask, spacing, p, stream=None):
        _check_cuda(grad, "grad")
        _check_cuda(p, "p")
        mptr = None if mask is None else mask.data_ptr()
        st = lib().osmodi_net_forward(self.handle, grad.data_ptr(), _dtype_code(grad), mptr, float(spacing),
                                      p.data_ptr(), _dtype_code(p), _stream_ptr(stream))
        if st != OK:
            raise OsmodiError(st, "osmodi_net_forward")

    def backward(self, grad, mask, spacing, target, want_loss=True, stream=None):
        _check_cuda(grad, "grad")
        _check_cuda(target, "target")
        if target.dtype != torch.float64:
            raise TypeError("target must be float64")
        mptr = None if mask is None else mask.data_ptr()
        loss = ctypes.c_double(0.0)
        st = lib().osmodi_net_backward(self.handle, grad.data_ptr(), _dtype_code(grad), mptr, float(spacing),
                                       target.data_ptr(), ctypes.byref(loss) if want_loss else None,
                                       _stream_ptr(stream))
        if st != OK:
            raise OsmodiError(st, "osmodi_net_backward")
        return loss.value

    def adam(self, lr, beta1=0.9, beta2=0.999, eps=1e-8, batch=1, stream=None):
        st = lib().osmodi_net_adam(self.handle, float(lr), float(beta1), float(beta2), float(eps), int(batch),
                                   _stream_ptr(stream))
        if st != OK:
            raise OsmodiError(st, "osmodi_net_adam")

    def close(self):
        if getattr(self, "handle", None):
            lib().osmodi_net_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def osmodi_create(ndim, dims, spacing, mask=None, **opt) -> Plan:
    return Plan(ndim, dims, spacing, mask, **opt)


def osmodi_solve(plan: Plan, grad, p, tol, max_iter=1 << 30, stream=None) -> osmodi_result:
    return plan.solve(grad, p, tol, max_iter, stream)


def osmodi_destroy(plan: Plan):
    plan.close()


def debug_set(knob: int, value: int) -> int:
    """osmodi_debug_set: set a test knob, return its previous value."""
    return int(lib().osmodi_debug_set(int(knob), int(value)))


def probe_fp64(stream=None):
    """osmodi_probe_fp64: the device's measured FP64 FMA throughput (GFLOP/s)."""
    g, ms = ctypes.c_double(0.0), ctypes.c_double(0.0)
    st = lib().osmodi_probe_fp64(ctypes.byref(g), ctypes.byref(ms), _stream_ptr(stream))
    if st != OK:
        raise OsmodiError(st, "osmodi_probe_fp64")
    return g.value


def probe_convert(d_in: torch.Tensor, f_in: torch.Tensor, stream=None):
    """osmodi_probe_convert: (d_in rounded to FP32, f_in widened to FP64) by
    the library's integer-unit conversions; 1-D CUDA tensors of one length."""
    _check_cuda(d_in, "d_in")
    _check_cuda(f_in, "f_in")
    if d_in.dtype != torch.float64 or f_in.dtype != torch.float32 or d_in.dim() != 1 or f_in.shape != d_in.shape:
        raise TypeError("d_in: 1-D float64, f_in: float32 of the same length")
    f_out = torch.empty_like(f_in)
    d_out = torch.empty_like(d_in)
    st = lib().osmodi_probe_convert(d_in.data_ptr(), f_out.data_ptr(), f_in.data_ptr(), d_out.data_ptr(), d_in.numel(),
                                    _stream_ptr(stream))
    if st != OK:
        raise OsmodiError(st, "osmodi_probe_convert")
    return f_out, d_out


def tc_gemm(A: torch.Tensor, B: torch.Tensor, stream=None):
    """osmodi_tc_gemm: D = A B^T (A 128 x K, B N x K, BF16 CUDA tensors) on
    the tensor cores; returns (D FP32, error flag)."""
    _check_cuda(A, "A")
    _check_cuda(B, "B")
    if A.dtype != torch.bfloat16 or B.dtype != torch.bfloat16 or A.shape[0] != 128 or A.shape[1] != B.shape[1]:
        raise TypeError("A: 128 x K bf16, B: N x K bf16")
    D = torch.empty((128, B.shape[0]), dtype=torch.float32, device=A.device)
    err = torch.zeros(1, dtype=torch.int32, device=A.device)
    st = lib().osmodi_tc_gemm(A.data_ptr(), B.data_ptr(), D.data_ptr(), int(B.shape[0]), int(A.shape[1]),
                              err.data_ptr(), _stream_ptr(stream))
    if st != OK:
        raise OsmodiError(st, "osmodi_tc_gemm")
    return D, int(err.item())


def conv3d(x: torch.Tensor, w: torch.Tensor, bias=None, relu=False, path=0, stream=None):
    """osmodi_conv3d: x (D, H, W, cin) bf16, w (27, cin, cout) bf16, bias
    (cout,) float32 or None; returns (y (D, H, W, cout) bf16, error flag)."""
    _check_cuda(x, "x")
    _check_cuda(w, "w")
    D, H, W, cin = x.shape
    cout = w.shape[2]
    y = torch.empty((D, H, W, cout), dtype=torch.bfloat16, device=x.device)
    scratch = torch.empty(2 * (27 * cin + 64) * ((cout + 15) // 16 * 16) + 4096, dtype=torch.uint8, device=x.device)
    err = torch.zeros(1, dtype=torch.int32, device=x.device)
    st = lib().osmodi_conv3d(x.data_ptr(), w.data_ptr(), None if bias is None else bias.data_ptr(), y.data_ptr(),
                             D, H, W, cin, cout, 1 if relu else 0, int(path), scratch.data_ptr(), scratch.numel(),
                             err.data_ptr(), _stream_ptr(stream))
    if st != OK:
        raise OsmodiError(st, "osmodi_conv3d")
    return y, int(err.item())
