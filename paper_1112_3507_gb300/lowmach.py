"""Thin Python binding of the C ABI in include/lowmach.h (ctypes).

Argument marshalling only: every computation runs in liblowmach.so's CUDA
kernels.  Fields are passed either as numpy float64 arrays (host memory,
on_device = 0) or as contiguous CUDA torch tensors (device memory,
on_device = 1); torch supplies device memory and the current stream.

The library must have been built (paper_1112_3507_gb300.build); loading
fails loudly otherwise -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from .build import LIB

# status codes and enums (mirror include/lowmach.h)
LM_OK = 0
LM_ERR_INVALID_ARG = -1
LM_ERR_NOT_POSITIVE = -2
LM_ERR_NO_CONVERGENCE = -3
LM_ERR_BREAKDOWN = -4
LM_ERR_TIMEOUT = -5
LM_ERR_CUDA = -6
LM_ERR_NETWORK = -7
LM_ERR_OUT_OF_MEMORY = -8
LM_ERR_STATE = -9
BC_PERIODIC, BC_NEUMANN = 0, 1
FP64_JACOBI_PCG, FP64_MG_PCG, MIXED_MG_IR, MIXED_LEARNED_FCG_IR = 0, 1, 2, 3
PREC_FP64, PREC_FP32 = 0, 1
MODES = {"jacobi": FP64_JACOBI_PCG, "fp64-mg": FP64_MG_PCG, "mixed": MIXED_MG_IR,
         "learned": MIXED_LEARNED_FCG_IR}


class SolveOpts(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int), ("rtol", ctypes.c_double), ("max_iter", ctypes.c_int),
                ("use_x0", ctypes.c_int), ("max_outer", ctypes.c_int), ("nu1", ctypes.c_int),
                ("nu2", ctypes.c_int), ("inner_rtol", ctypes.c_double), ("inner_max_iter", ctypes.c_int),
                ("check_every", ctypes.c_int), ("net_precond", ctypes.c_int),
                ("cuda_stream", ctypes.c_void_p)]


class SolveResult(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("iters", ctypes.c_int), ("outer_iters", ctypes.c_int),
                ("vcycles", ctypes.c_int), ("rel_residual", ctypes.c_double), ("seconds", ctypes.c_double)]


class LowMachError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {status_string(code)} ({code})")


_lib = None
_P = ctypes.c_void_p
_I64_3 = ctypes.c_int64 * 3
_D3 = ctypes.c_double * 3
_I3 = ctypes.c_int * 3
_I4 = ctypes.c_int * 4

_SIGNATURES = {
    "lm_default_opts": (None, [ctypes.POINTER(SolveOpts)]),
    "lm_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "lm_kernel_launches": (ctypes.c_int64, []),
    "lm_grid_create": (ctypes.c_int, [ctypes.c_int, _I64_3, _D3, _I3, ctypes.POINTER(_P)]),
    "lm_grid_destroy": (None, [_P]),
    "lm_grid_size": (ctypes.c_int64, [_P]),
    "lm_set_coefficients": (ctypes.c_int, [_P, _P, _P, _P, ctypes.c_double, ctypes.c_int, _P]),
    "lm_set_coefficients_raw": (ctypes.c_int, [_P, _P, _P, ctypes.c_int, _P]),
    "lm_set_rhs": (ctypes.c_int, [_P, _P, ctypes.c_int, _P]),
    "lm_set_initial_guess": (ctypes.c_int, [_P, _P, ctypes.c_int, _P]),
    "lm_load_network": (ctypes.c_int, [_P, ctypes.c_char_p]),
    "lm_solve": (ctypes.c_int, [_P, ctypes.POINTER(SolveOpts), ctypes.POINTER(SolveResult)]),
    "lm_get_solution": (ctypes.c_int, [_P, _P, ctypes.c_int, _P]),
    "lm_get_residual_history": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_double), ctypes.c_int,
                                               ctypes.POINTER(ctypes.c_int)]),
    "lm_get_coefficients": (ctypes.c_int, [_P, _P, _P, _P, _P, _P]),
    "lm_apply": (ctypes.c_int, [_P, ctypes.c_int, _P, _P, ctypes.POINTER(ctypes.c_double), _P]),
    "lm_mg_vcycle": (ctypes.c_int, [_P, _P, _P, ctypes.c_int, ctypes.c_int, _P]),
    "lm_mg_sweep": (ctypes.c_int, [_P, _P, _P, _P, ctypes.c_int, _P]),
    "lm_mg_level_shape": (ctypes.c_int, [_P, ctypes.c_int, _I64_3, ctypes.POINTER(ctypes.c_int)]),
    "lm_net_create": (ctypes.c_int, [_I4, ctypes.POINTER(_P)]),
    "lm_net_destroy": (None, [_P]),
    "lm_net_num_params": (ctypes.c_int, [_P]),
    "lm_net_set_params": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_float), ctypes.c_int]),
    "lm_net_get_params": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_float), ctypes.c_int]),
    "lm_net_get_grads": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_float), ctypes.c_int]),
    "lm_net_forward": (ctypes.c_int, [_P, _P, _P, ctypes.c_int, ctypes.c_int, ctypes.c_int, _P]),
    "lm_net_backward": (ctypes.c_int, [_P, _P, _P]),
    "lm_net_mse": (ctypes.c_int, [_P, _P, _P, _P, ctypes.c_longlong, ctypes.POINTER(ctypes.c_double), _P]),
    "lm_net_adam": (ctypes.c_int, [_P, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float, _P]),
    "lm_net_save": (ctypes.c_int, [_P, ctypes.c_char_p]),
    "lm_net_load": (ctypes.c_int, [ctypes.c_char_p, ctypes.POINTER(_P)]),
    "lm_net_features": (ctypes.c_int, [_P, _P, _P, ctypes.POINTER(ctypes.c_double), _P]),
    "lm_batch_solve": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int, ctypes.POINTER(SolveOpts),
                                       ctypes.POINTER(SolveResult)]),
    "lm_autotune_set_cache": (ctypes.c_int, [ctypes.c_char_p]),
    "lm_batch_set_coefficients": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int, ctypes.POINTER(_P),
                                                  ctypes.POINTER(_P), ctypes.POINTER(_P),
                                                  ctypes.POINTER(ctypes.c_double), _P]),
    "lm_halo_pack": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int,
                                     _P, ctypes.c_int, _P]),
    "lm_vec_axpby": (ctypes.c_int, [ctypes.c_int64, ctypes.c_double, _P, ctypes.c_int, ctypes.c_double, _P,
                                     ctypes.c_int, _P, ctypes.c_int, _P]),
    "lm_vec_dot": (ctypes.c_int, [ctypes.c_int64, _P, ctypes.c_int, _P, ctypes.c_int, _P,
                                   ctypes.POINTER(ctypes.c_double), _P]),
    "lm_vec_mul": (ctypes.c_int, [ctypes.c_int64, _P, _P, _P, _P]),
    "lm_jacobi_inverse_diagonal": (ctypes.c_int, [_P, _P, _P]),
    "lm_mg_restrict_residual": (ctypes.c_int, [_P, _P, _P, _P, _P]),
    "lm_mg_prolong_add": (ctypes.c_int, [_P, _P, _P, _P]),
    "lm_mg_level_coefficients": (ctypes.c_int, [_P, ctypes.c_int, _P, _P, ctypes.POINTER(ctypes.c_double), _P]),
    "lm_projection_rhs": (ctypes.c_int, [ctypes.c_int, _I64_3, _D3, _I3, ctypes.c_double] + [_P] * 10),
    "lm_projection_update": (ctypes.c_int, [ctypes.c_int, _I64_3, _D3, _I3, ctypes.c_double] + [_P] * 9),
    "lm_advect": (ctypes.c_int, [ctypes.c_int, _I64_3, _D3, _I3, ctypes.c_double] + [_P] * 9),
    "lm_eos_ideal": (ctypes.c_int, [ctypes.c_int64, ctypes.c_double, _P, _P, _P, _P, _P, _P]),
    "lm_diffusion4": (ctypes.c_int, [ctypes.c_int, _I64_3, _D3, _I3, ctypes.c_int, ctypes.c_double, _P,
                                      ctypes.c_double, _P, _P]),
    "lm_probe_rate": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double), _P]),
    "lm_fe_create": (ctypes.c_int, [ctypes.c_int, _I64_3, _D3, _I3, ctypes.POINTER(_P)]),
    "lm_fe_destroy": (None, [_P]),
    "lm_fe_set_coefficients": (ctypes.c_int, [_P, _P, _P, ctypes.c_int, _P]),
    "lm_fe_set_state": (ctypes.c_int, [_P, _P, _P, _P, ctypes.c_double, ctypes.c_int, _P]),
    "lm_fe_lumped_mass": (ctypes.c_int, [_P, _P, ctypes.c_int, _P]),
    "lm_fe_mass_times": (ctypes.c_int, [_P, _P, _P, ctypes.c_int, _P]),
    "lm_fe_apply": (ctypes.c_int, [_P, ctypes.c_int, _P, _P, ctypes.POINTER(ctypes.c_double), _P]),
    "lm_fe_solve": (ctypes.c_int, [_P, _P, _P, ctypes.c_int, ctypes.POINTER(SolveOpts),
                                    ctypes.POINTER(SolveResult)]),
    "lm_apply_dot_noalloc": (ctypes.c_int, [ctypes.c_int, _I64_3, _I3, _P, _P, _P, _P, _P, _P, _P, _P]),
}


def declared_symbols():
    return list(_SIGNATURES)


def lib():
    """Load liblowmach.so (once).  Raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB):
            raise RuntimeError(f"{LIB} not found: build it with `python -m paper_1112_3507_gb300.build` "
                               "(there is no CPU fallback)")
        L = ctypes.CDLL(LIB)
        for name, (res, args) in _SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def kernel_launches() -> int:
    return int(lib().lm_kernel_launches())


def status_string(code: int) -> str:
    try:
        return lib().lm_status_string(code).decode()
    except RuntimeError:
        return f"status {code}"


def _check(code: int, where: str, ok=(LM_OK,)):
    if code not in ok:
        raise LowMachError(code, where)
    return code


def _stream_ptr(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        except ImportError:
            pass
        return ctypes.c_void_p(0)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _field(a, N: int, dtype=np.float64):
    """(pointer, on_device, keepalive) for a host numpy array or a CUDA tensor."""
    try:
        import torch
        if isinstance(a, torch.Tensor):
            if not a.is_cuda:
                a = a.detach().numpy()
            else:
                want = torch.float64 if dtype == np.float64 else torch.float32
                if a.dtype != want or not a.is_contiguous() or a.numel() != N:
                    raise ValueError(f"device field must be a contiguous {want} tensor of {N} values")
                return ctypes.c_void_p(a.data_ptr()), 1, a
    except ImportError:
        pass
    arr = np.ascontiguousarray(np.asarray(a, dtype=dtype)).ravel()
    if arr.size != N:
        raise ValueError(f"field has {arr.size} values, grid has {N}")
    return ctypes.c_void_p(arr.ctypes.data), 0, arr


class Grid:
    """A solver grid: n = (nx, ny, nz) cells (ny = 1 for 2D), spacings h,
    one boundary condition per axis (BC_PERIODIC / BC_NEUMANN)."""

    def __init__(self, n, h, bc, ndim: int | None = None):
        n = tuple(int(v) for v in n)
        if ndim is None:
            ndim = 2 if n[1] == 1 else 3
        self.n, self.h, self.bc, self.ndim = n, tuple(float(v) for v in h), tuple(int(b) for b in bc), ndim
        self.N = n[0] * n[1] * n[2]
        ptr = _P()
        _check(lib().lm_grid_create(ndim, _I64_3(*n), _D3(*self.h), _I3(*self.bc), ctypes.byref(ptr)),
               "lm_grid_create")
        self._g = ptr

    @classmethod
    def for_problem(cls, p):
        return cls(p.n, p.h, p.bc, p.ndim)

    def close(self):
        if getattr(self, "_g", None):
            lib().lm_grid_destroy(self._g)
            self._g = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # ---- inputs
    def set_coefficients(self, rho_old, rho_new, cs2, dt, stream=None):
        a, d1, k1 = _field(rho_old, self.N)
        b, d2, k2 = _field(rho_new, self.N)
        c, d3, k3 = _field(cs2, self.N)
        if not d1 == d2 == d3:
            raise ValueError("all fields must live on the same side (host or device)")
        return _check(lib().lm_set_coefficients(self._g, a, b, c, float(dt), d1, _stream_ptr(stream)),
                      "lm_set_coefficients")

    def set_coefficients_raw(self, ctilde, rho_face_src, stream=None):
        a, d1, k1 = _field(ctilde, self.N)
        b, d2, k2 = _field(rho_face_src, self.N)
        if d1 != d2:
            raise ValueError("all fields must live on the same side (host or device)")
        return _check(lib().lm_set_coefficients_raw(self._g, a, b, d1, _stream_ptr(stream)),
                      "lm_set_coefficients_raw")

    def set_problem(self, p, stream=None):
        self.set_coefficients(p.rho_old, p.rho_new, p.cs2, p.dt, stream)
        self.set_rhs(p.f, stream)

    def set_rhs(self, f, stream=None):
        a, d, k = _field(f, self.N)
        return _check(lib().lm_set_rhs(self._g, a, d, _stream_ptr(stream)), "lm_set_rhs")

    def set_initial_guess(self, x0, stream=None):
        a, d, k = _field(x0, self.N)
        return _check(lib().lm_set_initial_guess(self._g, a, d, _stream_ptr(stream)), "lm_set_initial_guess")

    # ---- solve
    def solve(self, mode="mixed", rtol=1e-8, stream=None, allow=(LM_OK,), **kw) -> dict:
        o = SolveOpts()
        lib().lm_default_opts(ctypes.byref(o))
        o.mode = MODES[mode] if isinstance(mode, str) else int(mode)
        o.rtol = float(rtol)
        for k, v in kw.items():
            if not hasattr(o, k):
                raise TypeError(f"unknown solve option {k}")
            setattr(o, k, v)
        o.cuda_stream = _stream_ptr(stream)
        r = SolveResult()
        code = lib().lm_solve(self._g, ctypes.byref(o), ctypes.byref(r))
        _check(code, "lm_solve", ok=allow)
        return dict(status=r.status, iters=r.iters, outer_iters=r.outer_iters, vcycles=r.vcycles,
                    rel_residual=r.rel_residual, seconds=r.seconds)

    def solution(self, out=None, stream=None):
        if out is None:
            out = np.empty(self.N, dtype=np.float64)
        a, d, k = _field(out, self.N)
        _check(lib().lm_get_solution(self._g, a, d, _stream_ptr(stream)), "lm_get_solution")
        return out

    def residual_history(self):
        n = ctypes.c_int(0)
        lib().lm_get_residual_history(self._g, None, 0, ctypes.byref(n))
        buf = (ctypes.c_double * max(n.value, 1))()
        _check(lib().lm_get_residual_history(self._g, buf, n.value, ctypes.byref(n)), "lm_get_residual_history")
        return np.array(buf[: n.value])

    # ---- row-level entry points (device tensors)
    def coefficients(self, stream=None):
        import torch
        outs = [torch.empty(self.N, dtype=torch.float64, device="cuda") for _ in range(4)]
        _check(lib().lm_get_coefficients(self._g, *[ctypes.c_void_p(t.data_ptr()) for t in outs],
                                         _stream_ptr(stream)), "lm_get_coefficients")
        return outs

    def apply(self, x, y, prec=PREC_FP64, with_dot=False, stream=None):
        dt = np.float64 if prec == PREC_FP64 else np.float32
        xp, dx, kx = _field(x, self.N, dt)
        yp, dy, ky = _field(y, self.N, dt)
        if not (dx and dy):
            raise ValueError("lm_apply takes device tensors")
        dot = ctypes.c_double(0.0)
        _check(lib().lm_apply(self._g, prec, xp, yp, ctypes.byref(dot) if with_dot else None,
                              _stream_ptr(stream)), "lm_apply")
        return dot.value if with_dot else None

    def mg_vcycle(self, r, z, nu1=1, nu2=1, stream=None):
        rp, dr, kr = _field(r, self.N, np.float32)
        zp, dz, kz = _field(z, self.N, np.float32)
        if not (dr and dz):
            raise ValueError("lm_mg_vcycle takes device tensors")
        _check(lib().lm_mg_vcycle(self._g, rp, zp, nu1, nu2, _stream_ptr(stream)), "lm_mg_vcycle")

    def mg_sweep(self, x_in, f, x_out, order=0, stream=None):
        """One float32 red-black (order 0) or black-red (1) sweep on the finest level; x_in None = 0."""
        fp, df, kf = _field(f, self.N, np.float32)
        op, do, ko = _field(x_out, self.N, np.float32)
        xp, dx = None, 1
        if x_in is not None:
            xp, dx, kx = _field(x_in, self.N, np.float32)
        if not (df and do and dx):
            raise ValueError("lm_mg_sweep takes device tensors")
        _check(lib().lm_mg_sweep(self._g, xp, fp, op, int(order), _stream_ptr(stream)), "lm_mg_sweep")

    def load_network(self, path):
        return _check(lib().lm_load_network(self._g, str(path).encode()), "lm_load_network")

    def features(self, v, feat, stream=None):
        """Network input of this (2D) grid from device float64 v into device float32 feat (N*3)."""
        vp, dv, kv = _field(v, self.N)
        fp, df, kf = _field(feat, 3 * self.N, np.float32)
        if not (dv and df):
            raise ValueError("lm_net_features takes device tensors")
        sc = ctypes.c_double(0.0)
        _check(lib().lm_net_features(self._g, vp, fp, ctypes.byref(sc), _stream_ptr(stream)), "lm_net_features")
        return sc.value

    def mg_levels(self):
        shapes = []
        nl = ctypes.c_int(0)
        out = _I64_3()
        _check(lib().lm_mg_level_shape(self._g, 0, out, ctypes.byref(nl)), "lm_mg_level_shape")
        for l in range(nl.value):
            _check(lib().lm_mg_level_shape(self._g, l, out, ctypes.byref(nl)), "lm_mg_level_shape")
            shapes.append(tuple(out))
        return shapes


class FEGrid:
    """The operator in Q1 finite elements on n = (nx, ny, nz) points (ny = 1
    for 2D), spacings h, one boundary condition per axis (lm_fe_*)."""

    def __init__(self, n, h, bc, ndim: int | None = None):
        n = tuple(int(v) for v in n)
        if ndim is None:
            ndim = 2 if n[1] == 1 else 3
        self.n, self.h, self.bc, self.ndim = n, tuple(float(v) for v in h), tuple(int(b) for b in bc), ndim
        self.N = n[0] * n[1] * n[2]
        ptr = _P()
        _check(lib().lm_fe_create(ndim, _I64_3(*n), _D3(*self.h), _I3(*self.bc), ctypes.byref(ptr)), "lm_fe_create")
        self._h = ptr

    def close(self):
        if getattr(self, "_h", None):
            lib().lm_fe_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_coefficients(self, ctilde, rho, stream=None):
        a, d1, k1 = _field(ctilde, self.N)
        b, d2, k2 = _field(rho, self.N)
        if d1 != d2:
            raise ValueError("all fields must live on the same side (host or device)")
        return _check(lib().lm_fe_set_coefficients(self._h, a, b, d1, _stream_ptr(stream)), "lm_fe_set_coefficients")

    def set_state(self, rho_old, rho_new, cs2, dt, stream=None):
        a, d1, k1 = _field(rho_old, self.N)
        b, d2, k2 = _field(rho_new, self.N)
        c, d3, k3 = _field(cs2, self.N)
        if not d1 == d2 == d3:
            raise ValueError("all fields must live on the same side (host or device)")
        return _check(lib().lm_fe_set_state(self._h, a, b, c, float(dt), d1, _stream_ptr(stream)), "lm_fe_set_state")

    def mass_times(self, f, out, stream=None):
        a, d1, k1 = _field(f, self.N)
        b, d2, k2 = _field(out, self.N)
        if d1 != d2:
            raise ValueError("f and out must live on the same side (host or device)")
        _check(lib().lm_fe_mass_times(self._h, a, b, d1, _stream_ptr(stream)), "lm_fe_mass_times")
        return out

    def lumped_mass(self, out=None, stream=None):
        if out is None:
            out = np.empty(self.N, dtype=np.float64)
        a, d, k = _field(out, self.N)
        _check(lib().lm_fe_lumped_mass(self._h, a, d, _stream_ptr(stream)), "lm_fe_lumped_mass")
        return out

    def apply(self, x, y, prec=PREC_FP64, with_dot=False, stream=None):
        dt = np.float64 if prec == PREC_FP64 else np.float32
        xp, dx, kx = _field(x, self.N, dt)
        yp, dy, ky = _field(y, self.N, dt)
        if not (dx and dy):
            raise ValueError("lm_fe_apply takes device tensors")
        dot = ctypes.c_double(0.0)
        _check(lib().lm_fe_apply(self._h, prec, xp, yp, ctypes.byref(dot) if with_dot else None,
                                 _stream_ptr(stream)), "lm_fe_apply")
        return dot.value if with_dot else None

    def solve(self, b, x, mode="mixed", rtol=1e-8, stream=None, allow=(LM_OK,), **kw) -> dict:
        """lm_fe_solve: B x = b; x (same side as b) is overwritten with the solution."""
        o = SolveOpts()
        lib().lm_default_opts(ctypes.byref(o))
        o.mode = MODES[mode] if isinstance(mode, str) else int(mode)
        o.rtol = float(rtol)
        for k, v in kw.items():
            if not hasattr(o, k):
                raise TypeError(f"unknown solve option {k}")
            setattr(o, k, v)
        o.cuda_stream = _stream_ptr(stream)
        bp, db, kb = _field(b, self.N)
        if isinstance(x, np.ndarray) and (x.dtype != np.float64 or not x.flags.c_contiguous):
            raise ValueError("x must be a contiguous float64 array")
        xp, dx, kx = _field(x, self.N)
        if db != dx:
            raise ValueError("b and x must live on the same side (host or device)")
        r = SolveResult()
        code = lib().lm_fe_solve(self._h, bp, xp, db, ctypes.byref(o), ctypes.byref(r))
        _check(code, "lm_fe_solve", ok=allow)
        return dict(status=r.status, iters=r.iters, outer_iters=r.outer_iters, vcycles=r.vcycles,
                    rel_residual=r.rel_residual, seconds=r.seconds)


class Net:
    """The learned U-Net (lm_net_*): forward/backward/Adam on device float32 tensors."""

    def __init__(self, ch=(16, 32, 48, 64), _handle=None):
        if _handle is not None:
            self._n = _handle
        else:
            h = _P()
            _check(lib().lm_net_create(_I4(*ch), ctypes.byref(h)), "lm_net_create")
            self._n = h
        self.nparams = lib().lm_net_num_params(self._n)

    @classmethod
    def load(cls, path):
        h = _P()
        _check(lib().lm_net_load(str(path).encode(), ctypes.byref(h)), "lm_net_load")
        return cls(_handle=h)

    def close(self):
        if getattr(self, "_n", None):
            lib().lm_net_destroy(self._n)
            self._n = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, p):
        a = np.ascontiguousarray(p, dtype=np.float32)
        _check(lib().lm_net_set_params(self._n, a.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), a.size),
               "lm_net_set_params")

    def params(self):
        a = np.empty(self.nparams, dtype=np.float32)
        _check(lib().lm_net_get_params(self._n, a.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), a.size),
               "lm_net_get_params")
        return a

    def grads(self):
        a = np.empty(self.nparams, dtype=np.float32)
        _check(lib().lm_net_get_grads(self._n, a.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), a.size),
               "lm_net_get_grads")
        return a

    def forward(self, x, y, B, H, W, stream=None):
        _check(lib().lm_net_forward(self._n, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()), B, H, W,
                                    _stream_ptr(stream)), "lm_net_forward")

    def backward(self, gy, stream=None):
        _check(lib().lm_net_backward(self._n, ctypes.c_void_p(gy.data_ptr()), _stream_ptr(stream)), "lm_net_backward")

    def mse(self, y, t, gy, want_loss=True, stream=None):
        loss = ctypes.c_double(0.0)
        _check(lib().lm_net_mse(self._n, ctypes.c_void_p(y.data_ptr()), ctypes.c_void_p(t.data_ptr()),
                                ctypes.c_void_p(gy.data_ptr()), y.numel(), ctypes.byref(loss) if want_loss else None,
                                _stream_ptr(stream)), "lm_net_mse")
        return loss.value

    def adam(self, lr, b1=0.9, b2=0.999, eps=1e-8, stream=None):
        _check(lib().lm_net_adam(self._n, lr, b1, b2, eps, _stream_ptr(stream)), "lm_net_adam")

    def save(self, path):
        _check(lib().lm_net_save(self._n, str(path).encode()), "lm_net_save")


def autotune_set_cache(path=None):
    return _check(lib().lm_autotune_set_cache(path.encode() if path else None), "lm_autotune_set_cache")


def batch_set_coefficients(grids, rho_old, rho_new, cs2, dts, stream=None):
    """lm_batch_set_coefficients: lists (one entry per grid) of CUDA float64 tensors and host dt values."""
    n = len(grids)
    ptrs = []
    for arrs in (rho_old, rho_new, cs2):
        row = []
        for g, t in zip(grids, arrs):
            p, on_dev, keep = _field(t, g.N)
            if not on_dev:
                raise ValueError("lm_batch_set_coefficients takes device tensors")
            row.append(p.value)
        ptrs.append((_P * n)(*row))
    handles = (_P * n)(*[g._g for g in grids])
    dt = (ctypes.c_double * n)(*[float(v) for v in dts])
    return _check(lib().lm_batch_set_coefficients(handles, n, ptrs[0], ptrs[1], ptrs[2], dt, _stream_ptr(stream)),
                  "lm_batch_set_coefficients")


def batch_solve(grids, rtol=1e-8, stream=None, allow=(LM_OK,), **kw):
    """lm_batch_solve over a list of Grid objects; returns one result dict per grid."""
    o = SolveOpts()
    lib().lm_default_opts(ctypes.byref(o))
    o.mode = MIXED_MG_IR
    o.rtol = float(rtol)
    o.inner_rtol = 1e-3
    for k, v in kw.items():
        if not hasattr(o, k):
            raise TypeError(f"unknown solve option {k}")
        setattr(o, k, v)
    o.cuda_stream = _stream_ptr(stream)
    n = len(grids)
    handles = (_P * n)(*[g._g for g in grids])
    res = (SolveResult * n)()
    code = lib().lm_batch_solve(handles, n, ctypes.byref(o), res)
    _check(code, "lm_batch_solve", ok=allow)
    return [dict(status=r.status, iters=r.iters, outer_iters=r.outer_iters, vcycles=r.vcycles,
                 rel_residual=r.rel_residual, seconds=r.seconds) for r in res]


def apply_dot_noalloc(ndim, n, bc, ctilde, gx, gy, gz, x, y, dot_out, stream=None):
    """y = A x and dot_out[0] = x^T A x through lm_apply_dot_noalloc: all
    arguments are CUDA float64 tensors except n, bc; nothing is allocated."""
    n = tuple(int(v) for v in n)
    N = n[0] * n[1] * n[2]
    ptrs = []
    for t, size in ((ctilde, N), (gx, N), (gy, N), (gz, N), (x, N), (y, N), (dot_out, 1)):
        ptr, on_dev, keep = _field(t, size)
        if not on_dev:
            raise ValueError("lm_apply_dot_noalloc takes device tensors")
        ptrs.append(ptr)
    return _check(lib().lm_apply_dot_noalloc(int(ndim), _I64_3(*n), _I3(*bc), *ptrs, _stream_ptr(stream)),
                  "lm_apply_dot_noalloc")


def probe_rate(which: int, steps: int = 20000, stream=None) -> float:
    """lm_probe_rate: measured operations per second of the current device
    (0 = float64 FMA, 1 = float32 FMA, 2 = float64 <-> float32 conversions)."""
    out = ctypes.c_double(0.0)
    _check(lib().lm_probe_rate(int(which), int(steps), ctypes.byref(out), _stream_ptr(stream)), "lm_probe_rate")
    return out.value


def advect(n, h, bc, dt, rho, mom, e, rho_new, mom_star, e_star, rho_c=None, rho_c_new=None, stream=None):
    """lm_advect (steps (i)-(iii)): device float64 tensors; mom and mom_star
    hold the three components consecutively (3N values)."""
    n = tuple(int(v) for v in n)
    ndim = 2 if n[1] == 1 else 3
    N = n[0] * n[1] * n[2]
    names = ("rho", "mom", "e", "rho_c", "rho_new", "mom_star", "e_star", "rho_c_new")
    sizes = (N, 3 * N, N, N, N, 3 * N, N, N)
    ts = (rho, mom, e, rho_c, rho_new, mom_star, e_star, rho_c_new)
    ptrs = [_dev_ptr(t, sz, nm) for t, sz, nm in zip(ts, sizes, names)]
    return _check(lib().lm_advect(ndim, _I64_3(*n), _D3(*h), _I3(*bc), float(dt), *ptrs, _stream_ptr(stream)),
                  "lm_advect")


def eos_ideal(gamma, rho, mom, e, p, cs2=None, stream=None):
    """lm_eos_ideal (step (ix)): device float64 tensors, mom 3N values."""
    N = int(rho.numel())
    return _check(lib().lm_eos_ideal(N, float(gamma), _dev_ptr(rho, N, "rho"), _dev_ptr(mom, 3 * N, "mom"),
                                      _dev_ptr(e, N, "e"), _dev_ptr(p, N, "p"), _dev_ptr(cs2, N, "cs2"),
                                      _stream_ptr(stream)), "lm_eos_ideal")


def diffusion4(u, out, n, h, bc, alpha=1.0, beta=0.0, stream=None):
    """lm_diffusion4: out = beta u + alpha (sum over axes of the dissipative
    fourth-order second derivative); u, out CUDA tensors (float64 or float32)."""
    n = tuple(int(v) for v in n)
    N = n[0] * n[1] * n[2]
    import torch
    prec = PREC_FP64 if u.dtype == torch.float64 else PREC_FP32
    dt = np.float64 if prec == PREC_FP64 else np.float32
    up, du, ku = _field(u, N, dt)
    op, do, ko = _field(out, N, dt)
    if not (du and do):
        raise ValueError("lm_diffusion4 takes device tensors")
    ndim = 2 if n[1] == 1 else 3
    return _check(lib().lm_diffusion4(ndim, _I64_3(*n), _D3(*h), _I3(*bc), prec, float(alpha), up, float(beta), op,
                                      _stream_ptr(stream)), "lm_diffusion4")


def _dev_ptr(t, size, name):
    if t is None:
        return None
    p, on_dev, keep = _field(t, size)
    if not on_dev:
        raise ValueError(f"{name}: device tensors only")
    return p


def projection_rhs(n, h, bc, dt, p_old, rho_old, cs2_old, mom_old, mom_star, rho_new, f, uface_star, source=None,
                   stream=None):
    """lm_projection_rhs on CUDA float64 tensors (momenta and faces: 3N values)."""
    n = tuple(int(v) for v in n)
    N = n[0] * n[1] * n[2]
    args = [_dev_ptr(t, s_, "lm_projection_rhs") for t, s_ in
            ((p_old, N), (rho_old, N), (cs2_old, N), (mom_old, 3 * N), (mom_star, 3 * N), (rho_new, N), (source, N),
             (f, N), (uface_star, 3 * N))]
    ndim = 2 if n[1] == 1 else 3
    return _check(lib().lm_projection_rhs(ndim, _I64_3(*n), _D3(*h), _I3(*bc), float(dt), *args, _stream_ptr(stream)),
                  "lm_projection_rhs")


def projection_update(n, h, bc, dt, p_pred, rho_new, mom_star, uface_star, e_star, mom_new, uface_new, e_new,
                      stream=None):
    """lm_projection_update on CUDA float64 tensors (momenta and faces: 3N values)."""
    n = tuple(int(v) for v in n)
    N = n[0] * n[1] * n[2]
    args = [_dev_ptr(t, s_, "lm_projection_update") for t, s_ in
            ((p_pred, N), (rho_new, N), (mom_star, 3 * N), (uface_star, 3 * N), (e_star, N), (mom_new, 3 * N),
             (uface_new, 3 * N), (e_new, N))]
    ndim = 2 if n[1] == 1 else 3
    return _check(lib().lm_projection_update(ndim, _I64_3(*n), _D3(*h), _I3(*bc), float(dt), *args,
                                             _stream_ptr(stream)), "lm_projection_update")
