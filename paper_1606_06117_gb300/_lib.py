"""Thin ctypes binding of libsl (include/sl.h).

Argument marshalling only: every step of the advection runs in the CUDA
kernels of libsl.  Functions named ``sl_*`` mirror the C entry points one to
one; they accept torch tensors (or raw integer addresses) for pointers and
raise :class:`SLError` with the library's message on a non-zero status.

There is no fallback: if ``libsl.so`` has not been built (``build()`` in
``paper_1606_06117_gb300.build``) the first call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

from . import build as _build

CIR, FEC, BEC, CEC = 0, 1, 2, 3
SCHEMES = {"CIR": CIR, "FEC": FEC, "BEC": BEC, "CEC": CEC}
F32, F64, F32_D64 = 0, 1, 2
DTYPES = {"f32": F32, "f64": F64, "f32_d64": F32_D64}
DEV_CFL, DEV_TIMEOUT = 1, 2
STATUS = {0: "SL_OK", -1: "SL_ERR_ARG", -2: "SL_ERR_ALIAS", -3: "SL_ERR_CFL", -4: "SL_ERR_CUDA",
          -5: "SL_ERR_TIMEOUT", -6: "SL_ERR_UNSUPPORTED", -7: "SL_ERR_NOMEM"}

#: every symbol include/sl.h declares
EXPORTS = ("sl_version", "sl_last_error", "sl_init", "sl_advect", "sl_advect_multi", "sl_advect_host",
           "sl_release_host_staging", "sl_courant_max", "sl_norms", "sl_device_status", "sl_batch_create",
           "sl_batch_step", "sl_batch_destroy", "sl_autotune", "sl_norms_static",
           "sl_corrector_param_count", "sl_corrector_create", "sl_corrector_destroy", "sl_corrector_get_params",
           "sl_corrector_set_params", "sl_corrector_add_samples", "sl_corrector_get_rows", "sl_corrector_train",
           "sl_corrector_reset", "sl_advect_learned", "sl_selftest_wait_timeout", "sl_advect_wide_workspace",
           "sl_advect_wide", "sl_autotune_scheme", "sl_tuning_get", "sl_tuning_save", "sl_tuning_load",
           "sl_tuning_clear", "sl_batch_autotune", "sl_batch_tuning", "sl_field_save", "sl_field_load",
           "sl_corrector_save", "sl_corrector_load", "sl_rb_create", "sl_rb_set_state", "sl_rb_get_state",
           "sl_rb_step", "sl_rb_destroy")
KERNELS = {1: "cec_fast", 2: "cec_split", 3: "cir_groups", 4: "unsplit"}


class SLError(RuntimeError):
    def __init__(self, code, message):
        super().__init__(f"{STATUS.get(code, code)}: {message}")
        self.code = code


class Tuning(ctypes.Structure):
    """sl_tuning"""
    _fields_ = [("kernel", ctypes.c_int), ("tile_x", ctypes.c_int), ("tile_y", ctypes.c_int),
                ("tile_z", ctypes.c_int), ("ctas_per_sm", ctypes.c_int), ("ms", ctypes.c_float)]

    def as_dict(self):
        return {"kernel": KERNELS.get(self.kernel, self.kernel), "tile": [self.tile_x, self.tile_y],
                "tile_z": self.tile_z, "ctas_per_sm": self.ctas_per_sm, "ms": float(self.ms)}


class Instance(ctypes.Structure):
    """sl_instance"""
    _fields_ = [("a", ctypes.c_void_p), ("b", ctypes.c_void_p), ("vel", ctypes.c_void_p),
                ("dims", ctypes.c_int64 * 3), ("spacing", ctypes.c_double * 3), ("dt", ctypes.c_double)]


_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _build.LIB


def load(path: str | None = None):
    """Load libsl.so (raises if it is missing; never builds implicitly)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = path or _build.LIB
        if not os.path.exists(path):
            raise RuntimeError(f"libsl.so not found at {path}: run paper_1606_06117_gb300.build.build() first")
        lib = ctypes.CDLL(path)
        vp, i, i64p, dp, d = ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int64), \
            ctypes.POINTER(ctypes.c_double), ctypes.c_double
        sig = {
            "sl_version": ([], i),
            "sl_last_error": ([], ctypes.c_char_p),
            "sl_init": ([], i),
            "sl_advect": ([vp, vp, vp, i, i64p, dp, d, i, i, i, vp], i),
            "sl_advect_multi": ([ctypes.POINTER(vp), ctypes.POINTER(vp), i, vp, i, i64p, dp, d, i, i, i, vp], i),
            "sl_advect_host": ([vp, vp, vp, i, i64p, dp, d, i, i, i, vp], i),
            "sl_release_host_staging": ([], i),
            "sl_courant_max": ([vp, i, i64p, dp, d, i, dp, vp], i),
            "sl_norms": ([vp, vp, ctypes.c_int64, i, dp, vp], i),
            "sl_norms_static": ([vp, vp, ctypes.c_int64, i, vp, vp], i),
            "sl_device_status": ([vp, ctypes.POINTER(ctypes.c_uint)], i),
            "sl_batch_create": ([ctypes.POINTER(vp), ctypes.POINTER(Instance), i, i, i, i], i),
            "sl_batch_step": ([vp, i, vp], i),
            "sl_batch_destroy": ([vp], i),
            "sl_autotune": ([vp, vp, vp, i, i64p, dp, d, i, ctypes.POINTER(i), vp], i),
            "sl_corrector_param_count": ([], i),
            "sl_corrector_create": ([ctypes.POINTER(vp), ctypes.c_uint64], i),
            "sl_corrector_destroy": ([vp], i),
            "sl_corrector_get_params": ([vp, ctypes.POINTER(ctypes.c_float), i], i),
            "sl_corrector_set_params": ([vp, ctypes.POINTER(ctypes.c_float), i], i),
            "sl_corrector_add_samples": ([vp, vp, vp, vp, i64p, dp, d, i, ctypes.c_uint64, vp], i),
            "sl_corrector_get_rows": ([vp, ctypes.POINTER(ctypes.c_float), ctypes.c_int64, ctypes.c_int64], i),
            "sl_corrector_train": ([vp, i, i, ctypes.c_float, ctypes.c_uint64, ctypes.POINTER(ctypes.c_float), vp], i),
            "sl_corrector_reset": ([vp], i),
            "sl_advect_learned": ([vp, vp, vp, vp, i, i64p, dp, d, i, i, d, ctypes.POINTER(i), dp, vp], i),
            "sl_selftest_wait_timeout": ([ctypes.c_uint, vp], i),
            "sl_advect_wide_workspace": ([i, i64p, i, i], ctypes.c_int64),
            "sl_advect_wide": ([vp, vp, vp, i, i64p, dp, d, i, i, i, vp, ctypes.c_int64, vp], i),
            "sl_autotune_scheme": ([vp, vp, vp, i, i64p, dp, d, i, i, ctypes.POINTER(Tuning), vp], i),
            "sl_tuning_get": ([i64p, i, i, ctypes.POINTER(Tuning)], i),
            "sl_tuning_save": ([ctypes.c_char_p], i),
            "sl_tuning_load": ([ctypes.c_char_p], i),
            "sl_tuning_clear": ([], i),
            "sl_batch_autotune": ([vp, ctypes.POINTER(Tuning), vp], i),
            "sl_batch_tuning": ([vp, ctypes.POINTER(Tuning)], i),
            "sl_field_save": ([ctypes.c_char_p, vp, i, i64p, i, ctypes.c_int64, vp], i),
            "sl_field_load": ([ctypes.c_char_p, vp, i, i64p, i, ctypes.POINTER(ctypes.c_int64), vp], i),
            "sl_corrector_save": ([vp, ctypes.c_char_p], i),
            "sl_corrector_load": ([vp, ctypes.c_char_p], i),
            "sl_rb_create": ([ctypes.POINTER(vp), i, i, d, d, d, d, i, i], i),
            "sl_rb_set_state": ([vp, vp, vp, vp, vp], i),
            "sl_rb_get_state": ([vp, vp, vp, vp, vp], i),
            "sl_rb_step": ([vp, d, i, vp], i),
            "sl_rb_destroy": ([vp], i),
        }
        for name, (args, res) in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
        return lib


def _check(rc):
    if rc != 0:
        raise SLError(rc, load().sl_last_error().decode())
    return rc


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, torch.Tensor):
        return ctypes.c_void_p(x.data_ptr())
    if isinstance(x, int):
        return ctypes.c_void_p(x)
    if isinstance(x, ctypes.c_void_p):
        return x
    raise TypeError(f"cannot pass {type(x)} as a pointer")


def _stream(s):
    if s is None:
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream) if torch.cuda.is_available() else None
    if isinstance(s, torch.cuda.Stream):
        return ctypes.c_void_p(s.cuda_stream)
    return ctypes.c_void_p(int(s))


def _i64(v):
    v = list(v) + [1] * (3 - len(v))
    return (ctypes.c_int64 * 3)(*v)


def _f64(v):
    v = list(v) + [1.0] * (3 - len(v))
    return (ctypes.c_double * 3)(*v)


# ------------------------------------------------------------------ C mirrors
def sl_version():
    return load().sl_version()


def sl_last_error():
    return load().sl_last_error().decode()


def sl_init():
    return _check(load().sl_init())


def sl_advect(out, inp, vel, ndim, dims, spacing, dt, scheme, dtype, step_parity=0, stream=None):
    return _check(load().sl_advect(_ptr(out), _ptr(inp), _ptr(vel), ndim, _i64(dims), _f64(spacing), float(dt),
                                   int(scheme), int(dtype), int(step_parity), _stream(stream)))


def sl_advect_multi(outs, ins, vel, ndim, dims, spacing, dt, scheme, dtype, step_parity=0, stream=None):
    n = len(outs)
    if len(ins) != n:
        raise ValueError("outs and ins must have the same length")
    po = (ctypes.c_void_p * n)(*[_ptr(o).value for o in outs])
    pi = (ctypes.c_void_p * n)(*[_ptr(i).value for i in ins])
    return _check(load().sl_advect_multi(po, pi, n, _ptr(vel), ndim, _i64(dims), _f64(spacing), float(dt),
                                         int(scheme), int(dtype), int(step_parity), _stream(stream)))


def sl_advect_host(out, inp, vel, ndim, dims, spacing, dt, scheme, dtype, step_parity=0, stream=None):
    return _check(load().sl_advect_host(_ptr(out), _ptr(inp), _ptr(vel), ndim, _i64(dims), _f64(spacing), float(dt),
                                        int(scheme), int(dtype), int(step_parity), _stream(stream)))


def sl_advect_wide_workspace(ndim, dims, scheme, dtype):
    n = load().sl_advect_wide_workspace(int(ndim), _i64(dims), int(scheme), int(dtype))
    if n < 0:
        raise SLError(int(n), load().sl_last_error().decode())
    return n


def sl_advect_wide(out, inp, vel, ndim, dims, spacing, dt, scheme, dtype, step_parity=0, workspace=None,
                   workspace_bytes=0, stream=None):
    return _check(load().sl_advect_wide(_ptr(out), _ptr(inp), _ptr(vel), ndim, _i64(dims), _f64(spacing), float(dt),
                                        int(scheme), int(dtype), int(step_parity), _ptr(workspace),
                                        int(workspace_bytes), _stream(stream)))


def sl_release_host_staging():
    return _check(load().sl_release_host_staging())


def sl_courant_max(vel, ndim, dims, spacing, dt, dtype, stream=None):
    out = ctypes.c_double()
    _check(load().sl_courant_max(_ptr(vel), ndim, _i64(dims), _f64(spacing), float(dt), int(dtype),
                                 ctypes.byref(out), _stream(stream)))
    return out.value


def sl_norms(a, b, n, dtype, stream=None):
    out = (ctypes.c_double * 3)()
    _check(load().sl_norms(_ptr(a), _ptr(b), int(n), int(dtype), out, _stream(stream)))
    return tuple(out)


def sl_norms_static(a, b, n, dtype, out, stream=None):
    """Norms into the device buffer ``out`` (3 float64) with no allocation."""
    return _check(load().sl_norms_static(_ptr(a), _ptr(b), int(n), int(dtype), _ptr(out), _stream(stream)))


def sl_selftest_wait_timeout(polls=1000, stream=None):
    """Returns the status code (SL_ERR_TIMEOUT = -5 when the bounded wait gave up)."""
    rc = load().sl_selftest_wait_timeout(int(polls), _stream(stream))
    if rc not in (0, -5):
        raise SLError(rc, load().sl_last_error().decode())
    return rc


def sl_device_status(stream=None):
    bits = ctypes.c_uint()
    _check(load().sl_device_status(_stream(stream), ctypes.byref(bits)))
    return bits.value


def sl_batch_create(instances, scheme=CEC, dtype=F32, tile_z=0):
    arr = (Instance * len(instances))(*instances)
    h = ctypes.c_void_p()
    _check(load().sl_batch_create(ctypes.byref(h), arr, len(instances), int(scheme), int(dtype), int(tile_z)))
    return h


def sl_batch_step(batch, step_index, stream=None):
    return _check(load().sl_batch_step(batch, int(step_index), _stream(stream)))


def sl_batch_destroy(batch):
    return _check(load().sl_batch_destroy(batch))


def sl_autotune(out, inp, vel, ndim, dims, spacing, dt, dtype, stream=None):
    tz = ctypes.c_int()
    _check(load().sl_autotune(_ptr(out), _ptr(inp), _ptr(vel), ndim, _i64(dims), _f64(spacing), float(dt),
                              int(dtype), ctypes.byref(tz), _stream(stream)))
    return tz.value


def sl_autotune_scheme(out, inp, vel, ndim, dims, spacing, dt, scheme, dtype, stream=None):
    t = Tuning()
    _check(load().sl_autotune_scheme(_ptr(out), _ptr(inp), _ptr(vel), ndim, _i64(dims), _f64(spacing), float(dt),
                                     int(scheme), int(dtype), ctypes.byref(t), _stream(stream)))
    return t


def sl_tuning_get(dims, scheme, dtype):
    """The cached launch shape, or None when nothing is cached."""
    t = Tuning()
    rc = load().sl_tuning_get(_i64(dims), int(scheme), int(dtype), ctypes.byref(t))
    if rc == -1:
        return None
    _check(rc)
    return t


def sl_tuning_save(path):
    return _check(load().sl_tuning_save(os.fsencode(path)))


def sl_tuning_load(path):
    return _check(load().sl_tuning_load(os.fsencode(path)))


def sl_tuning_clear():
    return _check(load().sl_tuning_clear())


def sl_batch_autotune(batch, stream=None):
    t = Tuning()
    _check(load().sl_batch_autotune(batch, ctypes.byref(t), _stream(stream)))
    return t


def sl_batch_tuning(batch):
    t = Tuning()
    _check(load().sl_batch_tuning(batch, ctypes.byref(t)))
    return t


def sl_field_save(path, field, ndim, dims, dtype, step=0, stream=None):
    return _check(load().sl_field_save(os.fsencode(path), _ptr(field), int(ndim), _i64(dims), int(dtype),
                                       int(step), _stream(stream)))


def sl_field_load(path, field, ndim, dims, dtype, stream=None):
    """Returns the saved step."""
    step = ctypes.c_int64()
    _check(load().sl_field_load(os.fsencode(path), _ptr(field), int(ndim), _i64(dims), int(dtype),
                                ctypes.byref(step), _stream(stream)))
    return step.value


def sl_corrector_save(c, path):
    return _check(load().sl_corrector_save(c, os.fsencode(path)))


def sl_corrector_load(c, path):
    return _check(load().sl_corrector_load(c, os.fsencode(path)))


def sl_corrector_param_count():
    return load().sl_corrector_param_count()


def sl_corrector_create(seed=0):
    h = ctypes.c_void_p()
    _check(load().sl_corrector_create(ctypes.byref(h), int(seed)))
    return h


def sl_corrector_destroy(c):
    return _check(load().sl_corrector_destroy(c))


def sl_corrector_get_params(c):
    import numpy as np
    out = np.empty(sl_corrector_param_count(), dtype=np.float32)
    _check(load().sl_corrector_get_params(c, out.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), out.size))
    return out


def sl_corrector_set_params(c, params):
    import numpy as np
    a = np.ascontiguousarray(params, dtype=np.float32)
    return _check(load().sl_corrector_set_params(c, a.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), a.size))


def sl_corrector_add_samples(c, phi, target, vel, dims, spacing, dt, nsamples, seed=0, stream=None):
    return _check(load().sl_corrector_add_samples(c, _ptr(phi), _ptr(target), _ptr(vel), _i64(dims), _f64(spacing),
                                                  float(dt), int(nsamples), int(seed), _stream(stream)))


def sl_corrector_get_rows(c, first, n):
    import numpy as np
    out = np.empty((n, 68), dtype=np.float32)
    _check(load().sl_corrector_get_rows(c, out.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), int(first), int(n)))
    return out


def sl_corrector_train(c, iters, batch, lr, seed=0, stream=None):
    loss = ctypes.c_float()
    _check(load().sl_corrector_train(c, int(iters), int(batch), float(lr), int(seed), ctypes.byref(loss),
                                     _stream(stream)))
    return loss.value


def sl_corrector_reset(c):
    return _check(load().sl_corrector_reset(c))


def sl_advect_learned(c, out, inp, vel, ndim, dims, spacing, dt, step_parity=0, check=0, fallback_ratio=2.0,
                      stream=None):
    """Returns (used_plain, (learned_error, plain_error) or None)."""
    used = ctypes.c_int()
    errs = (ctypes.c_double * 2)(-1.0, -1.0)
    _check(load().sl_advect_learned(c, _ptr(out), _ptr(inp), _ptr(vel), ndim, _i64(dims), _f64(spacing), float(dt),
                                    int(step_parity), int(check), float(fallback_ratio), ctypes.byref(used), errs,
                                    _stream(stream)))
    return used.value, ((errs[0], errs[1]) if check else None)


# ------------------------------------------------------------- conveniences
def dtype_code(t: torch.dtype, delta64: bool = False) -> int:
    if t == torch.float64:
        return F64
    if t == torch.float32:
        return F32_D64 if delta64 else F32
    raise TypeError(f"unsupported field dtype {t}")


def geometry(phi: torch.Tensor, spacing=None):
    """(ndim, dims (x,y,z), spacing (x,y,z)) of a (ny, nx) or (nz, ny, nx) field."""
    if phi.dim() not in (2, 3):
        raise ValueError("fields must be 2D (ny, nx) or 3D (nz, ny, nx)")
    ndim = phi.dim()
    dims = list(phi.shape)[::-1] + ([1] if ndim == 2 else [])
    if spacing is None:
        spacing = [1.0 / n for n in dims[:ndim]]
    sp = list(spacing) + ([1.0] if ndim == 2 else [])
    return ndim, dims, sp


def advect(phi: torch.Tensor, vel: torch.Tensor, dt: float, spacing=None, scheme="CEC", parity: int = 0,
           out: torch.Tensor | None = None, delta64: bool = False, stream=None) -> torch.Tensor:
    """One step of ``scheme`` on a CUDA field; returns ``out`` (allocated if None)."""
    ndim, dims, sp = geometry(phi, spacing)
    if not (phi.is_cuda and vel.is_cuda):
        raise ValueError("advect runs on CUDA tensors only")
    if vel.shape != (ndim,) + tuple(phi.shape) or vel.dtype != phi.dtype:
        raise ValueError("vel must be (ndim, *phi.shape) with phi's dtype")
    phi = phi.contiguous()
    vel = vel.contiguous()
    if out is None:
        out = torch.empty_like(phi)
    sc = SCHEMES[scheme] if isinstance(scheme, str) else int(scheme)
    sl_advect(out, phi, vel, ndim, dims, sp, dt, sc, dtype_code(phi.dtype, delta64), parity, stream)
    return out


def advect_wide(phi: torch.Tensor, vel: torch.Tensor, dt: float, spacing=None, scheme="CEC", parity: int = 0,
                out: torch.Tensor | None = None, workspace: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """One step at any Courant number (sl_advect_wide) on CUDA tensors; allocates
    ``out`` and the workspace (a uint8 CUDA tensor) when they are None."""
    ndim, dims, sp = geometry(phi, spacing)
    if not (phi.is_cuda and vel.is_cuda):
        raise ValueError("advect_wide runs on CUDA tensors only")
    if vel.shape != (ndim,) + tuple(phi.shape) or vel.dtype != phi.dtype:
        raise ValueError("vel must be (ndim, *phi.shape) with phi's dtype")
    phi = phi.contiguous()
    vel = vel.contiguous()
    if out is None:
        out = torch.empty_like(phi)
    sc = SCHEMES[scheme] if isinstance(scheme, str) else int(scheme)
    dc = dtype_code(phi.dtype)
    need = sl_advect_wide_workspace(ndim, dims, sc, dc)
    if workspace is None and need > 0:
        workspace = torch.empty(need + 256, dtype=torch.uint8, device=phi.device)
    ws, nbytes = None, 0
    if workspace is not None:
        base = workspace.data_ptr()
        off = (-base) % 256
        ws, nbytes = base + off, workspace.numel() * workspace.element_size() - off
    sl_advect_wide(out, phi, vel, ndim, dims, sp, dt, sc, dc, parity, ws, nbytes, stream)
    return out


def sl_rb_create(nx, nz, Lx=2.0, Lz=1.0, Ra=1e5, Pr=1.0, scheme="CEC", dtype=F64):
    h = ctypes.c_void_p()
    sc = SCHEMES[scheme] if isinstance(scheme, str) else int(scheme)
    _check(load().sl_rb_create(ctypes.byref(h), int(nx), int(nz), float(Lx), float(Lz), float(Ra), float(Pr), sc,
                               int(dtype)))
    return h


def sl_rb_set_state(rb, u, w, theta, stream=None):
    return _check(load().sl_rb_set_state(rb, _ptr(u), _ptr(w), _ptr(theta), _stream(stream)))


def sl_rb_get_state(rb, u, w, theta, stream=None):
    return _check(load().sl_rb_get_state(rb, _ptr(u), _ptr(w), _ptr(theta), _stream(stream)))


def sl_rb_step(rb, dt, nsteps=1, stream=None):
    return _check(load().sl_rb_step(rb, float(dt), int(nsteps), _stream(stream)))


def sl_rb_destroy(rb):
    return _check(load().sl_rb_destroy(rb))


class RayleighBenard:
    """A Rayleigh-Benard box on the current CUDA device (sl_rb_*): the state
    as (nz, nx) CUDA tensors of the box's dtype."""

    def __init__(self, nx, nz, Lx=2.0, Lz=1.0, Ra=1e5, Pr=1.0, scheme="CEC", dtype=torch.float64):
        self.nx, self.nz, self.dtype = nx, nz, dtype
        self.h = sl_rb_create(nx, nz, Lx, Lz, Ra, Pr, scheme, dtype_code(dtype))

    def set_state(self, u, w, theta):
        t = [x.to(device="cuda", dtype=self.dtype).contiguous() for x in (u, w, theta)]
        if any(x.shape != (self.nz, self.nx) for x in t):
            raise ValueError("u, w and theta must be (nz, nx)")
        sl_rb_set_state(self.h, *t)
        torch.cuda.current_stream().synchronize()

    def state(self):
        out = [torch.empty((self.nz, self.nx), dtype=self.dtype, device="cuda") for _ in range(3)]
        sl_rb_get_state(self.h, *out)
        return out

    def step(self, dt, nsteps=1):
        sl_rb_step(self.h, dt, nsteps)

    def close(self):
        if self.h is not None:
            sl_rb_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
