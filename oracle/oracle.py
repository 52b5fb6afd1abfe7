"""FP64 CPU oracle of the multi-stage semi-Lagrangian schemes (arXiv 1606.06117).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import this module; the product path never
does.  It wraps ``sl_oracle.c`` (plain C, FP64, single thread, built with
``-ffp-contract=off``) through ctypes and shares nothing with the CUDA library.

Array conventions: fields are float64 numpy arrays of shape ``(nz, ny, nx)``
(``(ny, nx)`` in 2D, ``(nx,)`` in 1D), x fastest.  ``courant`` is a float64
array with one leading plane per axis, ``courant[d] = u_d * dt / dx_d`` taken at
each (arrival) cell, axis order x, y, z.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

CIR, FEC, BEC, CEC, CEC_DEF = 0, 1, 2, 3, 4
# large Courant numbers (Sec. 4, eq. intro:CECcoefSL), split CEC in two readings:
# correction at the departure cell (adopted) and the literal operator definitions
CEC_SL, CEC_SL_LIT = 5, 6
SCHEMES = {"CIR": CIR, "FEC": FEC, "BEC": BEC, "CEC": CEC}

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sl_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile sl_oracle.c into oracle/_build/liboracle.so (gcc, -O2, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
             "-Wall", "-Wextra", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.POINTER
            d, i64, i = ctypes.c_double, ctypes.c_int64, ctypes.c_int
            lib.orc_interp.argtypes = [P(d), P(d), P(d), P(i64), i, i]
            lib.orc_interp_axis.argtypes = [P(d), P(d), P(d), P(i64), i, i]
            lib.orc_scheme_on.argtypes = [P(d), P(d), P(d), P(i64), i, i, i]
            lib.orc_step.argtypes = [P(d), P(d), P(d), P(i64), i, i, i]
            lib.orc_sample.argtypes = [P(d), P(d), P(d), P(i64), i, i, i, P(i64), i64]
            lib.orc_norms.argtypes = [P(d), P(d), P(d), i64]
            for f in ("orc_interp", "orc_interp_axis", "orc_scheme_on", "orc_step",
                      "orc_sample", "orc_norms"):
                getattr(lib, f).restype = ctypes.c_int
            _lib = lib
    return _lib


def _ptr(a, ctype=ctypes.c_double):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _dims(shape):
    n = list(shape)[::-1]          # x, y, z
    ndim = len(n)
    while len(n) < 3:
        n.append(1)
    return np.asarray(n, dtype=np.int64), ndim


def _prep(phi, courant):
    phi = np.ascontiguousarray(phi, dtype=np.float64)
    n, ndim = _dims(phi.shape)
    courant = np.ascontiguousarray(courant, dtype=np.float64)
    if courant.shape != (ndim,) + phi.shape:
        raise ValueError(f"courant must have shape {(ndim,) + phi.shape}, got {courant.shape}")
    return phi, courant, n, ndim


def _check(rc, what):
    if rc != 0:
        raise RuntimeError(f"{what} failed with code {rc}")


def interp(phi, courant, direction=+1):
    """Multilinear L_U (direction=+1) or L_{-U} (direction=-1) on all axes."""
    phi, courant, n, ndim = _prep(phi, courant)
    out = np.empty_like(phi)
    _check(_load().orc_interp(_ptr(out), _ptr(phi), _ptr(courant), _ptr(n, ctypes.c_int64),
                              ndim, direction), "orc_interp")
    return out


def interp_axis(phi, courant_axis, axis, direction=+1):
    """1D linear interpolation along one axis (x=0, y=1, z=2)."""
    phi = np.ascontiguousarray(phi, dtype=np.float64)
    n, _ = _dims(phi.shape)
    ca = np.ascontiguousarray(courant_axis, dtype=np.float64)
    if ca.shape != phi.shape:
        raise ValueError("courant_axis must have the field's shape")
    out = np.empty_like(phi)
    _check(_load().orc_interp_axis(_ptr(out), _ptr(phi), _ptr(ca), _ptr(n, ctypes.c_int64),
                                   axis, direction), "orc_interp_axis")
    return out


def scheme_on(phi, courant, scheme, axis=-1):
    """One application of CIR/FEC/BEC (axis=-1: unsplit on all axes; axis>=0: 1D along it)
    or CEC / CEC_DEF (1D only)."""
    phi, courant, n, ndim = _prep(phi, courant)
    out = np.empty_like(phi)
    _check(_load().orc_scheme_on(_ptr(out), _ptr(phi), _ptr(courant), _ptr(n, ctypes.c_int64),
                                 ndim, axis, scheme), "orc_scheme_on")
    return out


def step(phi, courant, scheme, parity=0):
    """One time step: CIR/FEC/BEC unsplit; CEC, CEC_SL, CEC_SL_LIT split with alternating sweep order."""
    phi, courant, n, ndim = _prep(phi, courant)
    out = np.empty_like(phi)
    _check(_load().orc_step(_ptr(out), _ptr(phi), _ptr(courant), _ptr(n, ctypes.c_int64),
                            ndim, scheme, parity), "orc_step")
    return out


def run(phi, courant_fn, scheme, nsteps, parity0=0):
    """nsteps steps; courant_fn(step_index) -> courant array (or a fixed array)."""
    for k in range(nsteps):
        c = courant_fn(k) if callable(courant_fn) else courant_fn
        phi = step(phi, c, scheme, parity0 + k)
    return phi


def sample(phi, courant, scheme, parity, cells):
    """The result of ``step`` at the given cells (array of (x, y, z) rows)."""
    phi, courant, n, ndim = _prep(phi, courant)
    cells = np.ascontiguousarray(cells, dtype=np.int64).reshape(-1, 3)
    out = np.empty(len(cells), dtype=np.float64)
    _check(_load().orc_sample(_ptr(out), _ptr(phi), _ptr(courant), _ptr(n, ctypes.c_int64),
                              ndim, scheme, parity, _ptr(cells, ctypes.c_int64), len(cells)),
           "orc_sample")
    return out


def norms(a, b):
    """(RMS of a-b, max |a-b|, ||a-b||_2/||b||_2), accumulated in FP64."""
    a = np.ascontiguousarray(a, dtype=np.float64).ravel()
    b = np.ascontiguousarray(b, dtype=np.float64).ravel()
    out = np.empty(3, dtype=np.float64)
    _check(_load().orc_norms(_ptr(out), _ptr(a), _ptr(b), a.size), "orc_norms")
    return tuple(float(v) for v in out)
