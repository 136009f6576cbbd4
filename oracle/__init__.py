"""FP64 CPU oracle for the scalar string field (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never calls it,
and it shares no code with the CUDA path: ``sp_oracle.c`` is plain C built
with gcc, driven here through ctypes with numpy arrays.

Functions and the passage each follows:

* :func:`level_coeffs` -- conformal time, scale factor a = (tau/tau_ref)^nu,
  friction d = nu dt / tau and the leapfrog factors at one level.  The model
  equation is the one the method is applied to; the paper (Sec. 5) evolves
  its strings in conformal time in a flat Robertson-Walker universe so that
  the causal structure stays Minkowskian, and the regions of Sec. 2 rely on
  exactly that.
* :func:`run` -- whole-grid FP64 leapfrog, the plain definition that the
  region decomposition (Sec. 1, Sec. 2) must reproduce.
* :func:`run_fp32_storage` -- the same steps with the state rounded to FP32
  after each one: how far storage in FP32 alone moves a run (the yardstick
  for the accuracy bar on chaotic runs).
* :func:`energy_parts`, :func:`lap_dot` -- energy of a stored state and the
  lattice-Laplacian bilinear form.
* :func:`winding` -- exact per-plaquette winding numbers (string detection).

Pins for each function are in ``tests/test_oracle_pins.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sp_oracle.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "libsp_oracle.so")
_lock = threading.Lock()
_lib = None


class Params(ctypes.Structure):
    """Mirror of ``or_params`` in sp_oracle.c."""

    _fields_ = [
        ("n", ctypes.c_int32 * 3),
        ("dx", ctypes.c_double),
        ("dt", ctypes.c_double),
        ("lam", ctypes.c_double),
        ("eta", ctypes.c_double),
        ("nu", ctypes.c_double),
        ("tau0", ctypes.c_double),
        ("tau_ref", ctypes.c_double),
        ("damp_steps", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
    ]


def make_params(n, dx=1.0, dt=0.25, lam=2.0, eta=1.0, nu=0.0, tau0=1.0, tau_ref=1.0, damp_steps=0):
    if isinstance(n, int):
        n = (n, n, n)
    p = Params()
    p.n[0], p.n[1], p.n[2] = (int(v) for v in n)
    p.dx, p.dt, p.lam, p.eta, p.nu = float(dx), float(dt), float(lam), float(eta), float(nu)
    p.tau0, p.tau_ref, p.damp_steps = float(tau0), float(tau_ref), int(damp_steps)
    return p


def build(force: bool = False) -> str:
    """Compile sp_oracle.c with gcc (OpenMP, no FMA contraction)."""
    os.makedirs(_LIB_DIR, exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off", "-std=c11",
           _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.POINTER(Params)
            dp = ctypes.POINTER(ctypes.c_double)
            lib.or_level_coeffs.argtypes = [P, ctypes.c_int64, dp]
            lib.or_step.argtypes = [P, ctypes.c_int64, dp, dp, ctypes.c_int]
            lib.or_run.argtypes = [P, ctypes.c_int64, ctypes.c_int64, dp, dp, ctypes.c_int]
            lib.or_run_fp32_storage.argtypes = [P, ctypes.c_int64, ctypes.c_int64, dp, dp, ctypes.c_int]
            lib.or_energy_parts.argtypes = [P, ctypes.c_int64, dp, dp, dp, ctypes.c_int]
            lib.or_lap_dot.argtypes = [ctypes.POINTER(ctypes.c_int32), ctypes.c_double, dp, dp, ctypes.c_int]
            lib.or_lap_dot.restype = ctypes.c_double
            lib.or_winding.argtypes = [ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_float),
                                       ctypes.POINTER(ctypes.c_int8), ctypes.c_int]
            lib.or_max_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _as_c128(a):
    """Complex field as a C-contiguous complex128 array (a copy)."""
    return np.ascontiguousarray(np.asarray(a), dtype=np.complex128).copy()


def max_threads() -> int:
    return int(_load().or_max_threads())


def level_coeffs(p: Params, level: int) -> dict:
    out = np.zeros(6)
    _load().or_level_coeffs(ctypes.byref(p), int(level), _dptr(out))
    return dict(zip(("tau", "a", "d", "c1", "c2", "m"), out.tolist()))


def run(p: Params, phi, pi, level0: int, nsteps: int, nthreads: int = 0):
    """Evolve (phi, pi) from level0 by nsteps in FP64; returns new complex128 arrays.

    ``phi`` holds phi at level0, ``pi`` holds pi at level0 - 1/2.  Arrays are
    (nz, ny, nx); any float or complex dtype is widened to FP64 first.
    """
    f = _as_c128(phi)
    v = _as_c128(pi)
    _load().or_run(ctypes.byref(p), int(level0), int(nsteps), _dptr(f.view(np.float64)),
                   _dptr(v.view(np.float64)), int(nthreads))
    return f, v


def run_fp32_storage(p: Params, phi, pi, level0: int, nsteps: int, nthreads: int = 0):
    """As :func:`run`, with phi and pi rounded to FP32 after every step: the
    error floor of any scheme that stores the field in FP32."""
    f = _as_c128(phi)
    v = _as_c128(pi)
    _load().or_run_fp32_storage(ctypes.byref(p), int(level0), int(nsteps), _dptr(f.view(np.float64)),
                                _dptr(v.view(np.float64)), int(nthreads))
    return f, v


def step(p: Params, phi, pi, level: int, nthreads: int = 0):
    return run(p, phi, pi, level, 1, nthreads)


def energy_parts(p: Params, phi, pi, level: int, nthreads: int = 0):
    """(sum |pi|^2, gradient sum, potential sum) of a stored state at ``level``."""
    f = _as_c128(phi)
    v = _as_c128(pi)
    out = np.zeros(3)
    _load().or_energy_parts(ctypes.byref(p), int(level), _dptr(f.view(np.float64)),
                            _dptr(v.view(np.float64)), _dptr(out), int(nthreads))
    return tuple(out.tolist())


def lap_dot(n, dx, phi, psi, nthreads: int = 0) -> float:
    """Re sum conj(phi) (-Lap7 psi) / dx^2 over the periodic grid."""
    n3 = (ctypes.c_int32 * 3)(*[int(v) for v in n])
    f = _as_c128(phi)
    g = _as_c128(psi)
    return float(_load().or_lap_dot(n3, float(dx), _dptr(f.view(np.float64)), _dptr(g.view(np.float64)),
                                    int(nthreads)))


def winding(phi32, nthreads: int = 0) -> np.ndarray:
    """Exact plaquette windings of an FP32 complex field (nz, ny, nx).

    Returns int8 array (3, nz, ny, nx): index 0 = plaquettes normal to x,
    1 = normal to y, 2 = normal to z.
    """
    f = np.ascontiguousarray(np.asarray(phi32), dtype=np.complex64)
    nz, ny, nx = f.shape
    n3 = (ctypes.c_int32 * 3)(nx, ny, nz)
    w = np.zeros((3, nz, ny, nx), dtype=np.int8)
    _load().or_winding(n3, f.view(np.float32).ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                       w.ctypes.data_as(ctypes.POINTER(ctypes.c_int8)), int(nthreads))
    return w
