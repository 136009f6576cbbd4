"""Python binding of the C ABI in include/sp.h (argument marshalling only).

The functions ``sp_grid_create``, ``sp_region_plan``, ``sp_evolve``,
``sp_read_surface``, ``sp_write_surface``, ``sp_destroy`` and
``sp_strerror`` have the names and meaning of the C entry points; every
site-update they cause runs in the CUDA kernels of ``libsp.so``.  There is no
Python or CPU compute path: if the library is not built, loading raises.

:class:`Grid` is a convenience wrapper that keeps the handle together with
the torch tensors (device memory) and stream it was created with.
"""
from __future__ import annotations

import ctypes
import os
import re
import threading

import numpy as np

from . import build as _build

SP_OK = 0
SP_EINVAL = -1
SP_ENOMEM = -2
SP_ECUDA = -3
SP_EUNSTABLE = -4
SP_ETIMEOUT = -5
SP_ENONFINITE = -6
SP_EFAULT_INJECTED = -7
SP_ENOTPLANNED = -8
SP_ESCRATCH = -9
SP_NOALLOC_MAX_SITES = 262144
SP_NOALLOC_MAX_STEPS = 8192

SP_ASYNC = 1
SP_MONOLITHIC = 2
SP_RESTART = 4
SP_TRACE = 8
SP_TIMING = 16
SP_FEATURES = 32

SP_SURF_STATE = 0
SP_SURF_DIAG = 1
SP_SURF_TRACE = 2
SP_SURF_WINDING = 3
SP_SURF_PLAN = 4
SP_SURF_TIMING = 5
SP_SURF_FEATURES = 6
SP_SURF_LEVEL = 7
SP_OPT_WAIT_LIMIT_NS = 1
SP_OPT_FAULT_DROP_RELEASE = 2
SP_OPT_GRAPHS = 3
SP_OPT_MAILBOX_SLOTS = 4
SP_OPT_REGION_SHAPE = 5
SP_SHAPE_SPLIT = 0
SP_SHAPE_LATTICE = 1
SP_MODEL_FEATURES = 16
SP_MODEL_PARAMS = 5313

SP_AUTOTUNE = -1
SP_ORDER_STATIC = 0
SP_ORDER_LEARNED = 1
SP_FP32_KAHAN = 0


class sp_params(ctypes.Structure):
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
        ("precision", ctypes.c_int32),
    ]


class sp_diag(ctypes.Structure):
    _fields_ = [
        ("level", ctypes.c_int64),
        ("tau", ctypes.c_double),
        ("a", ctypes.c_double),
        ("kinetic", ctypes.c_double),
        ("gradient", ctypes.c_double),
        ("potential", ctypes.c_double),
        ("total", ctypes.c_double),
        ("pierced", ctypes.c_int64 * 3),
        ("abs_winding", ctypes.c_int64),
        ("net_winding", ctypes.c_int64 * 3),
        ("string_length", ctypes.c_double),
    ]


class sp_plan_info(ctypes.Structure):
    _fields_ = [
        ("base_B", ctypes.c_int32),
        ("threads", ctypes.c_int32),
        ("ctas_per_sm", ctypes.c_int32),
        ("grid", ctypes.c_int32),
        ("regions_per_band", ctypes.c_int64),
        ("updates_per_band", ctypes.c_int64),
        ("bytes_read_per_band", ctypes.c_int64),
        ("bytes_written_per_band", ctypes.c_int64),
        ("bytes_per_update", ctypes.c_double),
        ("mailbox_bytes", ctypes.c_int64),
        ("autotuned", ctypes.c_int32),
        ("tune_candidates", ctypes.c_int32),
        ("tune_best_ms", ctypes.c_double),
        ("tune_default_ms", ctypes.c_double),
        ("mailbox_slots", ctypes.c_int32),
        ("region_shape", ctypes.c_int32),
    ]


class SpError(RuntimeError):
    def __init__(self, code, what=""):
        self.code = code
        super().__init__(f"{what}: {sp_strerror(code)} ({code})" if what else f"{sp_strerror(code)} ({code})")


_lock = threading.Lock()
_lib = None

HEADER = os.path.join(_build.ROOT, "include", "sp.h")


def declared_entry_points():
    """Function names declared in include/sp.h."""
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:int|const char \*)\s*(sp_\w+)\s*\(", text, flags=re.M)))


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Load libsp.so; raises if it is not built (no fallback exists)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if not os.path.exists(path):
            if not build_if_missing:
                raise RuntimeError(f"{path} is missing: build it with __graft_entry__.build() (needs nvcc)")
            _build.build()
        lib = ctypes.CDLL(path)
        vp = ctypes.c_void_p
        lib.sp_grid_create.argtypes = [ctypes.POINTER(sp_params), ctypes.c_int32, ctypes.POINTER(vp), vp,
                                       ctypes.POINTER(vp)]
        lib.sp_region_plan.argtypes = [vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_char_p]
        lib.sp_evolve.argtypes = [vp, ctypes.c_int64, ctypes.c_uint32]
        lib.sp_read_surface.argtypes = [vp, ctypes.c_int32, ctypes.c_int32, vp, ctypes.c_size_t, ctypes.c_int32]
        lib.sp_write_surface.argtypes = [vp, ctypes.c_int32, ctypes.c_int32, vp, ctypes.c_size_t, ctypes.c_int32]
        lib.sp_destroy.argtypes = [vp]
        lib.sp_sweep_noalloc.argtypes = [ctypes.POINTER(sp_params), vp, vp, ctypes.c_int64, ctypes.c_int64, vp]
        lib.sp_set_option.argtypes = [vp, ctypes.c_int32, ctypes.c_int64]
        lib.sp_measure_peaks.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
        i64p = ctypes.POINTER(ctypes.c_int64)
        lib.sp_lattice_call_bytes.argtypes = [ctypes.c_int32, ctypes.c_int64, i64p, i64p, i64p]
        lib.sp_strerror.argtypes = [ctypes.c_int]
        lib.sp_strerror.restype = ctypes.c_char_p
        fp = ctypes.POINTER(ctypes.c_float)
        lib.sp_model_create.argtypes = [ctypes.c_uint64, vp, ctypes.POINTER(vp)]
        lib.sp_model_destroy.argtypes = [vp]
        lib.sp_model_get_params.argtypes = [vp, fp, fp]
        lib.sp_model_set_params.argtypes = [vp, fp, fp]
        lib.sp_model_predict.argtypes = [vp, vp, ctypes.c_int64, vp]
        lib.sp_model_grad.argtypes = [vp, vp, vp, ctypes.c_int64, fp, ctypes.POINTER(ctypes.c_double)]
        lib.sp_model_adam_step.argtypes = [vp, fp, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float]
        lib.sp_model_train.argtypes = [vp, vp, vp, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, ctypes.c_float,
                                       ctypes.c_uint64, ctypes.POINTER(ctypes.c_int32), fp]
        lib.sp_model_save.argtypes = [vp, ctypes.c_char_p]
        lib.sp_model_load.argtypes = [ctypes.c_char_p, vp, ctypes.POINTER(vp)]
        for f in ("sp_grid_create", "sp_region_plan", "sp_evolve", "sp_read_surface", "sp_write_surface",
                  "sp_destroy", "sp_sweep_noalloc", "sp_model_create", "sp_model_destroy", "sp_model_get_params",
                  "sp_model_set_params", "sp_model_predict", "sp_model_grad", "sp_model_adam_step", "sp_model_train",
                  "sp_model_save", "sp_model_load", "sp_set_option", "sp_measure_peaks"):
            getattr(lib, f).restype = ctypes.c_int
        _lib = lib
        return lib


# ------------------------------------------------------------ C entry points
def sp_strerror(code: int) -> str:
    return load().sp_strerror(int(code)).decode()


def sp_grid_create(params, state_ptrs=None, stream: int = 0):
    """params: sequence of sp_params; state_ptrs: None or 3*len(params) device addresses."""
    n = len(params)
    arr = (sp_params * n)(*params)
    ptrs = None
    if state_ptrs is not None:
        ptrs = (ctypes.c_void_p * len(state_ptrs))(*[int(p) for p in state_ptrs])
    h = ctypes.c_void_p()
    rc = load().sp_grid_create(arr, n, ptrs, ctypes.c_void_p(int(stream)), ctypes.byref(h))
    return rc, h


def sp_region_plan(h, base_B=0, block_shape=0, order=SP_ORDER_STATIC, model_path=None):
    mp = model_path.encode() if model_path else None
    return load().sp_region_plan(h, int(base_B), int(block_shape), int(order), mp)


def sp_evolve(h, n_steps, flags=0):
    return load().sp_evolve(h, int(n_steps), int(flags))


def sp_read_surface(h, sim, what, dst_ptr, dst_bytes, dst_is_device):
    return load().sp_read_surface(h, int(sim), int(what), ctypes.c_void_p(int(dst_ptr)), int(dst_bytes),
                                  int(bool(dst_is_device)))


def sp_write_surface(h, sim, what, src_ptr, src_bytes, src_is_device):
    return load().sp_write_surface(h, int(sim), int(what), ctypes.c_void_p(int(src_ptr)), int(src_bytes),
                                   int(bool(src_is_device)))


def sp_destroy(h):
    return load().sp_destroy(h)


def sp_sweep_noalloc(params, phi_ptr, pic_ptr, level0, n_steps, stream=0):
    """Whole-grid steps with no memory allocation (see include/sp.h)."""
    return load().sp_sweep_noalloc(ctypes.byref(params), ctypes.c_void_p(int(phi_ptr)), ctypes.c_void_p(int(pic_ptr)),
                                   int(level0), int(n_steps), ctypes.c_void_p(int(stream)))


def sp_measure_peaks(stream=0):
    """(shared-memory GB/s, FP32 TFLOP/s) measured on the current device."""
    smem, fp32 = ctypes.c_double(), ctypes.c_double()
    rc = load().sp_measure_peaks(ctypes.c_void_p(int(stream)), ctypes.byref(smem), ctypes.byref(fp32))
    _check(rc, "sp_measure_peaks")
    return smem.value, fp32.value


def sp_lattice_call_bytes(B, n_steps):
    """(site-updates, bytes read, bytes written) of one lattice region column
    over a call of n_steps levels (host only)."""
    u, r, w = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    _check(load().sp_lattice_call_bytes(int(B), int(n_steps), ctypes.byref(u), ctypes.byref(r), ctypes.byref(w)),
           "sp_lattice_call_bytes")
    return u.value, r.value, w.value


# ------------------------------------------------------------ helpers
def make_params(n, dx=1.0, dt=0.25, lam=2.0, eta=1.0, nu=0.0, tau0=1.0, tau_ref=1.0, damp_steps=0) -> sp_params:
    if isinstance(n, int):
        n = (n, n, n)
    p = sp_params()
    p.n[0], p.n[1], p.n[2] = (int(v) for v in n)
    p.dx, p.dt, p.lam, p.eta, p.nu = float(dx), float(dt), float(lam), float(eta), float(nu)
    p.tau0, p.tau_ref, p.damp_steps, p.precision = float(tau0), float(tau_ref), int(damp_steps), SP_FP32_KAHAN
    return p


def pack_state(phi, pi, c) -> np.ndarray:
    """SP_SURF_STATE layout: phi (sites complex64) then pic (sites x (pi, c))."""
    phi = np.ascontiguousarray(phi, dtype=np.complex64).ravel()
    pic = np.stack([np.asarray(pi, dtype=np.complex64).ravel(), np.asarray(c, dtype=np.complex64).ravel()], axis=1)
    return np.concatenate([phi, pic.ravel()])


def unpack_state(buf, shape):
    """Inverse of pack_state: (phi, pi, c), each complex64 of ``shape``."""
    sites = int(np.prod(shape))
    buf = np.asarray(buf).view(np.complex64).ravel()
    phi = buf[:sites].reshape(shape)
    pic = buf[sites:3 * sites].reshape(sites, 2)
    return phi, pic[:, 0].reshape(shape).copy(), pic[:, 1].reshape(shape).copy()


def _fptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


class Model:
    """The region cost model (include/sp.h, sp_model_*): device parameters,
    trained and evaluated by the library's kernels.  Inputs of predict, grad
    and train are device addresses (e.g. torch tensors' data_ptr())."""

    def __init__(self, seed=0, stream=None, path=None):
        import torch

        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = ctypes.c_void_p()
        lib = load()
        if path is None:
            rc = lib.sp_model_create(int(seed), ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h))
        else:
            rc = lib.sp_model_load(str(path).encode(), ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h))
        _check(rc, "sp_model_create")
        self.h = h

    def params(self):
        p = np.empty(SP_MODEL_PARAMS, dtype=np.float32)
        t = np.empty(3, dtype=np.float32)
        _check(load().sp_model_get_params(self.h, _fptr(p), _fptr(t)), "sp_model_get_params")
        return p, t

    def set_params(self, params, thresholds=None):
        p = np.ascontiguousarray(params, dtype=np.float32)
        t = None if thresholds is None else np.ascontiguousarray(thresholds, dtype=np.float32)
        _check(load().sp_model_set_params(self.h, _fptr(p), None if t is None else _fptr(t)), "sp_model_set_params")

    def predict(self, x_ptr, n, y_ptr):
        _check(load().sp_model_predict(self.h, ctypes.c_void_p(int(x_ptr)), int(n), ctypes.c_void_p(int(y_ptr))),
               "sp_model_predict")

    def grad(self, x_ptr, y_ptr, n):
        g = np.empty(SP_MODEL_PARAMS, dtype=np.float32)
        loss = ctypes.c_double()
        _check(load().sp_model_grad(self.h, ctypes.c_void_p(int(x_ptr)), ctypes.c_void_p(int(y_ptr)), int(n),
                                    _fptr(g), ctypes.byref(loss)), "sp_model_grad")
        return float(loss.value), g

    def adam_step(self, grad, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
        g = np.ascontiguousarray(grad, dtype=np.float32)
        _check(load().sp_model_adam_step(self.h, _fptr(g), lr, beta1, beta2, eps), "sp_model_adam_step")

    def train(self, x_ptr, y_ptr, n, epochs, batch, lr=1e-3, order_seed=0, order=None):
        steps = epochs * ((n + batch - 1) // batch)
        losses = np.empty(steps, dtype=np.float32)
        o = None
        if order is not None:
            o = np.ascontiguousarray(np.concatenate(order), dtype=np.int32)
            o = o.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
        _check(load().sp_model_train(self.h, ctypes.c_void_p(int(x_ptr)), ctypes.c_void_p(int(y_ptr)), int(n),
                                     int(epochs), int(batch), float(lr), int(order_seed), o, _fptr(losses)),
               "sp_model_train")
        return losses

    def save(self, path):
        _check(load().sp_model_save(self.h, str(path).encode()), "sp_model_save")

    def close(self):
        if self.h:
            load().sp_model_destroy(self.h)
            self.h = None

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass


def _check(rc, what):
    if rc != SP_OK:
        raise SpError(rc, what)


class Grid:
    """Handle + the torch device tensors of each simulation + stream.

    A simulation's state is (phi, pic): phi complex64 (nz, ny, nx) and pic
    complex64 (nz, ny, nx, 2) holding (pi, c) per site, the library layout."""

    def __init__(self, params, states=None, stream=None, device="cuda"):
        import torch

        self.params = list(params)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        if states is None:
            states = []
            for p in self.params:
                shape = (p.n[2], p.n[1], p.n[0])
                states.append((torch.zeros(shape, dtype=torch.complex64, device=device),
                               torch.zeros(shape + (2,), dtype=torch.complex64, device=device)))
        self.states = states
        ptrs = [t.data_ptr() for st in states for t in st]
        rc, self.h = sp_grid_create(self.params, ptrs, self.stream.cuda_stream)
        _check(rc, "sp_grid_create")

    def plan(self, base_B=0, threads=0, order=SP_ORDER_STATIC, model_path=None, shape=None):
        """Region plan; shape (SP_SHAPE_SPLIT or SP_SHAPE_LATTICE) sets
        SP_OPT_REGION_SHAPE first when given."""
        if shape is not None:
            self.set_option(SP_OPT_REGION_SHAPE, shape)
        _check(sp_region_plan(self.h, base_B, threads, order, model_path), "sp_region_plan")

    def set_option(self, option, value):
        _check(load().sp_set_option(self.h, int(option), int(value)), "sp_set_option")

    def level(self, sim=0):
        out = ctypes.c_int64()
        _check(sp_read_surface(self.h, sim, SP_SURF_LEVEL, ctypes.addressof(out), 8, 0), "sp_read_surface")
        return int(out.value)

    def set_level(self, sim, level):
        v = ctypes.c_int64(int(level))
        _check(sp_write_surface(self.h, sim, SP_SURF_LEVEL, ctypes.addressof(v), 8, 0), "sp_write_surface")

    def evolve(self, n_steps, flags=0):
        _check(sp_evolve(self.h, n_steps, flags), "sp_evolve")

    def write_state(self, sim, phi, pi, c):
        buf = pack_state(phi, pi, c)
        _check(sp_write_surface(self.h, sim, SP_SURF_STATE, buf.ctypes.data, buf.nbytes, 0), "sp_write_surface")
        self.stream.synchronize()

    def read_state(self, sim):
        p = self.params[sim]
        shape = (p.n[2], p.n[1], p.n[0])
        out = np.empty(3 * int(np.prod(shape)), dtype=np.complex64)
        _check(sp_read_surface(self.h, sim, SP_SURF_STATE, out.ctypes.data, out.nbytes, 0), "sp_read_surface")
        return unpack_state(out, shape)

    def diag(self, sim=0) -> dict:
        d = sp_diag()
        _check(sp_read_surface(self.h, sim, SP_SURF_DIAG, ctypes.addressof(d), ctypes.sizeof(d), 0),
               "sp_read_surface")
        return {f: (list(getattr(d, f)) if f in ("pierced", "net_winding") else getattr(d, f))
                for f, _ in sp_diag._fields_}

    def winding(self, sim=0):
        p = self.params[sim]
        out = np.empty((3, p.n[2], p.n[1], p.n[0]), dtype=np.int8)
        _check(sp_read_surface(self.h, sim, SP_SURF_WINDING, out.ctypes.data, out.nbytes, 0), "sp_read_surface")
        return out

    def plan_info(self, sim=0) -> dict:
        d = sp_plan_info()
        _check(sp_read_surface(self.h, sim, SP_SURF_PLAN, ctypes.addressof(d), ctypes.sizeof(d), 0),
               "sp_read_surface")
        return {f: getattr(d, f) for f, _ in sp_plan_info._fields_}

    def timing(self):
        """(reset_ms, region_kernel_ms, remainder_ms) of the last SP_TIMING evolve."""
        out = np.zeros(3, dtype=np.float64)
        _check(sp_read_surface(self.h, 0, SP_SURF_TIMING, out.ctypes.data, out.nbytes, 0), "sp_read_surface")
        return tuple(out.tolist())

    def features(self, sim, n_regions):
        """Cost-model features [n_regions, 16] of the last SP_FEATURES call."""
        out = np.empty((n_regions, SP_MODEL_FEATURES), dtype=np.float32)
        _check(sp_read_surface(self.h, sim, SP_SURF_FEATURES, out.ctypes.data, out.nbytes, 0), "sp_read_surface")
        return out

    def trace(self, sim, n_regions):
        out = np.empty((n_regions, 2), dtype=np.uint64)
        _check(sp_read_surface(self.h, sim, SP_SURF_TRACE, out.ctypes.data, out.nbytes, 0), "sp_read_surface")
        return out

    def close(self):
        if self.h:
            sp_destroy(self.h)
            self.h = None

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass
