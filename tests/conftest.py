import ctypes
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: longer CPU test")


def gpu_available() -> bool:
    try:
        import torch

        return torch.cuda.is_available()
    except Exception:  # pragma: no cover
        return False


@pytest.fixture(scope="session")
def oracle_mod():
    import oracle

    oracle.build()
    return oracle


@pytest.fixture(scope="session")
def rx():
    """The test-only CPU scaffold (cpu_exec/region_exec.cpp) linked with the
    region planner: the planner's tables, checked and executed on the host."""
    here = os.path.dirname(os.path.abspath(__file__))
    csrc = os.path.join(ROOT, "paper_1011_4046_gb300", "csrc")
    out_dir = os.path.join(here, "cpu_exec", "_build")
    os.makedirs(out_dir, exist_ok=True)
    lib = os.path.join(out_dir, "librx.so")
    srcs = [os.path.join(here, "cpu_exec", "region_exec.cpp"), os.path.join(csrc, "planner.cpp")]
    deps = srcs + [os.path.join(csrc, "planner.h"), os.path.join(csrc, "sp_update.h")]
    if not os.path.exists(lib) or any(os.path.getmtime(s) > os.path.getmtime(lib) for s in deps):
        tmp = lib + f".tmp{os.getpid()}"
        subprocess.run(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-ffp-contract=off", f"-I{csrc}", *srcs,
                        "-o", tmp], check=True)
        os.replace(tmp, lib)
    L = ctypes.CDLL(lib)
    L.rx_check.argtypes = [ctypes.c_int] * 5 + [ctypes.c_char_p, ctypes.c_int, ctypes.c_int]
    fp = ctypes.POINTER(ctypes.c_float)
    L.rx_run.argtypes = [ctypes.c_int] * 6 + [ctypes.c_uint64, fp, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                              fp, fp, fp, ctypes.c_char_p, ctypes.c_int, ctypes.c_int]
    L.rx_bytes_per_update.argtypes = [ctypes.c_int] + [ctypes.POINTER(ctypes.c_int64)] * 3
    L.rx_bytes_per_update.restype = ctypes.c_double
    L.rx_reuse.argtypes = [ctypes.c_int] + [ctypes.POINTER(ctypes.c_int)] * 3
    L.rx_same_succ.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.c_int]
    L.rx_reduced_dag.argtypes = [ctypes.c_int, ctypes.c_int] + [ctypes.POINTER(ctypes.c_int)] * 2
    L.rx_active_box.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int32)]
    return L


@pytest.fixture(scope="session")
def lx():
    """The test-only CPU scaffold of the 4-cube lattice regions
    (cpu_exec/lattice_exec.cpp) linked with their table builder."""
    here = os.path.dirname(os.path.abspath(__file__))
    csrc = os.path.join(ROOT, "paper_1011_4046_gb300", "csrc")
    out_dir = os.path.join(here, "cpu_exec", "_build")
    os.makedirs(out_dir, exist_ok=True)
    lib = os.path.join(out_dir, "liblx.so")
    srcs = [os.path.join(here, "cpu_exec", "lattice_exec.cpp"), os.path.join(csrc, "lattice.cpp")]
    deps = srcs + [os.path.join(csrc, "lattice.h"), os.path.join(csrc, "sp_update.h")]
    if not os.path.exists(lib) or any(os.path.getmtime(s) > os.path.getmtime(lib) for s in deps):
        tmp = lib + f".tmp{os.getpid()}"
        subprocess.run(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-ffp-contract=off", f"-I{csrc}", *srcs,
                        "-o", tmp], check=True)
        os.replace(tmp, lib)
    L = ctypes.CDLL(lib)
    fp = ctypes.POINTER(ctypes.c_float)
    i64p = ctypes.POINTER(ctypes.c_int64)
    L.lx_sweep.argtypes = [ctypes.c_int] * 4 + [fp, ctypes.c_float, ctypes.c_float, ctypes.c_float, fp, fp]
    L.lx_run.argtypes = [ctypes.c_int] * 6 + [ctypes.c_uint64, fp, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                              fp, fp, ctypes.c_char_p, ctypes.c_int, i64p]
    L.lx_stats.argtypes = [ctypes.c_int, i64p]
    L.lx_level.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int32), ctypes.c_int]
    L.lx_plant.argtypes = [ctypes.c_int]
    L.lx_epochs.argtypes = [ctypes.POINTER(ctypes.c_int), ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
    return L
