"""The C-ABI library: it builds for sm_103a, loads without a GPU, exports every
entry point include/sp.h declares, and rejects bad arguments before touching
the device.  No compute call is made here."""
import ctypes

import pytest

from paper_1011_4046_gb300 import build, sp


@pytest.fixture(scope="module")
def lib():
    build.build()
    return sp.load()


def test_every_declared_symbol_is_exported(lib):
    names = sp.declared_entry_points()
    assert set(names) >= {"sp_grid_create", "sp_region_plan", "sp_evolve", "sp_read_surface", "sp_destroy",
                          "sp_write_surface", "sp_strerror"}
    for n in names:
        assert hasattr(lib, n), n


def test_strerror_names_every_code(lib):
    codes = [sp.SP_OK, sp.SP_EINVAL, sp.SP_ENOMEM, sp.SP_ECUDA, sp.SP_EUNSTABLE, sp.SP_ETIMEOUT,
             sp.SP_ENONFINITE, sp.SP_EFAULT_INJECTED, sp.SP_ENOTPLANNED]
    msgs = [sp.sp_strerror(c) for c in codes]
    assert len(set(msgs)) == len(msgs) and "unknown" not in " ".join(msgs)
    assert sp.sp_strerror(-999) == "unknown error"


def test_create_validates_before_any_cuda_call(lib):
    bad = [sp.make_params(16, dt=-1.0), sp.make_params(16, dx=0.0), sp.make_params((2, 16, 16)),
           sp.make_params(16, tau0=0.0), sp.make_params(16, lam=-1.0)]
    for p in bad:
        rc, h = sp.sp_grid_create([p], None, 0)
        assert rc == sp.SP_EINVAL and not h.value
    rc, h = sp.sp_grid_create([], None, 0)
    assert rc == sp.SP_EINVAL
    p = sp.make_params(16)
    p.reserved = 1
    rc, h = sp.sp_grid_create([p], None, 0)
    assert rc == sp.SP_EINVAL


def test_null_handles_are_rejected(lib):
    assert lib.sp_evolve(None, 4, 0) == sp.SP_EINVAL
    assert lib.sp_region_plan(None, 8, 0, 0, None) == sp.SP_EINVAL
    assert lib.sp_destroy(None) == sp.SP_EINVAL
    buf = ctypes.create_string_buffer(64)
    assert lib.sp_read_surface(None, 0, sp.SP_SURF_DIAG, buf, 64, 0) == sp.SP_EINVAL


def test_struct_layouts_match_the_header(lib):
    # sp_params: 3 int32 + 7 double + 2 int32 with natural alignment
    assert ctypes.sizeof(sp.sp_params) == 12 + 4 + 7 * 8 + 8
    assert ctypes.sizeof(sp.sp_diag) == 8 + 6 * 8 + 3 * 8 + 8 + 3 * 8 + 8
