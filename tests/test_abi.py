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
    p.precision = 1  # only SP_FP32_KAHAN is built
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
    # sp_plan_info: 4 int32, 4 int64, double, int64, 2 int32, 2 double, 2 int32
    assert ctypes.sizeof(sp.sp_plan_info) == 16 + 32 + 8 + 8 + 8 + 16 + 8


def test_model_entry_points_reject_bad_input_without_a_gpu(lib, tmp_path):
    out = ctypes.c_void_p()
    assert lib.sp_model_load(None, None, ctypes.byref(out)) == sp.SP_EINVAL
    bad = tmp_path / "not_a_model.bin"
    bad.write_bytes(b"NOTAMODEL" + bytes(64))
    assert lib.sp_model_load(str(bad).encode(), None, ctypes.byref(out)) == sp.SP_EINVAL and not out.value
    truncated = tmp_path / "truncated.bin"
    truncated.write_bytes(b"SPMLP001" + (5313).to_bytes(4, "little") + bytes(100))
    assert lib.sp_model_load(str(truncated).encode(), None, ctypes.byref(out)) == sp.SP_EINVAL
    assert lib.sp_model_destroy(None) == sp.SP_EINVAL
    assert lib.sp_model_predict(None, None, 0, None) == sp.SP_EINVAL
    assert lib.sp_model_train(None, None, None, 0, 1, 1, ctypes.c_float(1e-3), 0, None, None) == sp.SP_EINVAL


def test_options_and_levels_reject_null_handles(lib):
    assert lib.sp_set_option(None, sp.SP_OPT_WAIT_LIMIT_NS, 10 ** 9) == sp.SP_EINVAL
    v = ctypes.c_int64(3)
    assert lib.sp_write_surface(None, 0, sp.SP_SURF_LEVEL, ctypes.byref(v), 8, 0) == sp.SP_EINVAL


def _header_struct_fields(text, name):
    """Field names, in order, of `typedef struct { ... } name;` in the header."""
    import re
    m = re.search(r"typedef struct \{([^{}]*)\}\s*" + name + r"\s*;", text)
    assert m, name
    body = re.sub(r"/\*.*?\*/", "", m.group(1), flags=re.S)
    fields = []
    for decl in body.split(";"):
        decl = decl.strip()
        if not decl:
            continue
        _, names = decl.split(None, 1)
        for n in names.split(","):
            fields.append(re.sub(r"\[.*\]", "", n).strip())
    return fields


@pytest.mark.parametrize("name", ["sp_params", "sp_diag", "sp_plan_info"])
def test_binding_structs_mirror_the_header(name):
    """The ctypes mirrors of the ABI structs list the header's fields in the
    header's order (a field added on one side only would shift the rest)."""
    text = open(sp.HEADER).read()
    renamed = {"lambda": "lam"}  # a Python keyword
    want = [renamed.get(f, f) for f in _header_struct_fields(text, name)]
    assert [f for f, _ in getattr(sp, name)._fields_] == want


def test_header_constants_match_the_binding():
    text = open(sp.HEADER).read()
    import re
    for name in ("SP_AUTOTUNE", "SP_FEATURES", "SP_SURF_FEATURES", "SP_SURF_LEVEL", "SP_OPT_WAIT_LIMIT_NS",
                 "SP_OPT_FAULT_DROP_RELEASE", "SP_OPT_GRAPHS", "SP_OPT_MAILBOX_SLOTS", "SP_OPT_REGION_SHAPE",
                 "SP_SHAPE_SPLIT", "SP_SHAPE_LATTICE", "SP_MODEL_PARAMS",
                 "SP_MODEL_FEATURES",
                 "SP_ORDER_STATIC", "SP_ORDER_LEARNED", "SP_TIMING", "SP_TRACE", "SP_FP32_KAHAN",
                 "SP_NOALLOC_MAX_SITES", "SP_NOALLOC_MAX_STEPS"):
        m = re.search(r"#define\s+" + name + r"\s+\(?(-?\d+)u?\)?", text)
        assert m, name
        assert int(m.group(1)) == getattr(sp, name), name


def test_noalloc_rejects_bad_sizes_before_any_cuda_call(lib):
    """sp_sweep_noalloc bounds every side before it forms the site count: a
    grid whose product would wrap a 64-bit integer (2^30 x 2^18 x 2^16) is
    rejected, as are sides below 4 and a non-zero precision; sizes beyond its
    fixed scratch give SP_ESCRATCH.  All return before any CUDA call (no GPU
    here); the pointers are never dereferenced."""
    fake = 1 << 20  # 16-byte aligned stand-ins
    for n in ((1 << 30, 1 << 18, 1 << 16), (1 << 15, 8, 8), (2, 16, 16)):
        p = sp.make_params(n, nu=0.0)
        assert sp.sp_sweep_noalloc(p, fake, fake, 0, 4, 0) == sp.SP_EINVAL, n
    p = sp.make_params(16, nu=0.0)
    p.precision = 1
    assert sp.sp_sweep_noalloc(p, fake, fake, 0, 4, 0) == sp.SP_EINVAL
    p = sp.make_params((16384, 16384, 4), nu=0.0)  # sides in range, too many sites
    assert sp.sp_sweep_noalloc(p, fake, fake, 0, 4, 0) == sp.SP_ESCRATCH
    p = sp.make_params(16, nu=0.0)
    assert sp.sp_sweep_noalloc(p, fake, fake, 0, sp.SP_NOALLOC_MAX_STEPS + 1, 0) == sp.SP_ESCRATCH
    assert sp.sp_sweep_noalloc(p, fake + 4, fake, 0, 4, 0) == sp.SP_EINVAL  # misaligned phi
