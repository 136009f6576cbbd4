"""The 4-cube lattice regions (paper Sec. 2, Figs. 2-5) on the CPU.

The table builder (csrc/lattice.cpp) checks its own tables; these tests pin
the geometry to closed forms and run the test-only scaffold
(cpu_exec/lattice_exec.cpp), which executes the regions of one call with the
kernel's data flow in several topological orders, checks every global read
and write against the dependency DAG, and must reproduce a whole-grid sweep
bit for bit.
"""
import ctypes

import numpy as np
import pytest

from paper_1011_4046_gb300 import inputs

I64 = ctypes.c_int64


def _stats(lx, s):
    out = (I64 * 12)()
    assert lx.lx_stats(s, out) == 0
    keys = ("updates", "slots", "foot", "imp_full", "imp_phi", "exp_phi", "exp_pc", "bytes_read", "bytes_written",
            "max_level", "pc_slots", "halo")
    return dict(zip(keys, list(out)))


def _level(lx, s, k):
    buf = (ctypes.c_int32 * (3 * 4000))()
    n = lx.lx_level(s, k, buf, 4000)
    assert n >= 0
    return np.array(buf[: 3 * n], dtype=np.int64).reshape(n, 3)


@pytest.mark.parametrize("s", [1, 2, 3, 4, 5, 6])
def test_region_volume_is_16_s4(lx, s):
    """A 4-cube of edge 4s in the forms f_i holds (4s)^4 lattice points of
    the form lattice, which has index 16 in Z^4 (the forms' matrix is a 4x4
    Hadamard matrix, determinant 16): 16 s^4 site-updates per region."""
    st = _stats(lx, s)
    assert st["updates"] == 16 * s ** 4


@pytest.mark.parametrize("s", [2, 3, 4, 5])
def test_levels_grow_as_tetrahedra_and_mirror(lx, s):
    """Below level s a region's cross-section is the tetrahedron
    sigma_i . r >= -k (no upper face yet), whose lattice-point count is
    (8k^3 + 12k^2 + 10k + 3) / 3 (1, 11, 45, 119, 249, ...); the region is
    symmetric under (k, r) -> (4s - 1 - k, -r); its first and last levels are
    the single centre cell (the bottom and top vertices)."""
    K = 4 * s
    sizes = [len(_level(lx, s, k)) for k in range(K)]
    for k in range(s):
        assert sizes[k] == (8 * k ** 3 + 12 * k ** 2 + 10 * k + 3) // 3
    assert sizes == sizes[::-1]
    assert sum(sizes) == 16 * s ** 4
    for k in (0, K - 1):
        assert _level(lx, s, k).tolist() == [[0, 0, 0]]
    for k in range(K):
        a = {tuple(r) for r in _level(lx, s, k).tolist()}
        b = {tuple(-v for v in r) for r in _level(lx, s, K - 1 - k).tolist()}
        assert a == b


def test_middle_level_is_an_octahedron(lx):
    """At the middle of the region (levels 2s - 1, 2s) the four slabs become
    |sigma . r| bounds for all eight sign patterns: the cross-section is an
    octahedron |x| + |y| + |z| <= 2s - 1, cut by one face of each pair."""
    s = 4
    cells = _level(lx, s, 2 * s)
    assert (np.abs(cells).sum(axis=1) <= 2 * s).all()
    assert (np.abs(cells).sum(axis=1) <= 2 * s - 1).sum() >= len(cells) * 0.6
    # the footprint's x extent is 4s - 1 cells
    assert cells[:, 0].min() == -(2 * s - 1) or cells[:, 0].max() == 2 * s - 1


def test_bytes_per_update_fall_with_region_size(lx):
    """Surface over volume (paper Sec. 3): this design's bytes per site-update
    fall roughly as 1/s; at s = 4 (16 levels, 4096 site-updates, the volume of
    a base-16 split-tiling region) a region moves 14.7 B per site-update, and
    every footprint cell enters once (one full import) and leaves once (one
    (pi, c) export)."""
    prev = None
    for s in (2, 3, 4, 5, 6):
        st = _stats(lx, s)
        assert st["imp_full"] == st["foot"] == st["exp_pc"]
        assert st["bytes_read"] == 24 * st["imp_full"] + 8 * st["imp_phi"]
        assert st["bytes_written"] == 8 * st["exp_phi"] + 16 * st["exp_pc"]
        b = (st["bytes_read"] + st["bytes_written"]) / st["updates"]
        if prev is not None:
            assert b < prev
        prev = b
    st = _stats(lx, 4)
    assert abs((st["bytes_read"] + st["bytes_written"]) / st["updates"] - 14.69) < 0.01
    assert st["foot"] == 847 and st["foot"] + st["halo"] == 1225 and st["max_level"] == 659


@pytest.mark.parametrize("s", [2, 3, 4, 5, 6])
def test_bank_layout_pads_little(lx, s):
    """The shared-memory layout that puts every slot on its bank residue
    (x + a y + b z mod 16) pads the compact layout by at most 25 %, and by at
    most 5 % at the sizes the kernel runs by default (s = 4, 6)."""
    st = _stats(lx, s)
    compact_phi, compact_pc = st["foot"] + st["halo"], st["foot"]
    assert compact_phi <= st["slots"] <= 1.25 * compact_phi
    assert compact_pc <= st["pc_slots"] <= 1.25 * compact_pc
    if s in (4, 6):
        assert st["slots"] <= 1.05 * compact_phi and st["pc_slots"] <= 1.05 * compact_pc


def _coef_table(levels, nu, dt, lam, tau0, tau_ref):
    out = np.zeros((levels, 4), dtype=np.float32)
    for n in range(levels):
        tau = tau0 + n * dt
        a = (tau / tau_ref) ** nu
        d = nu * dt / tau
        out[n] = ((1 - d) / (1 + d), dt / (1 + d), a * a * lam, 0.0)
    return out


def _state(n, seed):
    phi, _, c = inputs.initial_state(n, seed, "gaussian")
    pi = inputs.gaussian_field(n, seed + 100, sigma=0.2)
    pc = np.stack([pi.real, pi.imag, c.real, c.imag], axis=-1).astype(np.float32)
    return np.ascontiguousarray(phi, dtype=np.complex64), np.ascontiguousarray(pc)


def _run(lx, s, n, steps, mode, order_seed, phi0, pc0, coef):
    fp = ctypes.POINTER(ctypes.c_float)
    f, p = phi0.copy(), pc0.copy()
    msg = ctypes.create_string_buffer(256)
    st = (I64 * 6)()
    rc = lx.lx_run(s, *n, steps, mode, order_seed, coef.ctypes.data_as(fp), 0.25, 1.0, 1.0,
                   f.view(np.float32).ctypes.data_as(fp), p.ctypes.data_as(fp), msg, 256, st)
    assert rc == 0, msg.value.decode()
    return f, p, list(st)


def _sweep(lx, n, steps, phi0, pc0, coef):
    fp = ctypes.POINTER(ctypes.c_float)
    f, p = phi0.copy(), pc0.copy()
    lx.lx_sweep(*n, steps, coef.ctypes.data_as(fp), 0.25, 1.0, 1.0, f.view(np.float32).ctypes.data_as(fp),
                p.ctypes.data_as(fp))
    return f, p


@pytest.mark.parametrize("s,n,steps", [
    (1, (4, 4, 4), 7),          # one region per period (M = 1), odd step count
    (1, (8, 4, 12), 9),
    (2, (8, 8, 8), 16),         # M = 1: four regions per layer
    (2, (16, 8, 24), 21),       # anisotropic, ragged top
    (2, (16, 16, 16), 1),       # a single level: every region cut at both ends
    (3, (12, 24, 12), 14),
    (4, (16, 16, 16), 19),
    (4, (32, 16, 16), 40),
])
def test_lattice_executor_bit_exact_and_race_free(lx, s, n, steps):
    """Ticket order, random ready orders and last-ready-first: every order
    passes the race check and equals the sweep bit for bit (phi, pi, c)."""
    phi0, pc0 = _state(n, 7 + s)
    coef = _coef_table(steps, 2.0, 0.25, 2.0, 10.0, 10.0 + steps * 0.25)
    ref_f, ref_p = _sweep(lx, n, steps, phi0, pc0, coef)
    assert np.all(np.isfinite(ref_f))
    for mode, seed in ((0, 0), (1, 3), (1, 4), (2, 0)):
        f, p, st = _run(lx, s, n, steps, mode, seed, phi0, pc0, coef)
        assert np.array_equal(f.view(np.uint32), ref_f.view(np.uint32)), f"mode {mode}"
        assert np.array_equal(p.view(np.uint32), ref_p.view(np.uint32)), f"mode {mode}"
        M = [v // (4 * s) for v in n]
        assert st[0] == ((steps - 1) // s + 4) * 4 * M[0] * M[1] * M[2]
        assert st[1] > 0 and st[2] > 0


def test_lattice_executor_counts_each_region_once_per_layer(lx):
    """A layer of a grid of sides 4 s M_d holds 4 M_x M_y M_z regions, and a
    call of T levels meets (T - 1) // s + 4 layers (three cut by its first
    level)."""
    s, n, steps = 2, (16, 24, 8), 12
    phi0, pc0 = _state(n, 3)
    coef = _coef_table(steps, 0.0, 0.25, 2.0, 1.0, 1.0)
    _, _, st = _run(lx, s, n, steps, 0, 0, phi0, pc0, coef)
    assert st[0] == (11 // 2 + 4) * 4 * 2 * 3 * 1


@pytest.mark.parametrize("plant,expect", [
    (1, ("a write may overtake a read", "import of phi sees level", "reads a phi slot")),
    (2, ("a read not preceded by its writer", "a write may overtake a read", "import of")),
])
def test_race_check_catches_planted_mistakes(lx, plant, expect):
    """The checks are not vacuous: with one phi buffer for both level
    parities a region overwrites values its neighbours still read, and
    without the edge n - e_1 -> n a region reads faces its DAG does not
    order before it; both are reported (in ticket order the dynamic tags may
    not see the first, the DAG check does)."""
    s, n, steps = 2, (8, 8, 16), 12
    phi0, pc0 = _state(n, 5)
    coef = _coef_table(steps, 0.0, 0.25, 2.0, 1.0, 1.0)
    fp = ctypes.POINTER(ctypes.c_float)
    lx.lx_plant(plant)
    try:
        for mode, seed in ((0, 0), (1, 9)):
            f, p = phi0.copy(), pc0.copy()
            msg = ctypes.create_string_buffer(256)
            rc = lx.lx_run(s, *n, steps, mode, seed, coef.ctypes.data_as(fp), 0.25, 1.0, 1.0,
                           f.view(np.float32).ctypes.data_as(fp), p.ctypes.data_as(fp), msg, 256, None)
            assert rc == -1
            assert any(e in msg.value.decode() for e in expect), msg.value.decode()
    finally:
        lx.lx_plant(0)


@pytest.mark.parametrize("s,n,steps", [(2, (16, 16, 16), 12), (4, (16, 16, 16), 12)])
def test_pair_imports_need_the_pair_bit(lx, s, n, steps):
    """A phi import may copy its aligned 16-byte site pair into the aligned
    slot pair only where the table builder set the pair bit (the pair's other
    slot holds the row's neighbour, or nothing imported into that buffer):
    copying the pair for every import puts another site's value into a slot
    another import fills, and the executor reports it."""
    phi0, pc0 = _state(n, 6)
    coef = _coef_table(steps, 0.0, 0.25, 2.0, 1.0, 1.0)
    fp = ctypes.POINTER(ctypes.c_float)
    f, p = phi0.copy(), pc0.copy()
    msg = ctypes.create_string_buffer(256)
    assert lx.lx_run(s, *n, steps, 0, 0, coef.ctypes.data_as(fp), 0.25, 1.0, 1.0, f.view(np.float32).ctypes.data_as(fp),
                     p.ctypes.data_as(fp), msg, 256, None) == 0, msg.value.decode()
    lx.lx_plant(3)
    try:
        f, p = phi0.copy(), pc0.copy()
        rc = lx.lx_run(s, *n, steps, 0, 0, coef.ctypes.data_as(fp), 0.25, 1.0, 1.0,
                       f.view(np.float32).ctypes.data_as(fp), p.ctypes.data_as(fp), msg, 256, None)
    finally:
        lx.lx_plant(0)
    assert rc == -1
    assert any(e in msg.value.decode() for e in ("pair copy overwrites", "reads a phi slot")), msg.value.decode()


def test_cut_regions_load_only_their_levels_imports(lx):
    """All of a region's imports are final at its start only for the levels
    it computes: a region cut by the call's first or last level that loaded
    the imports of its other levels would read values of levels not yet (or
    no longer) in the state arrays, and the executor reports it."""
    s, n, steps = 2, (8, 8, 16), 12
    phi0, pc0 = _state(n, 8)
    coef = _coef_table(steps, 0.0, 0.25, 2.0, 1.0, 1.0)
    fp = ctypes.POINTER(ctypes.c_float)
    msg = ctypes.create_string_buffer(256)
    lx.lx_plant(4)
    try:
        f, p = phi0.copy(), pc0.copy()
        rc = lx.lx_run(s, *n, steps, 0, 0, coef.ctypes.data_as(fp), 0.25, 1.0, 1.0,
                       f.view(np.float32).ctypes.data_as(fp), p.ctypes.data_as(fp), msg, 256, None)
    finally:
        lx.lx_plant(0)
    assert rc == -1 and "sees" in msg.value.decode(), msg.value.decode()


def test_layer_numbers_of_successive_calls_never_reuse_flag_values(lx):
    """Done flags are never cleared: a call waits for 'flag >= its layer
    number - 1'.  For any sequence of calls (long ones followed by short
    ones included), every layer number a call waits for exceeds every value
    an earlier call wrote, and the first call waits only for values above
    the flags' initial 0."""
    rng = np.random.default_rng(3)
    for _ in range(50):
        n = int(rng.integers(1, 12))
        s = int(rng.integers(1, 7))
        steps = rng.integers(1, 200, size=n)
        layers = np.array([(int(t) - 1) // s + 4 for t in steps], dtype=np.int32)
        first = np.zeros(n, dtype=np.int32)
        lx.lx_epochs(layers.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), n,
                     first.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
        written_max = 0
        for i in range(n):
            waits_min = first[i]  # layer 1 of the call waits for its layer 0: number first
            assert waits_min > written_max
            written_max = max(written_max, first[i] + layers[i] - 1)


@pytest.mark.parametrize("s,n,steps", [(2, (16, 8, 24), 21), (4, (16, 16, 16), 19), (4, (32, 16, 16), 64),
                                       (3, (12, 24, 12), 1)])
def test_call_bytes_match_the_executed_accesses(lx, s, n, steps):
    """The library's per-call byte count (sp_lattice_call_bytes, one region
    column) times the regions per layer equals the bytes the scaffold's
    execution actually moved to and from the state arrays (its access log);
    its update count is the grid's sites times the call's levels."""
    from paper_1011_4046_gb300 import sp

    phi0, pc0 = _state(n, 4)
    coef = _coef_table(steps, 0.0, 0.25, 2.0, 1.0, 1.0)
    _, _, st = _run(lx, s, n, steps, 0, 0, phi0, pc0, coef)
    per_layer = 4 * np.prod([v // (4 * s) for v in n])
    upd, rd, wr = sp.sp_lattice_call_bytes(4 * s, steps)
    assert upd * per_layer == np.prod(n) * steps
    assert rd * per_layer == st[4]
    assert wr * per_layer == st[5]


def test_call_bytes_approach_the_region_figure():
    """Long calls converge to the full region's 14.69 B per site-update at
    s = 4; the cut layers at a call's two ends add a share that shrinks as
    1 / steps."""
    from paper_1011_4046_gb300 import sp

    prev = None
    for steps in (16, 64, 256, 2048):
        upd, rd, wr = sp.sp_lattice_call_bytes(16, steps)
        b = (rd + wr) / upd
        assert b > 14.69
        if prev is not None:
            assert b < prev
        prev = b
    assert prev < 14.69 * 1.02
