"""Region planner (host logic, CPU only).

The planner is checked on concrete periodic grids by a test-only C++
scaffold (tests/cpu_exec/region_exec.cpp) that uses the planner's tables
exactly as the GPU kernel does:

* exact cover -- every (site, level) is computed by exactly one region;
* the DAG the kernel releases is acyclic and its counters equal the
  number of releasing predecessors;
* hazards -- every base or mailbox read is produced by a predecessor, and
  nothing overwrites a value (band tops in the main arrays, the mailboxes
  as a ring of two band slots or as one slot for every band) before every
  reader of it is done;
* the regions executed one at a time in random topological orders with the
  FP32 site update reproduce a whole-grid FP32 sweep bit for bit.
"""
import ctypes

import numpy as np
import pytest

from paper_1011_4046_gb300 import inputs

@pytest.mark.parametrize("slots", [2, 1])
@pytest.mark.parametrize("B,n,bands", [(8, (16, 16, 16), 4), (8, (16, 24, 32), 4), (4, (8, 8, 12), 5),
                                       (6, (12, 18, 12), 4), (16, (32, 32, 32), 3)])
def test_tiling_dag_and_hazards(rx, B, n, bands, slots):
    msg = ctypes.create_string_buffer(256)
    ok = rx.rx_check(B, *n, bands, msg, 256, slots)
    assert ok == 1, msg.value.decode()


@pytest.mark.parametrize("B", [4, 6, 8, 16])
def test_reuse_edges_reduce_to_the_inverted_pyramids(rx, B):
    """Of the mailbox-reuse edges (every same-band edge mirrored one band
    later), the planner keeps those the rest of the DAG does not imply.  From
    base 6 on that is eight per position, all from the inverted pyramid of
    band b to pyramids of band b+1: every writer of band b+1 comes after its
    pyramids, and the inverted pyramid after every reader of band b.  At base
    4 the wedges have no same-band predecessors, so the pyramids order
    nothing and all 26 mirrored edges (all into the inverted pyramid's
    mailbox) stay."""
    n_succ, to_pyr, preds = ((ctypes.c_int * 8)() for _ in range(3))
    assert rx.rx_reuse(B, n_succ, to_pyr, preds) == 1
    assert list(n_succ)[:7] == [0] * 7
    if B == 4:
        assert n_succ[7] == 26 and sum(preds) == 26
    else:
        assert n_succ[7] == 8 and to_pyr[7] == 8
        assert list(preds) == [8, 0, 0, 0, 0, 0, 0, 0]


@pytest.mark.parametrize("B,n", [(8, (16, 16, 16)), (4, (8, 8, 12)), (16, (32, 32, 32))])
def test_one_slot_needs_the_reuse_edges(rx, B, n):
    """With one mailbox slot but without the reuse edges, some writer of the
    next band is not ordered after the reader of the mailbox it overwrites,
    and the hazard check must say so (slots = -1 asks for exactly that DAG)."""
    msg = ctypes.create_string_buffer(256)
    assert rx.rx_check(B, *n, 3, msg, 256, -1) == 0
    assert "reused before its reader finished" in msg.value.decode()


def test_traffic_counts_match_the_brute_force_figures(rx):
    """Read bytes per site-update reproduce the independent brute-force count
    (25.2 / 13.8 / 7.2 B at B = 8 / 16 / 32).  Writes are higher than a
    write-once design because a face cell is written into each consumer's
    mailbox."""
    got = {}
    for B in (8, 16, 32):
        r, w, u = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        total = rx.rx_bytes_per_update(B, ctypes.byref(r), ctypes.byref(w), ctypes.byref(u))
        assert u.value == (B // 2) * B ** 3  # every cell of one period, every level
        got[B] = (r.value / u.value, w.value / u.value, total)
    assert abs(got[8][0] - 25.2) < 0.05 and abs(got[16][0] - 13.8) < 0.05 and abs(got[32][0] - 7.2) < 0.05
    for B in got:
        assert abs(got[B][0] + got[B][1] - got[B][2]) < 1e-9
    assert got[16][2] < got[8][2] and got[32][2] < got[16][2]


def _coef_table(levels, nu, dt, lam, tau0, tau_ref):
    out = np.zeros((levels, 4), dtype=np.float32)
    for n in range(levels):
        tau = tau0 + n * dt
        a = (tau / tau_ref) ** nu
        d = nu * dt / tau
        out[n] = ((1 - d) / (1 + d), dt / (1 + d), a * a * lam, 0.0)
    return out


@pytest.mark.parametrize("B,n,steps,seed", [(8, (16, 16, 16), 16, 1), (4, (8, 12, 16), 10, 2),
                                            (6, (12, 12, 18), 9, 3), (16, (32, 32, 32), 16, 4)])
def test_region_executor_bit_exact_vs_sweep(rx, B, n, steps, seed):
    phi0, pi0, c0 = inputs.initial_state(n, seed, "gaussian")
    pi0 = inputs.gaussian_field(n, seed + 100, sigma=0.2)
    coef = _coef_table(steps, 2.0, 0.25, 2.0, 10.0, 10.0 + steps * 0.25)
    fp = ctypes.POINTER(ctypes.c_float)

    def run(mode, order_seed, slots):
        f, v, c = (np.ascontiguousarray(a, dtype=np.complex64).copy() for a in (phi0, pi0, c0))
        msg = ctypes.create_string_buffer(256)
        ok = rx.rx_run(B, *n, steps, mode, order_seed, coef.ctypes.data_as(fp), 0.25, 1.0, 1.0,
                       f.view(np.float32).ctypes.data_as(fp), v.view(np.float32).ctypes.data_as(fp),
                       c.view(np.float32).ctypes.data_as(fp), msg, 256, slots)
        assert ok == 1, msg.value.decode()
        return f, v, c

    ref = run(0, 0, 2)
    assert np.all(np.isfinite(ref[0]))
    for order_seed, slots in ((11, 2), (12, 2), (13, 1), (14, 1)):
        got = run(1, order_seed, slots)
        for a, b in zip(ref, got):
            assert np.array_equal(a.view(np.uint32), b.view(np.uint32))


@pytest.mark.parametrize("B,seeds", [(4, 7), (6, 1), (8, 1), (16, 1)])
def test_predecessor_free_types_lead(rx, B, seeds):
    """The band-0 regions that are ready at the start are those of the leading
    region types (the GPU queue reset seeds the first Jtot * m region ids).  At
    base 4 every type but the inverted pyramid computes a single level and
    imports nothing, so seven types are seeds; from base 6 on only the
    pyramid is."""
    assert rx.rx_seed_types(B) == seeds


# ------------------------------------------------ reduced region DAG (study)
def _reduced(rx, B, on):
    by_src, kind = (ctypes.c_int * 8)(), (ctypes.c_int * 3)()
    n = rx.rx_reduced_dag(B, 1 if on else 0, by_src, kind)
    return n, list(by_src), list(kind)


@pytest.mark.parametrize("B", [8, 16])
def test_reduced_dag_keeps_a_third_of_the_edges(rx, B):
    """Transitive reduction of the release pattern with one mailbox slot: of
    the 56 same-band, 2 x 27 next-band and 8 mailbox-reuse edges per position,
    24 same-band and the 8 reuse edges remain; every next-band edge is implied
    through the reuse edges.  A pyramid would release 6 successors instead of
    26, an inverted pyramid 8 instead of 35."""
    n, by_src, kind = _reduced(rx, B, False)
    assert n == 32 and kind == [24, 0, 8]
    assert by_src[0] == 6 and by_src[7] == 8


@pytest.mark.parametrize("B,n,bands", [(8, (16, 16, 16), 4), (8, (16, 24, 32), 4), (4, (8, 8, 12), 5),
                                       (6, (12, 18, 12), 4), (16, (32, 32, 32), 3)])
def test_reduced_dag_is_hazard_free(rx, B, n, bands):
    """The reduced pattern, released and counted on concrete periodic grids,
    passes the same cover, counter and hazard checks as the full one."""
    msg = ctypes.create_string_buffer(256)
    try:
        _reduced(rx, B, True)
        ok = rx.rx_check(B, *n, bands, msg, 256, 1)
    finally:
        _reduced(rx, B, False)
    assert ok == 1, msg.value.decode()


@pytest.mark.parametrize("B,n,steps,seed", [(8, (16, 16, 16), 16, 21), (16, (32, 32, 32), 16, 22)])
def test_reduced_dag_runs_bit_exact(rx, B, n, steps, seed):
    """Regions executed in random topological orders of the reduced DAG give
    the whole-grid sweep bit for bit."""
    phi0, pi0, c0 = inputs.initial_state(n, seed, "gaussian")
    coef = _coef_table(steps, 2.0, 0.25, 2.0, 10.0, 10.0 + steps * 0.25)
    fp = ctypes.POINTER(ctypes.c_float)

    def run(mode, order_seed):
        f, v, c = (np.ascontiguousarray(a, dtype=np.complex64).copy() for a in (phi0, pi0, c0))
        msg = ctypes.create_string_buffer(256)
        ok = rx.rx_run(B, *n, steps, mode, order_seed, coef.ctypes.data_as(fp), 0.25, 1.0, 1.0,
                       f.view(np.float32).ctypes.data_as(fp), v.view(np.float32).ctypes.data_as(fp),
                       c.view(np.float32).ctypes.data_as(fp), msg, 256, 1)
        assert ok == 1, msg.value.decode()
        return f, v, c

    ref = run(0, 0)
    try:
        _reduced(rx, B, True)
        got = [run(1, s) for s in (31, 32)]
    finally:
        _reduced(rx, B, False)
    for g in got:
        for a, b in zip(ref, g):
            assert np.array_equal(a.view(np.uint32), b.view(np.uint32))


@pytest.mark.parametrize("B", [6, 8, 16])
def test_a_band_runs_in_the_papers_four_layers(rx, B):
    """Same-band edges only go from a region type to a strict superset of its
    inverted axes, so a band's regions fall into dependency layers by |S|;
    the longest chain of same-band dependencies has as many regions as the
    paper has active layers (tests/golden/layers.txt).  (At base 4 a wedge
    computes one level and imports nothing, so only the inverted pyramid
    waits on same-band regions: two layers.)"""
    import os

    golden = os.path.join(os.path.dirname(__file__), "golden", "layers.txt")
    layers = int(next(ln.split()[1] for ln in open(golden) if ln.startswith("layers_per_band")))
    buf = (ctypes.c_int * 64)()
    succ = {}
    for S in range(8):
        n = rx.rx_same_succ(B, S, buf, 64)
        assert 0 <= n <= 26
        succ[S] = set(buf[:n])
        for T in succ[S]:
            assert T & S == S and T != S  # strict superset of inverted axes
    longest = {}
    for S in sorted(range(8), key=lambda s: -bin(s).count("1")):
        longest[S] = 1 + max((longest[T] for T in succ[S]), default=0)
    assert max(longest.values()) == layers


@pytest.mark.parametrize("B,n,steps,seed", [(32, (64, 64, 64), 32, 5), (32, (64, 96, 64), 48, 6),
                                            (16, (32, 48, 32), 24, 7), (8, (16, 16, 24), 12, 8)])
def test_octant_executor_bit_exact_vs_sweep(rx, B, n, steps, seed):
    """The octant tables (a region split over a 2 x 2 x 2 cluster, one octant
    per CTA, inner faces exchanged every level) executed on the host exactly
    as the cluster kernel moves data -- octant mailboxes, mirrored octant
    coordinates, consumer octant and position from the export's flip mask --
    reproduce the whole-grid FP32 sweep bit for bit in random region orders,
    with a ring of two mailbox slots and with one slot.  Every buffer starts
    as NaN, so a cell the tables fail to deliver cannot go unnoticed."""
    phi0, pi0, c0 = inputs.initial_state(n, seed, "gaussian", sigma=0.3)
    pi0 = inputs.gaussian_field(n, seed + 100, sigma=0.2)
    coef = _coef_table(steps, 2.0, 0.25, 2.0, 10.0, 10.0 + steps * 0.25)
    fp = ctypes.POINTER(ctypes.c_float)

    def run(mode, order_seed, slots):
        f, v, c = (np.ascontiguousarray(a, dtype=np.complex64).copy() for a in (phi0, pi0, c0))
        msg = ctypes.create_string_buffer(256)
        ok = rx.rx_run(B, *n, steps, mode, order_seed, coef.ctypes.data_as(fp), 0.25, 1.0, 1.0,
                       f.view(np.float32).ctypes.data_as(fp), v.view(np.float32).ctypes.data_as(fp),
                       c.view(np.float32).ctypes.data_as(fp), msg, 256, slots)
        assert ok == 1, msg.value.decode()
        return f, v, c

    ref = run(0, 0, 2)
    assert np.all(np.isfinite(ref[0]))
    for order_seed, slots in ((21, 2), (22, 1)):
        got = run(2, order_seed, slots)
        for a, b, name in zip(ref, got, ("phi", "pi", "c")):
            assert np.array_equal(a.view(np.uint32), b.view(np.uint32)), \
                f"{name}: {np.count_nonzero(a.view(np.uint32) != b.view(np.uint32))} sites differ"
