"""The 4-cube lattice regions (paper Sec. 2, Figs. 2-5) on the GPU.

Bars: the lattice path equals the monolithic sweep bit for bit (phi, pi, c)
for every lattice size s = 1..6, on isotropic and anisotropic grids, for step
counts below one region's height, odd and even, and across consecutive
calls; several simulations (same and different sizes) in one call; the
FP64-oracle bars of accuracy_bars.py on a 128^3 matter-era run; a dropped
done report ends the call with SP_ETIMEOUT and leaves the grid usable.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1011_4046_gb300 import inputs, sp  # noqa: E402

from accuracy_bars import check_run, format_report  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    sp.load()


def params_for(n, nu, steps):
    tau0 = 10.0 if nu > 0 else 1.0
    return sp.make_params(n, dx=1.0, dt=0.25, lam=2.0, eta=1.0, nu=nu, tau0=tau0, tau_ref=tau0 + steps * 0.25)


def run(p, st, calls, base_B=16, threads=0, mono=False, every=None):
    """calls: list of step counts, one sp_evolve each."""
    g = sp.Grid([p])
    try:
        g.write_state(0, *st)
        if not mono:
            g.plan(base_B=base_B, threads=threads, shape=sp.SP_SHAPE_LATTICE)
        out = {}
        lvl = 0
        for n in calls:
            g.evolve(n, sp.SP_MONOLITHIC if mono else 0)
            lvl += n
            if every:
                out[lvl] = g.read_state(0)
        info = None if mono else g.plan_info(0)
        return (out if every else g.read_state(0)), info
    finally:
        g.close()


def assert_bit_equal(x, y, tag=""):
    for a, b, name in zip(x, y, ("phi", "pi", "c")):
        d = np.count_nonzero(np.ascontiguousarray(a).view(np.uint32) != np.ascontiguousarray(b).view(np.uint32))
        assert d == 0, f"{tag}{name}: {d} sites differ"


@pytest.mark.parametrize("B,n,calls,nu", [
    (16, (64, 64, 64), [32], 2.0),          # s = 4: two region heights
    (16, (64, 48, 32), [21, 11], 1.0),      # anisotropic, odd calls, two calls
    (16, (32, 32, 32), [1, 2, 3], 0.0),     # fewer steps than one level band of regions
    (8, (32, 40, 24), [17], 2.0),           # s = 2
    (4, (16, 12, 20), [9, 6], 0.0),         # s = 1: 16 site-updates per region
    (12, (48, 36, 24), [25], 2.0),          # s = 3
    (20, (40, 60, 40), [33], 1.0),          # s = 5
    (24, (48, 48, 24), [50], 2.0),          # s = 6
])
def test_lattice_bit_exact_vs_monolithic(B, n, calls, nu):
    steps = sum(calls)
    p = params_for(n, nu, steps)
    st = inputs.initial_state(n, 11, "gaussian" if nu == 0 else "phase", sigma=0.3)
    reg, info = run(p, st, calls, base_B=B)
    assert info["region_shape"] == sp.SP_SHAPE_LATTICE and info["base_B"] == B and info["mailbox_slots"] == 0
    assert info["updates_per_band"] == info["regions_per_band"] * 16 * (B // 4) ** 4
    assert np.all(np.isfinite(reg[0]))
    assert_bit_equal(reg, run(p, st, calls, mono=True)[0])


@pytest.mark.parametrize("B,threads", [(16, 64), (16, 128), (16, 256), (16, 512), (8, 64), (12, 64), (20, 192)])
def test_lattice_worker_counts(B, threads):
    n, steps = ((48, 48, 48) if 48 % B == 0 else (40, 60, 40)), 24
    p = params_for(n, 2.0, steps)
    st = inputs.initial_state(n, 5, "phase")
    reg, info = run(p, st, [steps], base_B=B, threads=threads)
    assert info["threads"] == threads
    assert_bit_equal(reg, run(p, st, [steps], mono=True)[0])


def test_lattice_worker_count_not_offered_is_refused():
    """Worker counts without a kernel instance (here 96) are refused by the
    plan instead of running."""
    p = params_for((32, 32, 32), 0.0, 8)
    g = sp.Grid([p])
    try:
        g.set_option(sp.SP_OPT_REGION_SHAPE, sp.SP_SHAPE_LATTICE)
        assert sp.sp_region_plan(g.h, 16, 96, sp.SP_ORDER_STATIC, None) == sp.SP_EINVAL
    finally:
        g.close()


def test_lattice_several_simulations_in_one_call():
    """Simulations of sizes 16, 16, 8 and 4 in one plan (three launches,
    the two base-16 simulations sharing one), traced: each equals its own
    sweep, and every region of the call has a trace entry."""
    specs = [((32, 32, 32), 2.0, 16), ((48, 16, 32), 1.0, 16), ((24, 16, 32), 0.0, 8), ((24, 36, 12), 2.0, 12)]
    steps = 19
    params = [params_for(n, nu, steps) for n, nu, _ in specs]
    states = [inputs.initial_state(n, 30 + i, "phase", sigma=0.3) for i, (n, _, _) in enumerate(specs)]
    g = sp.Grid(params)
    try:
        for i, st in enumerate(states):
            g.write_state(i, *st)
        g.set_option(sp.SP_OPT_REGION_SHAPE, sp.SP_SHAPE_LATTICE)
        # per-simulation sizes through one explicit plan each would re-plan; the
        # mixed plan comes from the default rule (16 where it divides, else 8,
        # else 4) except for the last, so plan at 0 and check what was chosen
        g.plan(base_B=0)
        infos = [g.plan_info(i) for i in range(len(specs))]
        g.evolve(steps, sp.SP_TRACE)
        got = [g.read_state(i) for i in range(len(specs))]
        traces = []
        for i in range(len(specs)):
            nreg = infos[i]["regions_per_band"] * ((steps - 1) // (infos[i]["base_B"] // 4) + 4)
            buf = np.zeros(2 * nreg, dtype=np.uint64)
            sp._check(sp.sp_read_surface(g.h, i, sp.SP_SURF_TRACE, buf.ctypes.data, buf.nbytes, 0), "trace")
            traces.append(buf.reshape(-1, 2))
    finally:
        g.close()
    assert [i["base_B"] for i in infos] == [16, 16, 8, 4]
    for p, st, res, tr in zip(params, states, got, traces):
        assert_bit_equal(res, run(p, st, [steps], mono=True)[0])
        assert np.all(tr[:, 1] >= tr[:, 0]) and np.all(tr[:, 0] > 0)


def test_lattice_matter_era_128_against_oracle(oracle_mod):
    """128^3 matter era, random phases, 256 steps as eight 32-step calls at
    s = 4: equal to the sweep bit for bit, and the FP64-oracle bars (every
    32-step segment restarted from the GPU's own state; globally while the
    FP32-storage floor allows)."""
    n, steps = 128, 256
    p = params_for((n, n, n), 2.0, steps)
    st = inputs.initial_state((n, n, n), 0, "phase")
    cps, info = run(p, st, [32] * 8, every=True)
    assert info["base_B"] == 16
    assert_bit_equal(cps[steps], run(p, st, [steps], mono=True)[0])
    op = oracle_mod.make_params(n, dt=p.dt, lam=p.lam, eta=p.eta, nu=p.nu, tau0=p.tau0, tau_ref=p.tau_ref)
    rep = check_run(oracle_mod, op, st, cps, p.eta)
    assert rep["asserted_global"]
    print("\n" + format_report("128^3 matter era, 4-cube lattice s = 4", rep))


def test_lattice_dropped_done_report_times_out():
    """A region that never reports done (host-injected) makes its successors'
    bounded waits give up: the call returns SP_ETIMEOUT after about the wait
    limit, and after clearing the injection the grid runs again."""
    n, steps = (32, 32, 32), 16
    p = params_for(n, 0.0, steps)
    st = inputs.initial_state(n, 2, "gaussian", sigma=0.3)
    g = sp.Grid([p])
    try:
        g.write_state(0, *st)
        g.plan(base_B=8, shape=sp.SP_SHAPE_LATTICE)
        g.set_option(sp.SP_OPT_WAIT_LIMIT_NS, 200_000_000)
        per_layer = g.plan_info(0)["regions_per_band"]
        g.set_option(sp.SP_OPT_FAULT_DROP_RELEASE, 2 * per_layer + 5)  # a region of the third layer
        rc = sp.sp_evolve(g.h, steps, 0)
        assert rc == sp.SP_ETIMEOUT
        g.set_option(sp.SP_OPT_FAULT_DROP_RELEASE, -1)
        g.write_state(0, *st)
        g.set_level(0, 0)
        g.evolve(steps)
        got = g.read_state(0)
    finally:
        g.close()
    assert_bit_equal(got, run(p, st, [steps], mono=True)[0])


def test_lattice_rate_128():
    """Rate of the lattice path on the 128^3 matter-era workload (printed;
    the region path must at least run and agree with the sweep)."""
    import time
    n, steps = 128, 64
    p = params_for((n, n, n), 2.0, 256)
    st = inputs.initial_state((n, n, n), 0, "phase")
    rates = {}
    for B in (8, 16, 20):
        if n % B:
            continue
        g = sp.Grid([p])
        try:
            g.write_state(0, *st)
            g.plan(base_B=B, shape=sp.SP_SHAPE_LATTICE)
            g.evolve(steps)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(3):
                g.evolve(steps, sp.SP_TIMING)
                rates.setdefault(B, []).append(g.timing()[1])
            torch.cuda.synchronize()
            info = g.plan_info(0)
        finally:
            g.close()
        ms = min(rates[B])
        print(f"\nlattice B={B}: {ms:.3f} ms per {steps} steps = {n ** 3 * steps / ms * 1e3:.3e} site-updates/s "
              f"({info['threads']} workers, {info['ctas_per_sm']} CTAs/SM, {info['bytes_per_update']:.2f} B/upd)")
    assert rates


def test_lattice_autotune_picks_a_measured_size():
    """SP_AUTOTUNE with lattice regions times every size that divides the grid
    (and every worker count that fits) on scratch copies of the state, keeps
    the fastest per site-update, and leaves the state untouched: the plan it
    returns still evolves bit-exactly."""
    n, steps = (48, 48, 48), 20
    p = params_for(n, 2.0, steps)
    st = inputs.initial_state(n, 9, "phase")
    g = sp.Grid([p])
    try:
        g.write_state(0, *st)
        g.set_option(sp.SP_OPT_REGION_SHAPE, sp.SP_SHAPE_LATTICE)
        g.plan(base_B=sp.SP_AUTOTUNE, threads=sp.SP_AUTOTUNE)
        info = g.plan_info(0)
        assert info["autotuned"] == 1 and info["tune_candidates"] >= 3
        assert info["base_B"] in (8, 12, 16, 24) and info["region_shape"] == sp.SP_SHAPE_LATTICE
        assert_bit_equal(g.read_state(0), st)  # the trials ran on copies
        g.evolve(steps)
        got = g.read_state(0)
    finally:
        g.close()
    assert_bit_equal(got, run(p, st, [steps], mono=True)[0])
