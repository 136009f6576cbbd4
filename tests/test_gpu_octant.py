"""Base-32 regions on the GPU: one 32^3 region per 2 x 2 x 2 cluster of CTAs,
one octant per CTA, inner faces exchanged through distributed shared memory
every level.

Bars: the region path equals the monolithic sweep bit for bit (phi, pi, c) on
seeded shapes, eras and step counts (whole bands and ragged remainders), with
one mailbox slot and with the ring of two; mixed bases 32 / 16 / 8 in one
call; and the FP64-oracle bars of accuracy_bars.py on a 128^3 matter-era run.
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


def run(p, st, steps, flags=0, base_B=32, slots=None, every=None):
    g = sp.Grid([p])
    try:
        g.write_state(0, *st)
        if slots is not None:
            g.set_option(sp.SP_OPT_MAILBOX_SLOTS, slots)
        if not flags & sp.SP_MONOLITHIC:
            g.plan(base_B=base_B)
        if every:
            out = {}
            for lvl in range(every, steps + 1, every):
                g.evolve(every, flags)
                out[lvl] = g.read_state(0)
            return out, g.plan_info(0) if not flags & sp.SP_MONOLITHIC else None
        g.evolve(steps, flags)
        return g.read_state(0), (g.plan_info(0) if not flags & sp.SP_MONOLITHIC else None)
    finally:
        g.close()


def assert_bit_equal(x, y, tag=""):
    for a, b, name in zip(x, y, ("phi", "pi", "c")):
        d = np.count_nonzero(np.ascontiguousarray(a).view(np.uint32) != np.ascontiguousarray(b).view(np.uint32))
        assert d == 0, f"{tag}{name}: {d} sites differ"


@pytest.mark.parametrize("n,steps,nu,slots", [
    ((64, 64, 64), 32, 2.0, None),     # two bands, one mailbox slot (the default)
    ((64, 64, 64), 16, 0.0, 2),        # one band, ring of two slots
    ((64, 96, 128), 48, 2.0, None),    # anisotropic, three bands
    ((96, 64, 64), 40, 1.0, 1),        # ragged: two bands + 8 remainder steps
    ((64, 64, 96), 7, 2.0, None),      # fewer steps than a band: all remainder
])
def test_base32_bit_exact_vs_monolithic(n, steps, nu, slots):
    p = params_for(n, nu, steps)
    st = inputs.initial_state(n, 3, "gaussian" if nu == 0 else "phase", sigma=0.3)
    reg, info = run(p, st, steps, slots=slots)
    assert info["base_B"] == 32 and info["grid"] % 8 == 0 and info["threads"] == 384
    assert np.all(np.isfinite(reg[0]))
    assert_bit_equal(reg, run(p, st, steps, flags=sp.SP_MONOLITHIC)[0])


def test_base32_mixed_bases_in_one_call():
    """Simulations of bases 32, 16 and 8 in one call (one persistent launch
    per base): each equals its own sweep bit for bit."""
    specs = [((64, 64, 64), 2.0, 32), ((32, 32, 32), 1.0, 16), ((24, 16, 32), 0.0, 8), ((64, 128, 64), 2.0, 32)]
    steps = 32
    params = [params_for(n, nu, steps) for n, nu, _ in specs]
    states = [inputs.initial_state(n, 40 + i, "phase", sigma=0.3) for i, (n, _, _) in enumerate(specs)]
    g = sp.Grid(params)
    try:
        for i, st in enumerate(states):
            g.write_state(i, *st)
        g.plan(base_B=sp.SP_AUTOTUNE)
        g.evolve(steps)
        got = [g.read_state(i) for i in range(len(specs))]
        infos = [g.plan_info(i) for i in range(len(specs))]
    finally:
        g.close()
    for p, st, res, info in zip(params, states, got, infos):
        assert info["base_B"] in (8, 16, 32)
        assert_bit_equal(res, run(p, st, steps, flags=sp.SP_MONOLITHIC)[0])
    # an explicit mix: the first and last at 32 through their own plans
    for i in (0, 3):
        res, info = run(params[i], states[i], steps)
        assert info["base_B"] == 32
        assert_bit_equal(res, got[i])


def test_base32_matter_era_128_against_oracle(oracle_mod):
    """128^3 matter era, random phases, 256 steps at base 32: equal to the
    sweep bit for bit, and the FP64-oracle bars (every 32-step segment
    restarted from the GPU's own state; globally while the FP32-storage floor
    allows)."""
    n, steps = 128, 256
    p = params_for((n, n, n), 2.0, steps)
    st = inputs.initial_state((n, n, n), 0, "phase")
    cps, info = run(p, st, steps, every=32)
    assert info["base_B"] == 32
    assert_bit_equal(cps[steps], run(p, st, steps, flags=sp.SP_MONOLITHIC)[0])
    op = oracle_mod.make_params(n, dt=p.dt, lam=p.lam, eta=p.eta, nu=p.nu, tau0=p.tau0, tau_ref=p.tau_ref)
    rep = check_run(oracle_mod, op, st, cps, p.eta)
    assert rep["asserted_global"]
    print("\n" + format_report("128^3 matter era at base 32", rep))
