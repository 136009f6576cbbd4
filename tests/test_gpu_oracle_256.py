"""The physics of the two large workloads, against the FP64 oracle on a 256^3
grid (the largest the oracle finishes in about a minute on the host cores).

* damped matter era (the 512^3 workload's schedule): random phases (seed 0),
  64 levels with the velocity discarded each step (tau frozen at tau0 = 10),
  then 1024 matter-era steps (nu = 2, tau_ref = tau0 + 1024 dt);
* matter era (the 1280^3 workload's schedule): random phases (seed 0),
  2048 steps (nu = 2, tau0 = 10, tau_ref = tau0 + 2048 dt), energy and
  string length every 128 steps.

Both run the region path at base 16 in 32-step calls.  Bars: the region path
equals the monolithic sweep bit for bit at the end; the FP64-oracle bars of
accuracy_bars.py (1e-5 eta on 32-step segments restarted from the GPU's own
state -- every segment of the damped run, every fourth of the 2048-step run --
and globally while storing the field in FP32 alone costs at most a tenth of
that); at every 128-step checkpoint of the 2048-step run the GPU's plaquette
windings equal the oracle's on the same FP32 field exactly and its FP64
energy terms agree within the rounding bound of two FP64 sums of that many
terms taken in different orders (accuracy_bars.energy_tol).  The end-of-run
global error is printed beside the FP32-storage floor.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1011_4046_gb300 import inputs, sp  # noqa: E402

from accuracy_bars import Bars, energy_tol, format_report  # noqa: E402

pytestmark = pytest.mark.gpu

N = 256


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    sp.load()


def _bit_equal(x, y):
    return all(np.array_equal(np.ascontiguousarray(a).view(np.uint32), np.ascontiguousarray(b).view(np.uint32))
               for a, b in zip(x, y))


def _oracle_params(o, p):
    return o.make_params(tuple(p.n), dx=p.dx, dt=p.dt, lam=p.lam, eta=p.eta, nu=p.nu, tau0=p.tau0,
                         tau_ref=p.tau_ref, damp_steps=p.damp_steps)


def _run(oracle_mod, p, total, segment_every, diag_every=None):
    st = inputs.initial_state((N, N, N), 0, "phase")
    bars = Bars(oracle_mod, _oracle_params(oracle_mod, p), st, p.eta, seg=32, segment_every=segment_every,
                floor_to_end=False)
    g = sp.Grid([p])
    diags = 0
    try:
        g.write_state(0, *st)
        g.plan(base_B=16)
        for lvl in range(32, total + 1, 32):
            g.evolve(32)
            got = g.read_state(0)
            bars.feed(lvl, got)
            if diag_every and lvl % diag_every == 0:
                d = g.diag(0)
                w = g.winding(0)
                wo = oracle_mod.winding(got[0])
                assert np.array_equal(w, wo), f"level {lvl}: windings differ"
                assert d["string_length"] == float(np.count_nonzero(wo)) * p.dx
                kin, grad, pot = oracle_mod.energy_parts(bars.op, got[0], got[1], lvl)
                for x, ref in ((d["kinetic"], kin), (d["gradient"], grad), (d["potential"], pot)):
                    assert abs(x - ref) <= energy_tol(N ** 3) * abs(ref), f"level {lvl}: energy term {x} vs {ref}"
                diags += 1
    finally:
        g.close()
    m = sp.Grid([p])
    try:
        m.write_state(0, *st)
        m.evolve(total, sp.SP_MONOLITHIC)
        mono = m.read_state(0)
    finally:
        m.close()
    assert _bit_equal(got, mono), "region path differs from the monolithic sweep"
    return bars.report(), diags


def test_damped_matter_era_256_against_oracle(oracle_mod):
    damp, steps = 64, 1024
    p = sp.make_params(N, dt=0.25, lam=2.0, eta=1.0, nu=2.0, tau0=10.0, tau_ref=10.0 + steps * 0.25,
                       damp_steps=damp)
    rep, _ = _run(oracle_mod, p, damp + steps, segment_every=32)
    assert len(rep["segments"]) == (damp + steps) // 32
    assert rep["asserted_global"], "the global bar was asserted nowhere"
    print("\n" + format_report("256^3 damped matter era (64 + 1024 steps)", rep))


def test_matter_era_2048_steps_256_against_oracle(oracle_mod):
    steps = 2048
    p = sp.make_params(N, dt=0.25, lam=2.0, eta=1.0, nu=2.0, tau0=10.0, tau_ref=10.0 + steps * 0.25)
    rep, diags = _run(oracle_mod, p, steps, segment_every=128, diag_every=128)
    assert len(rep["segments"]) == steps // 128 and diags == steps // 128
    assert rep["asserted_global"], "the global bar was asserted nowhere"
    print("\n" + format_report("256^3 matter era (2048 steps)", rep))
