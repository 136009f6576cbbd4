"""The damped start (64 initial levels with the velocity discarded, tau frozen
at tau0) on the GPU: region path == sweep bit for bit, the FP64 oracle bar, the
relaxation's energy decrease, and the 512^3 damped matter-era workload at full
size (64 damped + 1024 steps; bit-exactness and diagnostics, the properties
that hold at any size)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1011_4046_gb300 import inputs, sp  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    sp.load()


def _params(n, damp, steps):
    return sp.make_params(n, dt=0.25, lam=2.0, eta=1.0, nu=2.0, tau0=10.0, tau_ref=10.0 + steps * 0.25,
                          damp_steps=damp)


def _bits_equal(x, y):
    return all(np.array_equal(np.ascontiguousarray(a).view(np.uint32), np.ascontiguousarray(b).view(np.uint32))
               for a, b in zip(x, y))


@pytest.mark.parametrize("B", [8, 16])
def test_damped_start_matches_sweep_and_oracle(oracle_mod, B):
    """48^3, 16 damped + 32 normal levels (the remainder of a band runs as
    whole-grid steps): bit-exact with the sweep, within 1e-5 eta of the FP64
    oracle, and the damped phase lowers the energy."""
    n, damp, steps = (48, 48, 48), 16, 32
    p = _params(n, damp, steps)
    st = inputs.initial_state(n, 2, "phase")
    g = sp.Grid([p])
    try:
        g.write_state(0, *st)
        e0 = g.diag(0)["total"]
        g.plan(base_B=B)
        g.evolve(damp)
        e1 = g.diag(0)["total"]
        g.evolve(steps)
        got = g.read_state(0)
    finally:
        g.close()
    assert e1 < e0
    m = sp.Grid([p])
    try:
        m.write_state(0, *st)
        m.evolve(damp + steps, sp.SP_MONOLITHIC)
        want = m.read_state(0)
    finally:
        m.close()
    assert _bits_equal(got, want)
    op = oracle_mod.make_params(48, dt=p.dt, lam=p.lam, eta=p.eta, nu=p.nu, tau0=p.tau0, tau_ref=p.tau_ref,
                                damp_steps=damp)
    f, _ = oracle_mod.run(op, st[0], st[1], 0, damp + steps)
    err = float(np.max(np.abs(got[0].astype(np.complex128) - f)))
    assert err <= 1e-5 * p.eta, f"max |dphi| = {err:.3e}"


def test_damped_512_matter_era_workload():
    """512^3 random phases, 64 damped levels then 1024 steps, region base 16:
    the region path equals the sweep bit for bit; the damped phase lowers the
    energy; the field stays finite and |phi| bounded; the net winding of every
    plaquette orientation is zero on the periodic grid."""
    n, damp, steps = 512, 64, 1024
    p = _params(n, damp, steps)
    st = inputs.initial_state((n, n, n), 0, "phase")
    g = sp.Grid([p])
    try:
        g.write_state(0, *st)
        e0 = g.diag(0)["total"]
        g.plan(base_B=16)
        g.evolve(damp)
        e1 = g.diag(0)["total"]
        g.evolve(steps)
        d = g.diag(0)
        got = g.read_state(0)
    finally:
        g.close()
    del st
    assert e1 < e0
    assert d["level"] == damp + steps and d["net_winding"] == [0, 0, 0] and d["pierced"][0] > 0
    assert np.all(np.isfinite(got[0])) and float(np.max(np.abs(got[0]))) < 4.0
    st = inputs.initial_state((n, n, n), 0, "phase")
    m = sp.Grid([p])
    try:
        m.write_state(0, *st)
        m.evolve(damp + steps, sp.SP_MONOLITHIC)
        want = m.read_state(0)
    finally:
        m.close()
    assert _bits_equal(got, want)
