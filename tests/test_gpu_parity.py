"""GPU parity: the CUDA path against the FP64 oracle and against itself.

Bars (stated per result):
* FP32 Kahan leapfrog on the GPU vs the FP64 oracle from the same FP32
  initial field: max |phi_gpu - phi_oracle| <= 1e-5 * eta at the end of the
  plain-method run; on the chaotic expanding-era runs the same bar on every
  32-step segment restarted from the GPU's own state and globally wherever
  storing the field in FP32 alone costs at most a tenth of it
  (accuracy_bars.py says why), the end-of-run error printed beside that
  FP32-storage floor;
* region-scheduled run vs the monolithic GPU sweep: bit-exact (phi, pi, c);
* diagnostics: plaquette windings equal the oracle's exactly on the same
  FP32 field; FP64 energy terms agree within the rounding bound of two FP64
  sums taken in different orders (accuracy_bars.energy_tol).
Every call goes through the C ABI (paper_1011_4046_gb300.sp).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1011_4046_gb300 import inputs, sp  # noqa: E402

from accuracy_bars import ETA_TOL, check_run, energy_tol, format_report  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    sp.load()


def params_for(n, nu, steps, dt=0.25, lam=2.0, eta=1.0, damp=0):
    tau0 = 10.0 if nu > 0 else 1.0
    return sp.make_params(n, dx=1.0, dt=dt, lam=lam, eta=eta, nu=nu, tau0=tau0,
                          tau_ref=tau0 + (steps - damp) * dt, damp_steps=damp)


def run_gpu(params, state, steps, flags=0, base_B=0, threads=0, slots=None):
    g = sp.Grid([params])
    try:
        g.write_state(0, *state)
        if slots is not None:
            g.set_option(sp.SP_OPT_MAILBOX_SLOTS, slots)
        if not flags & sp.SP_MONOLITHIC:
            g.plan(base_B=base_B, threads=threads)
        g.evolve(steps, flags)
        return g.read_state(0)
    finally:
        g.close()


def bits(a):
    return np.ascontiguousarray(a).view(np.uint32)


def assert_bit_equal(x, y):
    for a, b, name in zip(x, y, ("phi", "pi", "c")):
        diff = np.count_nonzero(bits(a) != bits(b))
        assert diff == 0, f"{name}: {diff} sites differ"


# ------------------------------------------------------------ vs the oracle
def gpu_checkpoints(params, state, steps, every=32, base_B=0, threads=0, shape=None):
    """Region-path run in calls of ``every`` steps; the state after each."""
    g = sp.Grid([params])
    out = {}
    try:
        g.write_state(0, *state)
        g.plan(base_B=base_B, threads=threads, shape=shape)
        for lvl in range(every, steps + 1, every):
            g.evolve(every)
            out[lvl] = g.read_state(0)
    finally:
        g.close()
    return out


def oracle_params(oracle_mod, p):
    return oracle_mod.make_params(tuple(p.n), dx=p.dx, dt=p.dt, lam=p.lam, eta=p.eta, nu=p.nu, tau0=p.tau0,
                                  tau_ref=p.tau_ref, damp_steps=p.damp_steps)


@pytest.mark.parametrize("shape", [None, sp.SP_SHAPE_LATTICE])
def test_gpu_matches_fp64_oracle_plain_method(oracle_mod, shape):
    """The plain-method workload: 32^3, nu = 0, Gaussian sigma = 0.5 (seed 0),
    64 steps, regions of base 8 (split tiling, and 4-cube lattice regions of
    edge 8): max |phi_gpu - phi_oracle| <= 1e-5 eta after the run, and on
    both 32-step segments."""
    n, steps = 32, 64
    p = params_for(n, 0.0, steps)
    st = inputs.initial_state((n, n, n), 0, "gaussian")
    cps = gpu_checkpoints(p, st, steps, base_B=8, shape=shape)
    reg = cps[steps]
    mono = run_gpu(p, st, steps, flags=sp.SP_MONOLITHIC)
    assert_bit_equal(reg, mono)
    op = oracle_params(oracle_mod, p)
    f, v = oracle_mod.run(op, st[0], st[1], 0, steps)
    err_phi = float(np.max(np.abs(reg[0].astype(np.complex128) - f)))
    err_pi = float(np.max(np.abs(reg[1].astype(np.complex128) - v)))
    assert err_phi <= ETA_TOL * p.eta, f"max |dphi| = {err_phi:.3e} (pi: {err_pi:.3e})"
    print("\n" + format_report("plain 32^3", check_run(oracle_mod, op, st, cps, p.eta)))


def matter_era_parity(oracle_mod, n, steps, B):
    """Matter era, random phases: the region path equals the sweep bit for
    bit and meets the accuracy bars (accuracy_bars.check_run)."""
    p = params_for(n, 2.0, steps)
    st = inputs.initial_state((n, n, n), 0, "phase")
    cps = gpu_checkpoints(p, st, steps, base_B=B)
    assert_bit_equal(cps[steps], run_gpu(p, st, steps, flags=sp.SP_MONOLITHIC))
    rep = check_run(oracle_mod, oracle_params(oracle_mod, p), st, cps, p.eta)
    assert rep["asserted_global"], "the global bar was asserted nowhere"
    print("\n" + format_report(f"{n}^3 matter era, {steps} steps", rep))
    return rep


def test_gpu_matches_fp64_oracle_matter_era_64(oracle_mod):
    matter_era_parity(oracle_mod, 64, 128, 16)


@pytest.mark.parametrize("n,B,steps,nu,threads", [
    ((16, 16, 16), 8, 12, 0.0, 0),      # smallest grid (2 regions per axis)
    ((16, 16, 16), 4, 11, 0.0, 0),      # base 4 (64 workers): 5 bands + 1 remainder step
    ((8, 12, 16), 4, 10, 2.0, 128),     # base 4, anisotropic, smallest sides
    ((32, 48, 64), 8, 20, 2.0, 0),      # anisotropic, 5 bands
    ((32, 32, 32), 16, 16, 1.0, 0),     # B = 16, 2 bands
    ((48, 32, 32), 16, 27, 2.0, 256),   # ragged: 3 bands + 3 remainder steps, 256 threads
    ((24, 24, 24), 8, 3, 0.0, 128),     # fewer steps than a band: all remainder
    ((32, 48, 64), 8, 20, 2.0, 128),    # 128 workers at base 8 (the default is 64)
    ((64, 32, 32), 8, 20, 1.0, 256),    # 256 workers at base 8
    ((48, 32, 32), 16, 27, 2.0, 320),   # ragged
    ((32, 32, 32), 16, 16, 1.0, 480),
    ((32, 32, 48), 16, 24, 2.0, 480),   # 480 workers
    ((32, 32, 32), 16, 16, 0.0, 128),   # 128 workers at base 16
])
def test_region_bit_exact_vs_monolithic(n, B, steps, nu, threads):
    p = params_for(n, nu, steps)
    # white noise at sigma = 0.3 stays well inside the local stability bound
    st = inputs.initial_state(n, 5, "gaussian", sigma=0.3)
    reg = run_gpu(p, st, steps, base_B=B, threads=threads)
    mono = run_gpu(p, st, steps, flags=sp.SP_MONOLITHIC)
    assert np.all(np.isfinite(reg[0]))
    assert_bit_equal(reg, mono)


def _random_cases(seed, count):
    """Seeded random configurations: base, per-axis sides (multiples of the
    base, 2 to 5 regions per axis), step counts with ragged remainders, eras
    and worker counts."""
    rng = np.random.default_rng(seed)
    cases = []
    for _ in range(count):
        B = int(rng.choice([4, 8, 16]))
        n = tuple(int(B * rng.integers(2, 6 if B < 16 else 4)) for _ in range(3))
        steps = int(rng.integers(1, 4 * B))
        nu = float(rng.choice([0.0, 1.0, 2.0]))
        threads = int(rng.choice({4: [0, 64, 128], 8: [0, 64, 128, 256], 16: [0, 256, 320, 480]}[B]))
        cases.append((n, B, steps, nu, threads))
    return cases


@pytest.mark.parametrize("n,B,steps,nu,threads", _random_cases(2026, 12))
def test_random_configurations_bit_exact(n, B, steps, nu, threads):
    """Region path == monolithic sweep, bit for bit, on seeded random shapes,
    step counts (whole bands plus any remainder), eras and block shapes."""
    p = params_for(n, nu, steps)
    st = inputs.initial_state(n, steps, "gaussian", sigma=0.3)
    reg = run_gpu(p, st, steps, base_B=B, threads=threads)
    assert all(np.all(np.isfinite(a)) for a in reg)
    assert_bit_equal(reg, run_gpu(p, st, steps, flags=sp.SP_MONOLITHIC))


@pytest.mark.parametrize("n,B,steps,nu,threads", [
    ((16, 16, 16), 4, 11, 0.0, 0),      # base 4: seven seed types, remainder step
    ((32, 48, 64), 8, 20, 2.0, 0),      # base 8, anisotropic, 5 bands
    ((48, 32, 32), 16, 27, 2.0, 0),     # base 16, ragged
    ((32, 48, 64), 8, 20, 2.0, 128),
    ((32, 32, 48), 16, 40, 1.0, 256),   # 5 bands
])
def test_one_mailbox_slot_bit_exact(n, B, steps, nu, threads):
    """One mailbox slot for every band instead of a ring of two: half the
    mailbox memory, with each region also waiting for the previous band's
    readers of the mailboxes it writes.  Results are bit-identical to the
    sweep."""
    p = params_for(n, nu, steps)
    st = inputs.initial_state(n, 17, "gaussian", sigma=0.3)
    reg = run_gpu(p, st, steps, base_B=B, threads=threads, slots=1)
    assert all(np.all(np.isfinite(a)) for a in reg)
    assert_bit_equal(reg, run_gpu(p, st, steps, flags=sp.SP_MONOLITHIC))


def test_one_mailbox_slot_halves_the_mailboxes_batched():
    """Mixed bases in one call with one mailbox slot: every simulation equals
    its sweep, and each plan holds half the mailbox bytes of the ring."""
    specs = [((16, 16, 16), 0.0), ((32, 32, 32), 1.0), ((24, 16, 32), 2.0), ((48, 48, 48), 2.0)]
    steps = 24
    params = [params_for(n, nu, steps) for n, nu in specs]
    states = [inputs.initial_state(n, 30 + i, "phase") for i, (n, _) in enumerate(specs)]
    mb = {}
    for slots in (2, 1):
        g = sp.Grid(params)
        try:
            for i, st in enumerate(states):
                g.write_state(i, *st)
            g.set_option(sp.SP_OPT_MAILBOX_SLOTS, slots)
            g.plan(base_B=0, threads=0)
            g.evolve(steps)
            got = [g.read_state(i) for i in range(len(specs))]
            mb[slots] = [g.plan_info(i)["mailbox_bytes"] for i in range(len(specs))]
        finally:
            g.close()
        for p, st, res in zip(params, states, got):
            assert_bit_equal(res, run_gpu(p, st, steps, flags=sp.SP_MONOLITHIC))
    assert all(a == 2 * b > 0 for a, b in zip(mb[2], mb[1]))
    # one slot is the default
    g = sp.Grid(params[:1])
    try:
        g.plan(base_B=8, threads=0)
        assert g.plan_info(0)["mailbox_slots"] == 1
        with pytest.raises(sp.SpError):
            g.set_option(sp.SP_OPT_MAILBOX_SLOTS, 3)
    finally:
        g.close()


def test_full_size_matter_era_workload(oracle_mod):
    """128^3, matter era, random phases, 256 steps, B = 16: the benchmark
    workload, on the full grid (region == sweep bit for bit inside)."""
    matter_era_parity(oracle_mod, 128, 256, 16)


def test_repeated_and_split_calls_are_consistent():
    """Two calls of 8 steps == one call of 16 steps (state fully in HBM between calls);
    SP_RESTART resets the clock so a rerun from the same state is identical."""
    n, B = (32, 32, 32), 8
    p = params_for(n, 2.0, 16)
    st = inputs.initial_state(n, 9, "phase")
    one = run_gpu(p, st, 16, base_B=B)
    g = sp.Grid([p])
    try:
        g.write_state(0, *st)
        g.plan(base_B=B)
        g.evolve(8)
        g.evolve(8)
        two = g.read_state(0)
        g.write_state(0, *st)
        g.evolve(16, sp.SP_RESTART)
        again = g.read_state(0)
    finally:
        g.close()
    assert_bit_equal(one, two)
    assert_bit_equal(one, again)


def test_batched_sims_in_one_launch():
    """Several simulations of different sizes, eras and bases in one persistent
    launch: each equals its own monolithic sweep bit for bit."""
    specs = [((16, 16, 16), 0.0, "gaussian"), ((32, 32, 32), 1.0, "phase"), ((24, 16, 32), 2.0, "phase"),
             ((48, 48, 48), 2.0, "gaussian")]
    steps = 24
    params = [params_for(n, nu, steps) for n, nu, _ in specs]
    states = [inputs.initial_state(n, i, kind, sigma=0.3) for i, (n, _, kind) in enumerate(specs)]
    g = sp.Grid(params)
    try:
        for i, st in enumerate(states):
            g.write_state(i, *st)
        g.plan(base_B=0)
        g.evolve(steps)
        got = [g.read_state(i) for i in range(len(specs))]
        infos = [g.plan_info(i) for i in range(len(specs))]
    finally:
        g.close()
    assert {i["base_B"] for i in infos} == {8, 16}
    for p, st, res in zip(params, states, got):
        assert_bit_equal(res, run_gpu(p, st, steps, flags=sp.SP_MONOLITHIC))


# ------------------------------------------------------------ diagnostics
@pytest.mark.parametrize("run_steps", [16, 64])
def test_diagnostics_match_oracle(oracle_mod, run_steps):
    """Windings exactly and the three FP64 energy terms within the summation
    rounding bound (accuracy_bars.energy_tol, 5.5e-12 relative here),
    after 16 steps of a matter-era run planned for run_steps: at its end
    (a = 1) and a quarter of the way in (a = (14/26)^2 = 0.29, where the
    potential's a^2 and the level it is taken at matter)."""
    n, steps = (32, 24, 16), 16
    p = params_for(n, 2.0, run_steps)
    st = inputs.initial_state(n, 4, "gaussian", sigma=0.3)
    g = sp.Grid([p])
    try:
        g.write_state(0, *st)
        g.plan(base_B=8)
        g.evolve(steps)
        phi, pi, _ = g.read_state(0)
        d = g.diag(0)
        w = g.winding(0)
    finally:
        g.close()
    wo = oracle_mod.winding(phi)
    assert np.array_equal(w, wo)
    assert d["pierced"] == [int(np.count_nonzero(wo[k])) for k in range(3)]
    assert d["abs_winding"] == int(np.abs(wo.astype(np.int64)).sum())
    assert d["net_winding"] == [0, 0, 0]
    op = oracle_mod.make_params(n, dt=p.dt, lam=p.lam, eta=p.eta, nu=p.nu, tau0=p.tau0, tau_ref=p.tau_ref)
    kin, grad, pot = oracle_mod.energy_parts(op, phi, pi, steps)
    for got, ref in ((d["kinetic"], kin), (d["gradient"], grad), (d["potential"], pot)):
        assert abs(got - ref) <= energy_tol(n[0] * n[1] * n[2]) * abs(ref)
    a_ref = oracle_mod.level_coeffs(op, steps)["a"]
    assert d["level"] == steps and abs(d["a"] - a_ref) <= 1e-15 * a_ref
    assert (abs(a_ref - 1.0) < 1e-15) == (run_steps == steps)


def test_four_string_winding_on_gpu(oracle_mod):
    N = 16
    z, y, x = np.meshgrid(np.arange(N), np.arange(N), np.arange(N), indexing="ij")
    phi = (np.sin(2 * np.pi * (x + 0.5) / N) + 1j * np.sin(2 * np.pi * (y + 0.5) / N)).astype(np.complex64)
    p = params_for(N, 0.0, 8)
    g = sp.Grid([p])
    try:
        g.write_state(0, phi, np.zeros_like(phi), np.zeros_like(phi))
        d = g.diag(0)
    finally:
        g.close()
    assert d["pierced"] == [0, 0, 4 * N] and d["abs_winding"] == 4 * N


# ------------------------------------------------------------ errors
def test_unstable_plan_is_rejected():
    p = params_for(16, 0.0, 8, dt=0.6)  # dt^2 * 12 > 4
    g = sp.Grid([p])
    try:
        g.plan(base_B=8)
        with pytest.raises(sp.SpError) as e:
            g.evolve(8)
        assert e.value.code == sp.SP_EUNSTABLE
    finally:
        g.close()


def test_bad_base_is_rejected():
    p = params_for((24, 24, 24), 0.0, 8)
    g = sp.Grid([p])
    try:
        with pytest.raises(sp.SpError) as e:
            g.plan(base_B=16)  # 24 is not a multiple of 16
        assert e.value.code == sp.SP_EINVAL
        with pytest.raises(sp.SpError) as e:
            g.plan(base_B=12)  # divides 24, but bases are powers of two
        assert e.value.code == sp.SP_EINVAL
        with pytest.raises(sp.SpError) as e:
            g.evolve(8)
        assert e.value.code == sp.SP_ENOTPLANNED
    finally:
        g.close()
