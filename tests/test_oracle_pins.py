"""Pins for the FP64 oracle: each checks it against something other than itself.

* closed forms: the discrete plane-wave dispersion relation (linear,
  flat), the exact Friedmann-era mode solutions tau^(1/2-nu) J_(nu-1/2)
  (linear, nu = 1, 2) and the textbook winding of a four-string field;
* invariants: the exactly conserved leapfrog energy of the linear flat case,
  the second-order energy error of the nonlinear case, cube closure and zero
  net winding of the windings;
* special cases that reduce to a library routine: a uniform field obeys the
  nonlinear ODE, solved here by scipy;
* symmetries (lattice translation, phi -> conj(phi), phi -> i phi), bit-exact;
* brute force: a second, independently written implementation in the
  three-level recurrence form on an 8^3 grid.

A plausible mistake in the oracle (a dropped Laplacian term, a wrong sign or
factor in the friction or potential, a transposed axis, a wrong a(tau)) fails
at least one of these.
"""
import math

import numpy as np
import pytest

from paper_1011_4046_gb300 import inputs


# ----------------------------------------------------------------- helpers
def grid_coords(n):
    nx, ny, nz = n
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return x, y, z


def lattice_k2(k, dx):
    return sum(4.0 / dx ** 2 * math.sin(ki * dx / 2) ** 2 for ki in k)


# ------------------------------------------------------- level coefficients
def test_level_coeffs_special_cases(oracle_mod):
    o = oracle_mod
    p = o.make_params(8, dt=0.25, lam=2.0, nu=0.0, tau0=1.0, tau_ref=1.0)
    for n in (0, 3, 100):
        c = o.level_coeffs(p, n)
        assert c["a"] == 1.0 and c["d"] == 0.0
        assert c["c1"] == 1.0 and c["c2"] == 0.25 and c["m"] == 2.0
        assert c["tau"] == 1.0 + 0.25 * n
    # matter era: a(tau_ref) = 1, a = (tau/tau_ref)^2, d = 2 dt / tau
    p = o.make_params(8, dt=0.25, lam=2.0, nu=2.0, tau0=10.0, tau_ref=74.0)
    c = o.level_coeffs(p, 256)
    assert c["tau"] == 74.0 and c["a"] == 1.0
    c = o.level_coeffs(p, 0)
    assert c["a"] == pytest.approx((10.0 / 74.0) ** 2, rel=1e-15)
    assert c["d"] == pytest.approx(0.05, rel=1e-15)
    assert c["c1"] == pytest.approx(0.95 / 1.05, rel=1e-15)
    assert c["c2"] == pytest.approx(0.25 / 1.05, rel=1e-15)
    # damping phase: velocity discarded, tau frozen
    p = o.make_params(8, dt=0.25, lam=2.0, nu=2.0, tau0=10.0, tau_ref=266.0, damp_steps=64)
    c = o.level_coeffs(p, 10)
    assert c["tau"] == 10.0 and c["c1"] == 0.0 and c["c2"] == 0.125
    c = o.level_coeffs(p, 64 + 4)
    assert c["tau"] == 11.0


# ------------------------------------------------------------ linear, flat
@pytest.mark.parametrize("n,m", [((16, 16, 16), (1, 2, 3)), ((8, 12, 16), (3, -1, 5))])
def test_plane_wave_discrete_dispersion(oracle_mod, n, m):
    """lambda = 0, nu = 0: phi_n = A exp(i (k.x - omega n dt)) exactly, with
    (2/dt)^2 sin^2(omega dt / 2) = (4/dx^2) sum_i sin^2(k_i dx / 2)."""
    o = oracle_mod
    dx, dt, steps = 1.0, 0.25, 64
    k = [2 * math.pi * mi / ni for mi, ni in zip(m, n)]
    omega = 2.0 / dt * math.asin(dt / 2 * math.sqrt(lattice_k2(k, dx)))
    x, y, z = grid_coords(n)
    phase = k[0] * x + k[1] * y + k[2] * z
    A = 0.7 - 0.2j
    phi0 = A * np.exp(1j * phase)
    pi0 = A * np.exp(1j * phase) * (1 - np.exp(1j * omega * dt)) / dt
    p = o.make_params(n, dx=dx, dt=dt, lam=0.0, nu=0.0)
    phi, pi = o.run(p, phi0, pi0, 0, steps)
    exact = A * np.exp(1j * (phase - omega * steps * dt))
    assert np.max(np.abs(phi - exact)) < 1e-11
    exact_pi = A * np.exp(1j * (phase - omega * (steps - 1) * dt)) * (np.exp(-1j * omega * dt) - 1) / dt
    assert np.max(np.abs(pi - exact_pi)) < 1e-11


def test_linear_energy_exact_invariant(oracle_mod):
    """lambda = 0, nu = 0: E_n = sum |pi_{n+1/2}|^2 + Re <phi_n, -Lap phi_{n+1}>
    is conserved by leapfrog to rounding."""
    o = oracle_mod
    n = (12, 10, 8)
    phi, _, _ = inputs.initial_state(n, seed=3, kind="gaussian")
    pi = inputs.gaussian_field(n, seed=4, sigma=0.3)
    p = o.make_params(n, lam=0.0, nu=0.0, dt=0.3)
    phi = phi.astype(np.complex128)
    pi = pi.astype(np.complex128)
    energies, kinetic = [], []
    for step in range(40):
        phi1, pi1 = o.step(p, phi, pi, step)
        kinetic.append(np.sum(np.abs(pi1) ** 2))
        energies.append(kinetic[-1] + o.lap_dot(n, 1.0, phi, phi1))
        phi, pi = phi1, pi1
    e = np.array(energies)
    assert np.max(np.abs(e - e[0])) / e[0] < 1e-12
    # the invariant is not trivially constant: its kinetic part moves a lot
    assert (max(kinetic) - min(kinetic)) / e[0] > 0.05


def _energy_error(o, dt, t_end, eta, n=(8, 8, 8)):
    phi, pi, _ = inputs.initial_state(n, seed=1, kind="gaussian")
    p = o.make_params(n, lam=2.0, eta=eta, nu=0.0, dt=dt)
    phi = phi.astype(np.complex128)
    pi = pi.astype(np.complex128)
    steps = int(round(t_end / dt))
    # state at level n holds pi_{n-1/2}; energy with the time-centred kinetic term
    es = []
    for s in range(steps):
        kin_old = np.sum(np.abs(pi) ** 2)
        phi1, pi1 = o.step(p, phi, pi, s)
        _, grad, pot = o.energy_parts(p, phi, pi1, s)
        kin_new = np.sum(np.abs(pi1) ** 2)
        if s > 0:
            es.append(0.5 * (kin_old + kin_new) + grad + pot)
        phi, pi = phi1, pi1
    es = np.array(es)
    return np.max(np.abs(es - es[0])) / abs(es[0])


@pytest.mark.parametrize("eta", [1.0, 0.7])
def test_nonlinear_energy_error_is_second_order(oracle_mod, eta):
    """lambda = 2, nu = 0: leapfrog energy error scales as dt^2, no drift."""
    o = oracle_mod
    errs = [_energy_error(o, dt, 4.0, eta) for dt in (0.1, 0.05, 0.025)]
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.0 < r1 < 5.5 and 3.0 < r2 < 5.5, errs


# -------------------------------------------------- linear, expanding eras
def _mode_exact(nu, K, tau):
    """Growing-oscillation solution of f'' + (2 nu / tau) f' + K^2 f = 0."""
    x = K * tau
    if nu == 1:
        return math.cos(x) / tau
    if nu == 2:  # tau^(-3/2) J_(3/2)(K tau) ~ j_1(K tau) / tau
        return (math.sin(x) / x ** 2 - math.cos(x) / x) / tau
    raise ValueError(nu)


@pytest.mark.parametrize("nu", [1, 2])
def test_friction_term_matches_bessel_modes(oracle_mod, nu):
    """lambda = 0, nu > 0: a lattice eigenmode follows the exact continuum-time
    solution tau^(1/2-nu) J_(nu-1/2)(K tau) to O(dt^2) (K^2 = lattice eigenvalue)."""
    o = oracle_mod
    n = (8, 8, 8)
    k = (2 * math.pi * 1 / 8, 2 * math.pi * 2 / 8, 0.0)
    K = math.sqrt(lattice_k2(k, 1.0))
    x, y, z = grid_coords(n)
    mode = np.exp(1j * (k[0] * x + k[1] * y + k[2] * z))
    tau0, t_span = 10.0, 8.0
    errs = []
    for dt in (0.1, 0.05, 0.025):
        steps = int(round(t_span / dt))
        f0 = _mode_exact(nu, K, tau0)
        fm = _mode_exact(nu, K, tau0 - dt)
        p = o.make_params(n, lam=0.0, nu=float(nu), dt=dt, tau0=tau0, tau_ref=tau0 + t_span)
        phi, pi = o.run(p, f0 * mode, (f0 - fm) / dt * mode, 0, steps)
        exact = _mode_exact(nu, K, tau0 + steps * dt) * mode
        errs.append(np.max(np.abs(phi - exact)))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.3 < r1 < 4.7 and 3.3 < r2 < 4.7, errs


# ------------------------------------------------------- uniform, nonlinear
@pytest.mark.parametrize("nu,eta", [(2.0, 1.0), (1.0, 1.5)])
def test_uniform_field_follows_nonlinear_ode(oracle_mod, nu, eta):
    """A uniform field has Lap7 phi = 0 exactly: every site stays identical and
    follows f'' + (2 nu/tau) f' + a^2 lambda (|f|^2 - eta^2) f = 0 (scipy
    reference) to O(dt^2)."""
    scipy_integrate = pytest.importorskip("scipy.integrate")
    o = oracle_mod
    n = (4, 4, 4)
    lam, tau0, span = 2.0, 10.0, 16.0
    tau_ref = tau0 + span
    f0 = 0.3 + 0.4j

    def rhs(t, u):
        f = u[0] + 1j * u[1]
        v = u[2] + 1j * u[3]
        a = (t / tau_ref) ** nu
        acc = -(2 * nu / t) * v - a * a * lam * (abs(f) ** 2 - eta ** 2) * f
        return [v.real, v.imag, acc.real, acc.imag]

    ref = scipy_integrate.solve_ivp(rhs, (tau0, tau0 + span), [f0.real, f0.imag, 0.0, 0.0],
                                    rtol=1e-12, atol=1e-14, dense_output=True)
    errs = []
    for dt in (0.1, 0.05, 0.025):
        steps = int(round(span / dt))
        # pi_{-1/2} = f'(tau0 - dt/2) to second order from f'(tau0) = 0
        back = scipy_integrate.solve_ivp(rhs, (tau0, tau0 - dt / 2), [f0.real, f0.imag, 0.0, 0.0],
                                         rtol=1e-12, atol=1e-14)
        v_half = back.y[2, -1] + 1j * back.y[3, -1]
        p = o.make_params(n, lam=lam, eta=eta, nu=nu, dt=dt, tau0=tau0, tau_ref=tau_ref)
        phi, _ = o.run(p, np.full((4, 4, 4), f0), np.full((4, 4, 4), v_half), 0, steps)
        assert np.all(phi == phi.flat[0])
        u = ref.sol(tau0 + steps * dt)
        errs.append(abs(phi.flat[0] - (u[0] + 1j * u[1])))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.3 < r1 < 4.7 and 3.3 < r2 < 4.7, errs


# ------------------------------------------------------------- symmetries
def _evolve(o, phi, pi, steps=10):
    n = phi.shape[::-1]
    p = o.make_params(n, lam=2.0, nu=2.0, dt=0.25, tau0=10.0, tau_ref=12.5)
    return o.run(p, phi, pi, 0, steps)


def test_symmetries_bit_exact(oracle_mod):
    o = oracle_mod
    n = (8, 6, 10)
    phi, _, _ = inputs.initial_state(n, seed=7, kind="gaussian")
    pi = inputs.gaussian_field(n, seed=8, sigma=0.2)
    f, v = _evolve(o, phi, pi)
    # periodic lattice translation
    sh = (2, -1, 3)
    ft, vt = _evolve(o, np.roll(phi, sh, axis=(0, 1, 2)), np.roll(pi, sh, axis=(0, 1, 2)))
    assert np.array_equal(ft, np.roll(f, sh, axis=(0, 1, 2)))
    assert np.array_equal(vt, np.roll(v, sh, axis=(0, 1, 2)))
    # phi -> conj(phi)
    fc, vc = _evolve(o, np.conj(phi), np.conj(pi))
    assert np.array_equal(fc, np.conj(f)) and np.array_equal(vc, np.conj(v))
    # phi -> i phi (Re/Im swap with sign)
    fi, vi = _evolve(o, 1j * phi.astype(np.complex128), 1j * pi.astype(np.complex128))
    assert np.array_equal(fi, 1j * f) and np.array_equal(vi, 1j * v)


# -------------------------------------------- brute force, second algorithm
def _brute_three_level(phi0, pi0, steps, dt, lam, eta, nu, tau0, tau_ref):
    """Independent implementation: eliminate pi and advance
    (1 + d_n) phi_{n+1} = 2 phi_n - (1 - d_n) phi_{n-1} + dt^2 F_n
    with explicit index arithmetic, starting from phi_{-1} = phi_0 - dt pi_{-1/2}."""
    nz, ny, nx = phi0.shape
    cur = [[[complex(phi0[z, y, x]) for x in range(nx)] for y in range(ny)] for z in range(nz)]
    prev = [[[cur[z][y][x] - dt * complex(pi0[z, y, x]) for x in range(nx)] for y in range(ny)]
            for z in range(nz)]
    for n in range(steps):
        tau = tau0 + n * dt
        a2 = (tau / tau_ref) ** (2 * nu)
        d = nu * dt / tau
        nxt = [[[0j] * nx for _ in range(ny)] for _ in range(nz)]
        for z in range(nz):
            for y in range(ny):
                for x in range(nx):
                    c = cur[z][y][x]
                    lap = (cur[z][y][(x + 1) % nx] + cur[z][y][(x - 1) % nx]
                           + cur[z][(y + 1) % ny][x] + cur[z][(y - 1) % ny][x]
                           + cur[(z + 1) % nz][y][x] + cur[(z - 1) % nz][y][x] - 6 * c)
                    force = lap - a2 * lam * (abs(c) ** 2 - eta ** 2) * c
                    nxt[z][y][x] = (2 * c - (1 - d) * prev[z][y][x] + dt * dt * force) / (1 + d)
        prev, cur = cur, nxt
    return np.array(cur)


@pytest.mark.parametrize("nu", [0.0, 2.0])
def test_brute_force_8cubed(oracle_mod, nu):
    o = oracle_mod
    n = (8, 8, 8)
    phi, _, _ = inputs.initial_state(n, seed=11, kind="gaussian")
    pi = inputs.gaussian_field(n, seed=12, sigma=0.1)
    steps, dt, lam, eta, tau0, tau_ref = 6, 0.25, 2.0, 1.0, 10.0, 11.5
    p = o.make_params(n, lam=lam, eta=eta, nu=nu, dt=dt, tau0=tau0, tau_ref=tau_ref)
    f, _ = o.run(p, phi, pi, 0, steps)
    ref = _brute_three_level(phi, pi, steps, dt, lam, eta, nu, tau0, tau_ref)
    assert np.max(np.abs(f - ref)) < 1e-13


# ----------------------------------------------------------------- winding
def test_winding_four_strings_closed_form(oracle_mod):
    """phi = sin(2 pi (x+1/2)/N) + i sin(2 pi (y+1/2)/N) has exactly four
    straight z-strings: 4N pierced z-plaquettes with signs +1, -1, -1, +1 and
    no x or y pierces."""
    o = oracle_mod
    N = 8
    x, y, z = grid_coords((N, N, N))
    phi = (np.sin(2 * np.pi * (x + 0.5) / N) + 1j * np.sin(2 * np.pi * (y + 0.5) / N)).astype(np.complex64)
    w = o.winding(phi)
    assert not w[0].any() and not w[1].any()
    wz = w[2]
    assert np.count_nonzero(wz) == 4 * N
    pierced = {(int(xx), int(yy)): int(wz[0, yy, xx]) for yy, xx in zip(*np.nonzero(wz[0]))}
    # zeros of Re at x + 1/2 in {N/2, N} -> plaquettes x = N/2 - 1 and x = N - 1
    h = N // 2 - 1
    assert pierced == {(h, h): 1, (N - 1, h): -1, (h, N - 1): -1, (N - 1, N - 1): 1}
    # straight strings: every z-plane identical
    assert all(np.array_equal(wz[k], wz[0]) for k in range(N))


def test_winding_cube_closure_and_plane_sums(oracle_mod):
    o = oracle_mod
    n = (10, 8, 6)
    phi = inputs.gaussian_field(n, seed=5)
    w = o.winding(phi).astype(np.int64)
    assert np.count_nonzero(w) > 0
    # divergence over every unit cube: sum_k [w_k(x + e_k) - w_k(x)] = 0
    div = (np.roll(w[0], -1, axis=2) - w[0]) + (np.roll(w[1], -1, axis=1) - w[1]) + \
          (np.roll(w[2], -1, axis=0) - w[2])
    assert not div.any()
    # zero net winding through every full periodic lattice plane
    assert not w[2].sum(axis=(1, 2)).any()
    assert not w[1].sum(axis=(0, 2)).any()
    assert not w[0].sum(axis=(0, 1)).any()


def test_winding_equals_geodesic_phase_rule(oracle_mod):
    """Away from degenerate edges (phase jump exactly pi), the crossing count
    equals the sum of wrapped phase differences / 2 pi."""
    o = oracle_mod
    n = (8, 8, 8)
    phi = inputs.gaussian_field(n, seed=9)
    w = o.winding(phi)
    ang = np.angle(phi.astype(np.complex128))
    for k in range(3):
        a_ax, b_ax = (k + 1) % 3, (k + 2) % 3
        arr_axis = {0: 2, 1: 1, 2: 0}
        def sh(arr, axis):
            return np.roll(arr, -1, axis=arr_axis[axis])
        c0 = ang
        c1 = sh(ang, a_ax)
        c2 = sh(sh(ang, a_ax), b_ax)
        c3 = sh(ang, b_ax)
        total = np.zeros_like(ang)
        for u, v in ((c0, c1), (c1, c2), (c2, c3), (c3, c0)):
            d = v - u
            total += (d + np.pi) % (2 * np.pi) - np.pi
        ref = np.rint(total / (2 * np.pi)).astype(np.int64)
        assert np.array_equal(ref, w[k].astype(np.int64))


# ------------------------------------------- energy balance in an expanding era
def _energy_balance_residual(o, dt, nu=2.0, lam=2.0, eta=1.0, tau0=10.0, span=4.0, n=12):
    """|E_end - E_0 - integral of dE/dtau| along the oracle's trajectory.

    For phi'' + (2 nu/tau) phi' - Lap phi + a^2 lambda (|phi|^2 - eta^2) phi = 0
    with a = (tau/tau_ref)^nu and E = sum |phi'|^2 + sum_links |d phi|^2 / dx^2 +
    a^2 (lambda/2) sum (|phi|^2 - eta^2)^2, the equation gives
    dE/dtau = -(4 nu/tau) sum |phi'|^2 + (2 nu/tau) a^2 (lambda/2) sum (|phi|^2 - eta^2)^2.
    Energies are taken at whole levels (kinetic term: mean of the two
    neighbouring half-step |pi|^2), the rate at half levels (pi_{n+1/2}, phi
    averaged), all computed here from those definitions.  A smooth field starts
    at rest, with pi_{-1/2} = -(dt/2) phi''(tau0)."""
    tau_ref = tau0 + span
    x = np.arange(n) * 2 * np.pi / n
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    phi = (0.6 + 0.3 * np.cos(X) + 0.2 * np.sin(Y + Z)) + 1j * (0.4 * np.sin(X) - 0.3 * np.cos(Z))

    def lap(f):
        return sum(np.roll(f, 1, ax) + np.roll(f, -1, ax) for ax in range(3)) - 6 * f

    def links(f):
        return sum(np.sum(np.abs(np.roll(f, -1, ax) - f) ** 2) for ax in range(3))

    def pot(f, tau):
        a = (tau / tau_ref) ** nu
        return a * a * lam / 2 * np.sum((np.abs(f) ** 2 - eta ** 2) ** 2)

    a0 = (tau0 / tau_ref) ** nu
    pi = -0.5 * dt * (lap(phi) - a0 * a0 * lam * (np.abs(phi) ** 2 - eta ** 2) * phi)
    p = o.make_params((n, n, n), lam=lam, eta=eta, nu=nu, dt=dt, tau0=tau0, tau_ref=tau_ref)
    steps = int(round(span / dt))
    e_first = e_last = None
    work = 0.0
    for s in range(steps):
        phi1, pi1 = o.step(p, phi, pi, s)
        tau = tau0 + s * dt
        e = 0.5 * (np.sum(np.abs(pi) ** 2) + np.sum(np.abs(pi1) ** 2)) + links(phi) + pot(phi, tau)
        e_first = e if e_first is None else e_first
        e_last = e
        if s < steps - 1:
            th = tau + dt / 2
            ah = (th / tau_ref) ** nu
            fb = 0.5 * (phi + phi1)
            work += dt * (-4 * nu / th * np.sum(np.abs(pi1) ** 2)
                          + 2 * nu / th * ah * ah * lam / 2 * np.sum((np.abs(fb) ** 2 - eta ** 2) ** 2))
        phi, pi = phi1, pi1
    return abs(e_last - e_first - work), abs(e_last - e_first)


def test_expanding_era_energy_balance_is_second_order(oracle_mod):
    """nu = 2, lambda = 2: friction, the growing mass a^2 lambda and the
    lattice gradient together obey the continuum energy balance, with a
    residual that falls as dt^2 (a dropped friction factor, a wrong power of
    a or a missing gradient term would leave an O(1) or O(dt) residual)."""
    res = [_energy_balance_residual(oracle_mod, dt) for dt in (0.02, 0.01, 0.005)]
    r1, r2 = res[0][0] / res[1][0], res[1][0] / res[2][0]
    assert 3.2 < r1 < 4.6 and 3.2 < r2 < 4.6, res
    assert all(r < 1e-4 * d for r, d in res), res


def _balance_with_energy_parts(o, dt, nu=2.0, lam=2.0, eta=1.0, tau0=10.0, span=4.0, n=12, tau_ref=None):
    """The expanding-era balance above, with every energy taken from
    ``energy_parts`` itself: its kinetic term (mean of the two half-step sums
    of |pi|^2), its gradient term and its potential a_n^2 (lambda/2) sum
    (|phi|^2 - eta^2)^2 at level n.  The rate of change is written out here
    from the continuum balance.  Returns (|residual|, |E_end - E_0|, a at the
    first and last level)."""
    tau_ref = tau0 + 3 * span if tau_ref is None else tau_ref  # a stays well below 1
    x = np.arange(n) * 2 * np.pi / n
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    phi = (0.6 + 0.3 * np.cos(X) + 0.2 * np.sin(Y + Z)) + 1j * (0.4 * np.sin(X) - 0.3 * np.cos(Z))
    p = o.make_params((n, n, n), lam=lam, eta=eta, nu=nu, dt=dt, tau0=tau0, tau_ref=tau_ref)
    a0 = o.level_coeffs(p, 0)["a"]
    lapf = sum(np.roll(phi, 1, ax) + np.roll(phi, -1, ax) for ax in range(3)) - 6 * phi
    pi = -0.5 * dt * (lapf - a0 * a0 * lam * (np.abs(phi) ** 2 - eta ** 2) * phi)
    steps = int(round(span / dt))
    e_first = e_last = None
    work = 0.0
    for s in range(steps):
        phi1, pi1 = o.step(p, phi, pi, s)
        kin_old, grad, pot = o.energy_parts(p, phi, pi, s)
        kin_new = o.energy_parts(p, phi, pi1, s)[0]
        e = 0.5 * (kin_old + kin_new) + grad + pot
        e_first = e if e_first is None else e_first
        e_last = e
        if s < steps - 1:
            th = tau0 + (s + 0.5) * dt
            ah = (th / tau_ref) ** nu
            fb = 0.5 * (phi + phi1)
            work += dt * (-4 * nu / th * np.sum(np.abs(pi1) ** 2)
                          + 2 * nu / th * ah * ah * lam / 2 * np.sum((np.abs(fb) ** 2 - eta ** 2) ** 2))
        phi, pi = phi1, pi1
    return abs(e_last - e_first - work), abs(e_last - e_first), a0, o.level_coeffs(p, steps - 1)["a"]


def test_energy_parts_obey_the_expanding_era_balance(oracle_mod):
    """``energy_parts`` at a != 1 (nu = 2, a from 0.21 to 0.40 over the run):
    the energies it returns, level by level, satisfy the continuum balance
    dE/dtau = -(4 nu/tau) sum |pi|^2 + (2 nu/tau) a^2 (lambda/2) sum (|phi|^2 -
    eta^2)^2 with a residual that falls as dt^2.  A potential carrying a
    instead of a^2, a taken one level off, or a kinetic term other than
    sum |pi|^2 leaves an O(dt) or O(1) residual instead."""
    res = [_balance_with_energy_parts(oracle_mod, dt) for dt in (0.02, 0.01, 0.005)]
    assert all(0.2 < r[2] < 0.21 and 0.4 < r[3] < 0.41 for r in res), res
    r1, r2 = res[0][0] / res[1][0], res[1][0] / res[2][0]
    assert 3.2 < r1 < 4.6 and 3.2 < r2 < 4.6, res
    assert all(r[0] < 1e-4 * r[1] for r in res), res


def test_energy_parts_of_a_uniform_field_at_a_below_one(oracle_mod):
    """A uniform field has no gradient energy; its potential scales with a^2
    at the stored level.  Two levels of one run (a = 0.25 and a = 0.49) give
    potentials in the ratio (a_1 / a_0)^2 = (tau_1 / tau_0)^4 for nu = 2, a
    property of the definition that does not retype it: the ratio of two
    oracle outputs against the ratio of two conformal times."""
    o = oracle_mod
    n = (4, 4, 4)
    p = o.make_params(n, lam=2.0, eta=1.0, nu=2.0, dt=0.25, tau0=10.0, tau_ref=20.0)
    phi = np.full((4, 4, 4), 0.3 + 0.4j)
    pi = np.full((4, 4, 4), 0.1 - 0.2j)
    k0, g0, v0 = o.energy_parts(p, phi, pi, 0)
    k1, g1, v1 = o.energy_parts(p, phi, pi, 16)  # tau = 14
    assert g0 == 0.0 and g1 == 0.0
    assert k0 == k1 == pytest.approx(64 * 0.05, rel=1e-15)
    assert v1 / v0 == pytest.approx((14.0 / 10.0) ** 4, rel=1e-14)


def test_fp32_storage_twin_rounds_after_every_step(oracle_mod):
    """run_fp32_storage is the plain FP64 step followed by rounding phi and pi
    to FP32, repeated: it equals that composition written out with numpy's
    own float32 rounding, bit for bit, and every value it returns is an FP32
    number."""
    o = oracle_mod
    n = (8, 6, 10)
    phi, _, _ = inputs.initial_state(n, seed=21, kind="phase")
    pi = inputs.gaussian_field(n, seed=22, sigma=0.2)
    p = o.make_params(n, lam=2.0, nu=2.0, dt=0.25, tau0=10.0, tau_ref=14.0)
    f, v = o.run_fp32_storage(p, phi, pi, 3, 7)
    g, w = phi.astype(np.complex128), pi.astype(np.complex128)
    for k in range(7):
        g, w = o.run(p, g, w, 3 + k, 1)
        g, w = g.astype(np.complex64).astype(np.complex128), w.astype(np.complex64).astype(np.complex128)
    assert np.array_equal(f, g) and np.array_equal(v, w)
    assert np.array_equal(f.astype(np.complex64).astype(np.complex128), f)
    assert not np.array_equal(f, o.run(p, phi, pi, 3, 7)[0])  # the rounding does move the run
