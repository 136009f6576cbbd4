"""Seeded input generators (CPU only).

The generators are shared by the CUDA path and the oracle, so they are
pinned on their own: SplitMix64 against published outputs of the generator
(Steele, Lea and Flood, OOPSLA 2014; the values are those of its public
reference implementation for seeds 0 and 1234567), the random-phase and
Gaussian fields against their distributions, and the slab-wise generator used
for grids too large to build at once against the whole-field one.
"""
import numpy as np
import pytest

from paper_1011_4046_gb300 import inputs

# First outputs of the SplitMix64 stream started from the given state.
SPLITMIX64_PUBLISHED = {
    0: [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F, 0xF88BB8A8724C81EC],
    1234567: [6457827717110365317, 3203168211198807973, 9817491932198370423],
}


@pytest.mark.parametrize("seed", sorted(SPLITMIX64_PUBLISHED))
def test_splitmix64_published_outputs(seed):
    want = SPLITMIX64_PUBLISHED[seed]
    got = inputs.splitmix64(seed, np.arange(len(want), dtype=np.uint64))
    assert [int(v) for v in got] == want


def test_uniforms_take_the_top_53_bits():
    c = np.arange(1000, dtype=np.uint64)
    u = inputs.uniform01(5, c)
    raw = inputs.splitmix64(5, c)
    assert np.all((u >= 0.0) & (u < 1.0))
    assert np.array_equal((u * 2.0 ** 53).astype(np.uint64), raw >> np.uint64(11))


@pytest.mark.parametrize("n,cuts", [((6, 5, 7), (2,)), ((8, 8, 8), (1, 3, 7)), ((4, 6, 5), (0, 5))])
def test_slabs_reassemble_the_whole_field(n, cuts):
    whole = inputs.random_phase_field(n, 3, eta=1.5)
    edges = [0, *cuts, n[2]]
    parts = [inputs.random_phase_slab(n, 3, a, b, eta=1.5) for a, b in zip(edges[:-1], edges[1:])]
    assert whole.shape == (n[2], n[1], n[0])
    assert np.array_equal(np.concatenate(parts).view(np.uint32), whole.view(np.uint32))


def test_random_phase_field_distribution():
    eta = 2.0
    phi = inputs.random_phase_field((32, 32, 32), 11, eta=eta).astype(np.complex128).ravel()
    # |phi| = eta up to the FP32 rounding of each component
    assert np.max(np.abs(np.abs(phi) - eta)) < 4 * eta * 2.0 ** -24
    # theta uniform on the circle: the mean of exp(i theta) is 0 within ~1/sqrt(N)
    m = np.mean(phi) / eta
    assert abs(m) < 4.0 / np.sqrt(phi.size)
    # and the phases fill the circle evenly (8 sectors, binomial bounds)
    sector = ((np.angle(phi) + np.pi) / (2 * np.pi) * 8).astype(int) % 8
    counts = np.bincount(sector, minlength=8)
    p = 1 / 8
    assert np.all(np.abs(counts - phi.size * p) < 5 * np.sqrt(phi.size * p * (1 - p)))


def test_gaussian_field_moments():
    sigma = 0.5
    phi = inputs.gaussian_field((32, 32, 32), 4, sigma=sigma).astype(np.complex128).ravel()
    n = phi.size
    for comp in (phi.real, phi.imag):
        assert abs(np.mean(comp)) < 5 * sigma / np.sqrt(n)
        # variance estimate: standard error sigma^2 sqrt(2 / n)
        assert abs(np.var(comp) - sigma ** 2) < 5 * sigma ** 2 * np.sqrt(2.0 / n)
        # fourth moment of a normal: 3 sigma^4
        k = np.mean(comp ** 4) / sigma ** 4
        assert abs(k - 3.0) < 0.15
    # Re and Im independent
    assert abs(np.mean(phi.real * phi.imag)) < 5 * sigma ** 2 / np.sqrt(n)


def test_initial_state_starts_at_rest():
    phi, pi, c = inputs.initial_state((8, 4, 6), 0, "phase")
    assert phi.dtype == np.complex64 and phi.shape == (6, 4, 8)
    assert not np.any(pi) and not np.any(c)
    with pytest.raises(ValueError):
        inputs.initial_state((8, 8, 8), 0, "uniform")


def test_batched_workload_draws():
    w = inputs.batched_workload()
    assert [s for s, _, _ in w] == list(range(64))
    sizes = {n for _, n, _ in w}
    eras = {nu for _, _, nu in w}
    assert sizes <= set(range(48, 161, 8)) and len(sizes) >= 10
    assert eras == {0, 1, 2}
    assert w == inputs.batched_workload()  # deterministic
