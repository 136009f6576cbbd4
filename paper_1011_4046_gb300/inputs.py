"""Seeded synthetic initial conditions for the scalar string field.

This module is the one place both the CUDA path and the CPU oracle take their
inputs from.  It holds no part of the evolution arithmetic: it only turns a
seed into an initial field (phi, pi, c) on a periodic grid, rounded to FP32
once, exactly as both sides receive it.

Random numbers come from the SplitMix64 generator (Steele, Lea and Flood,
"Fast splittable pseudorandom number generators", OOPSLA 2014), used as a
counter-based stream: output number ``i`` of the stream started from state
``seed`` is ``mix(seed + (i + 1) * GOLDEN)`` (mod 2**64), where ``mix`` is the
published SplitMix64 finaliser.  Uniforms take the top 53 bits.

Two families of initial data are used by the workloads:

* Gaussian: Re phi and Im phi i.i.d. normal with mean 0 and standard
  deviation ``sigma`` per site (Box-Muller on two uniforms per component),
  pi = 0.
* Random phase: phi = eta * exp(i * theta) with theta uniform in [0, 2 pi)
  per site, pi = 0.

The Kahan compensation array c starts at zero.

Arrays use the library layout: shape (n_z, n_y, n_x) complex64, x fastest,
site index ``x + n_x * (y + n_y * z)``.
"""
from __future__ import annotations

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, counters: np.ndarray) -> np.ndarray:
    """Output ``counters[k]`` of the SplitMix64 stream started at ``seed``.

    Vectorised over ``counters`` (uint64).  Wrap-around mod 2**64 is the
    generator's definition, so overflow warnings are silenced.
    """
    c = np.asarray(counters, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + (c + np.uint64(1)) * GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, counters: np.ndarray) -> np.ndarray:
    """Uniform doubles in [0, 1): top 53 bits of the SplitMix64 output."""
    return (splitmix64(seed, counters) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def _sites(n):
    nx, ny, nz = (int(v) for v in n)
    return nx * ny * nz


def gaussian_field(n, seed: int, sigma: float = 0.5) -> np.ndarray:
    """Re and Im phi ~ N(0, sigma) i.i.d. per site; returns complex64 (nz, ny, nx).

    Site i uses uniforms 4i, 4i+1 for Re and 4i+2, 4i+3 for Im (Box-Muller,
    radius from 1 - u so the logarithm never sees 0).  Computed in FP64 and
    rounded to FP32 once.
    """
    nx, ny, nz = (int(v) for v in n)
    s = _sites(n)
    i = np.arange(s, dtype=np.uint64)
    out = np.empty(s, dtype=np.complex128)
    parts = []
    for comp in range(2):
        u1 = uniform01(seed, np.uint64(4) * i + np.uint64(2 * comp))
        u2 = uniform01(seed, np.uint64(4) * i + np.uint64(2 * comp + 1))
        r = np.sqrt(-2.0 * np.log1p(-u1))
        parts.append(sigma * r * np.cos(2.0 * np.pi * u2))
    out.real, out.imag = parts
    return out.astype(np.complex64).reshape(nz, ny, nx)


def random_phase_slab(n, seed: int, z0: int, z1: int, eta: float = 1.0) -> np.ndarray:
    """Planes z0 <= z < z1 of the random-phase field: phi = eta * exp(i theta),
    theta = 2 pi u, u uniform from counter i (the global site index).

    cos and sin come from the host maths library in FP64; the result is
    rounded to FP32 once.  Returns complex64 (z1 - z0, ny, nx).
    """
    nx, ny, _ = (int(v) for v in n)
    plane = nx * ny
    i = np.arange(z0 * plane, z1 * plane, dtype=np.uint64)
    theta = 2.0 * np.pi * uniform01(seed, i)
    out = np.empty(i.size, dtype=np.complex128)
    out.real = eta * np.cos(theta)
    out.imag = eta * np.sin(theta)
    return out.astype(np.complex64).reshape(z1 - z0, ny, nx)


def random_phase_field(n, seed: int, eta: float = 1.0) -> np.ndarray:
    """The whole random-phase field, complex64 (nz, ny, nx); see random_phase_slab."""
    return random_phase_slab(n, seed, 0, int(n[2]), eta)


def initial_state(n, seed: int, kind: str, sigma: float = 0.5, eta: float = 1.0):
    """(phi, pi, c) complex64 arrays of shape (nz, ny, nx): phi from ``kind``,
    pi = 0 (phi' = 0 at the start), c = 0."""
    if kind == "gaussian":
        phi = gaussian_field(n, seed, sigma)
    elif kind == "phase":
        phi = random_phase_field(n, seed, eta)
    else:
        raise ValueError(f"unknown initial-condition kind {kind!r}")
    zeros = np.zeros_like(phi)
    return phi, zeros.copy(), zeros.copy()


def batched_workload(n_sims: int = 64, lo: int = 48, hi: int = 160, step: int = 8):
    """Sizes and eras of the batched workload: sim i draws N uniformly from the
    multiples of ``step`` in [lo, hi] and nu uniformly from {0, 1, 2}, both from
    its own seed i (counters 2**40 and 2**40 + 1 of its stream, clear of the
    field's counters).  Returns a list of (seed, N, nu)."""
    sizes = np.arange(lo, hi + 1, step)
    out = []
    for i in range(n_sims):
        u = uniform01(i, np.array([2 ** 40, 2 ** 40 + 1], dtype=np.uint64))
        n = int(sizes[min(int(u[0] * len(sizes)), len(sizes) - 1)])
        nu = int(min(int(u[1] * 3), 2))
        out.append((i, n, nu))
    return out


# ---------------------------------------------------------------- cost model
MLP_LAYERS = ((64, 16), (64, 64), (1, 64))  # (fan_out, fan_in) of W1, W2, W3
MLP_PARAMS = 64 * 16 + 64 + 64 * 64 + 64 + 64 + 1


def mlp_init(seed: int) -> np.ndarray:
    """He-uniform initial parameters of the 16-64-64-1 cost network, float32.

    Flat layout W1 [64][16], b1 [64], W2 [64][64], b2 [64], W3 [64], b3 [1];
    parameter k draws uniform number k of the stream ``seed``: a weight of a
    layer with fan-in f is (2u - 1) * sqrt(6 / f), computed in FP64 and
    rounded to FP32 once; biases are 0."""
    u = uniform01(seed, np.arange(MLP_PARAMS, dtype=np.uint64))
    out = np.zeros(MLP_PARAMS, dtype=np.float64)
    o = 0
    for fan_out, fan_in in MLP_LAYERS:
        n = fan_out * fan_in
        out[o:o + n] = (2.0 * u[o:o + n] - 1.0) * np.sqrt(6.0 / fan_in)
        o += n + fan_out  # the biases stay 0
    return out.astype(np.float32)


def epoch_orders(seed: int, n: int, epochs: int) -> list:
    """Sample order of each training epoch: the stable argsort of n uniforms,
    epoch e using counters 2**42 + e * 2**32 + i of the stream ``seed``."""
    out = []
    for e in range(epochs):
        c = np.uint64(2 ** 42 + e * 2 ** 32) + np.arange(n, dtype=np.uint64)
        out.append(np.argsort(uniform01(seed, c), kind="stable").astype(np.int32))
    return out
