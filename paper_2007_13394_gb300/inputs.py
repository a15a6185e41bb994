"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle checks.

Holds random numbers and plain arrays only, none of the method's arithmetic:
* ``white_noise``: unit Gaussian white noise on the N_c^3 Lagrangian lattice
  (float32), the random input of the Zel'dovich initial conditions;
* ``uniform_positions``: uniformly random uint32 fixed-point positions;
* ``uniform_masses`` / ``normal_values``: seeded arrays for linear-algebra checks;
* ``mlp_parameters``: initial parameters of the learned Green's-function factor
  (uniform in +-1/sqrt(fan_in) per layer, the last layer zero unless asked).

Every generator is numpy's PCG64 ``default_rng(seed)``; the same seed gives the
same array on every machine.
"""
from __future__ import annotations

import numpy as np


def white_noise(nc: int, seed: int, chunk: int = 1 << 24) -> np.ndarray:
    """omega(x) ~ N(0, 1) on an nc^3 lattice, x-major (float32, shape (nc, nc, nc))."""
    rng = np.random.default_rng(seed)
    out = np.empty(nc ** 3, dtype=np.float32)
    for lo in range(0, out.size, chunk):
        hi = min(out.size, lo + chunk)
        rng.standard_normal(hi - lo, dtype=np.float32, out=out[lo:hi])
    return out.reshape(nc, nc, nc)


def uniform_positions(n: int, seed: int) -> np.ndarray:
    """Uniformly random uint32 fixed-point positions, shape (3, n)."""
    rng = np.random.default_rng(seed)
    return rng.integers(0, 2 ** 32, size=(3, n), dtype=np.uint64).astype(np.uint32)


def uniform_masses(n: int, seed: int, lo: float = 0.1, hi: float = 2.0) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, size=n)


def normal_values(shape, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.standard_normal(shape)


def mlp_parameters(seed: int, hidden: int = 64, last_scale: float = 0.0) -> np.ndarray:
    """Flat float32 parameters in the library's order W1[h][2], b1[h], W2[h][h], b2[h], w3[h], b3.

    Layers 1 and 2 are uniform in +-1/sqrt(fan_in); w3 and b3 are uniform in
    +-last_scale/sqrt(hidden) (zero by default, which makes the factor exactly 1).
    """
    rng = np.random.default_rng(seed)
    u = lambda n, s: rng.uniform(-s, s, size=n)  # noqa: E731
    parts = [u(2 * hidden, 1 / np.sqrt(2)), u(hidden, 1 / np.sqrt(2)),
             u(hidden * hidden, 1 / np.sqrt(hidden)), u(hidden, 1 / np.sqrt(hidden)),
             u(hidden, last_scale / np.sqrt(hidden)), u(1, last_scale / np.sqrt(hidden))]
    return np.concatenate(parts).astype(np.float32)


def uniform_values(shape, seed: int) -> np.ndarray:
    """Uniform random float32 values in [0, 1) (the draws of pseudo-random sampling)."""
    rng = np.random.default_rng(seed)
    return rng.random(shape, dtype=np.float32)
