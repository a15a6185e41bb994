"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle checks.

Holds random numbers and plain arrays only, none of the method's arithmetic:
* ``white_noise``: unit Gaussian white noise on the N_c^3 Lagrangian lattice
  (float32), the random input of the Zel'dovich initial conditions;
* ``uniform_positions``: uniformly random uint32 fixed-point positions;
* ``uniform_masses`` / ``normal_values``: seeded arrays for linear-algebra checks.

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
