"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle checks.

This module only draws random numbers and lays them out; it holds none of
the method's arithmetic (no Green's function, no FFT, no solver), so the CPU
oracle and the GPU library can both be fed from it without sharing code.

Recipe (the workloads are synthetic: the paper uses no dataset):
* ``random_h_N(n, seed)``: ``numpy.random.default_rng(seed)``; draws in C-order
  [z][y][x]: Re h ~ U[0.5, 1.5] (all cells), then Im h ~ U[0.5, 1.5], then
  N ~ U[0.5, 1.5].  Returned as complex128 / float64 arrays of n^3 entries.
* ``constant_h_N(n, h, N)``: the paper's Section 4 style constant fields.
* ``fibonacci_directions(m)``: m unit vectors by the Fibonacci lattice
  z_j = 1 - (2j + 1)/m, phi_j = j pi (3 - sqrt 5).
* ``observation_cells(n, count, seed)``: distinct cell indices,
  ``default_rng(seed).choice(n^3, count, replace=False)``, sorted.
* ``random_complex(n_elems, seed)``: test vectors, Re and Im ~ N(0, 1).
"""

from __future__ import annotations

import math
import numpy as np


def random_h_N(n: int, seed: int):
    rng = np.random.default_rng(seed)
    m = n ** 3
    re = rng.uniform(0.5, 1.5, size=m)
    im = rng.uniform(0.5, 1.5, size=m)
    N = rng.uniform(0.5, 1.5, size=m)
    return (re + 1j * im).astype(np.complex128), N.astype(np.float64)


def constant_h_N(n: int, h: complex, N: float = 1.0):
    m = n ** 3
    return np.full(m, complex(h), dtype=np.complex128), np.full(m, float(N), dtype=np.float64)


def fibonacci_directions(m: int) -> np.ndarray:
    j = np.arange(m, dtype=np.float64)
    z = 1.0 - (2.0 * j + 1.0) / m
    phi = j * math.pi * (3.0 - math.sqrt(5.0))
    rxy = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    return np.stack([rxy * np.cos(phi), rxy * np.sin(phi), z], axis=1)


def observation_cells(n: int, count: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(n ** 3, size=count, replace=False)).astype(np.int64)


def random_complex(n_elems: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return (rng.standard_normal(n_elems) + 1j * rng.standard_normal(n_elems)).astype(np.complex128)
