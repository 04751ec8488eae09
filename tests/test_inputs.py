"""The seeded input generators shared by the oracle and the GPU tests hold the
stated input recipe: h = U[0.5, 1.5] + i U[0.5, 1.5] (real parts drawn
first, then imaginary parts, then N = U[0.5, 1.5], each in C order), the
Fibonacci-lattice incidence directions, and the observation cells."""

import math

import numpy as np

from paper_1602_04691_gb300 import inputs


def test_random_medium_recipe():
    n, seed = 6, 3
    h, N = inputs.random_h_N(n, seed)
    assert h.shape == (n ** 3,) and h.dtype == np.complex128
    assert N.shape == (n ** 3,) and N.dtype == np.float64
    rng = np.random.default_rng(seed)
    re, im, dens = (rng.uniform(0.5, 1.5, n ** 3) for _ in range(3))
    assert np.array_equal(h.real, re) and np.array_equal(h.imag, im) and np.array_equal(N, dens)
    assert h.real.min() >= 0.5 and h.real.max() < 1.5 and N.min() >= 0.5 and N.max() < 1.5


def test_constant_medium():
    h, N = inputs.constant_h_N(4, 2.65481e-9 + 5.30961e-6j)
    assert np.all(h == 2.65481e-9 + 5.30961e-6j) and np.all(N == 1.0) and h.size == 64


def test_fibonacci_directions():
    """z_j = 1 - (2j + 1)/m and azimuth j pi (3 - sqrt 5): unit vectors whose
    z values are equally spaced and whose azimuths advance by the golden angle,
    spread evenly enough that their mean is small."""
    m = 16
    d = inputs.fibonacci_directions(m)
    assert d.shape == (m, 3)
    assert np.allclose(np.linalg.norm(d, axis=1), 1.0, atol=1e-15)
    assert np.allclose(d[:, 2], 1.0 - (2.0 * np.arange(m) + 1.0) / m, atol=0)
    phi = np.arctan2(d[:, 1], d[:, 0])
    golden = math.pi * (3.0 - math.sqrt(5.0))
    step = np.angle(np.exp(1j * (phi[1:] - phi[:-1])) * np.exp(-1j * golden))
    assert np.max(np.abs(step)) < 1e-12
    assert np.linalg.norm(d.mean(axis=0)) < 0.1


def test_observation_cells():
    cells = inputs.observation_cells(128, 1024, 5)
    assert cells.dtype == np.int64 and cells.size == 1024
    assert np.all(np.diff(cells) > 0)                  # sorted, no repeats
    assert cells.min() >= 0 and cells.max() < 128 ** 3
    assert np.array_equal(cells, inputs.observation_cells(128, 1024, 5))


def test_random_complex_is_seeded():
    a = inputs.random_complex(1000, 7)
    assert a.dtype == np.complex128 and a.size == 1000
    assert np.array_equal(a, inputs.random_complex(1000, 7))
    assert not np.array_equal(a, inputs.random_complex(1000, 8))
