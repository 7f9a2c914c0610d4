"""Pins of the oracle's seeded Langevin noise (oracle/noise.py): the counter-based
generator against its published known-answer vectors, the array form against the
scalar form, the address mapping against single blocks, and the matrices against
the distribution the Langevin step's reading fixes (traceless Hermitian, xi_a ~ N(0,1)
on orthonormal generators: E|eta_ij|^2 = 1 off the diagonal, diagonal variance
1 - 1/N)."""
import math
import os

import numpy as np
import pytest
from scipy import stats

from oracle import noise as nz

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def kat_rows():
    for line in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")):
        if line.strip() and not line.startswith("#"):
            w = [int(x, 16) for x in line.split()]
            yield w[0:4], w[4:6], w[6:10]


def test_philox_known_answer_vectors():
    rows = list(kat_rows())
    assert len(rows) == 3
    for ctr, key, out in rows:
        assert list(nz.philox4x32_10(ctr, key)) == out


def test_philox_array_form_equals_scalar_form():
    g = np.random.default_rng(11)
    c = g.integers(0, 2 ** 32, size=(4, 50), dtype=np.uint64)
    k0, k1 = (int(x) for x in g.integers(0, 2 ** 32, size=2))
    arr = nz.philox4x32_10_array(c[0], c[1], c[2], c[3], k0, k1)
    for n in range(50):
        ref = nz.philox4x32_10([int(c[w][n]) for w in range(4)], (k0, k1))
        assert [int(a[n]) for a in arr] == list(ref)


def test_gaussian_addresses_follow_the_stated_mapping():
    """z numbers 2b and 2b + 1 of matrix c at counter t come from block (b, c, t_lo, t_hi)
    under key (seed_lo, seed_hi), by the stated uniforms and Box-Muller."""
    N, count, seed, t = 7, 3, (5 << 32) | 123, (9 << 32) | 77
    z = nz.gaussians(N, count, seed, t)
    for c, b in [(0, 0), (1, 5), (2, 24)]:
        w = nz.philox4x32_10((b, c, t & 0xFFFFFFFF, t >> 32), (seed & 0xFFFFFFFF, seed >> 32))
        u1 = (((w[0] >> 5) << 26) + (w[1] >> 6) + 1) / 2.0 ** 53
        u2 = (((w[2] >> 5) << 26) + (w[3] >> 6)) / 2.0 ** 53
        r = math.sqrt(-2.0 * math.log(u1))
        assert z[c, 2 * b] == pytest.approx(r * math.cos(2 * math.pi * u2), abs=1e-15)
        if 2 * b + 1 < N * N:
            assert z[c, 2 * b + 1] == pytest.approx(r * math.sin(2 * math.pi * u2), abs=1e-15)


def test_gaussians_are_standard_normal():
    z = nz.gaussians(40, 50, seed=2001, counter=3).ravel()       # 80,000 values
    assert abs(z.mean()) < 4 / math.sqrt(z.size)
    assert abs(z.var() - 1.0) < 4 * math.sqrt(2.0 / z.size)
    assert stats.kstest(z, "norm").pvalue > 1e-3


def test_noise_is_traceless_hermitian_with_unit_offdiagonal_variance():
    N, count = 30, 60
    eta = nz.langevin_noise(N, count, seed=7, counter=0)
    np.testing.assert_array_equal(eta, np.conj(np.swapaxes(eta, -1, -2)))
    assert np.abs(np.trace(eta, axis1=1, axis2=2)).max() < 1e-13
    off = ~np.eye(N, dtype=bool)
    m = np.mean(np.abs(eta[:, off]) ** 2)
    n_off = count * N * (N - 1) // 2                              # independent entries
    assert abs(m - 1.0) < 4 * math.sqrt(1.0 / n_off)
    d = np.real(np.diagonal(eta, axis1=1, axis2=2))
    assert abs(np.mean(d ** 2) - (1 - 1.0 / N)) < 4 * math.sqrt(2.0 / (count * N))
    # real and imaginary parts above the diagonal each carry variance 1/2, uncorrelated
    up = eta[:, np.triu(np.ones((N, N), dtype=bool), 1)]
    assert abs(np.mean(up.real ** 2) - 0.5) < 0.02 and abs(np.mean(up.imag ** 2) - 0.5) < 0.02
    assert abs(np.mean(up.real * up.imag)) < 0.02


def test_noise_depends_on_seed_and_counter_only():
    a = nz.langevin_noise(9, 4, seed=1, counter=0)
    np.testing.assert_array_equal(a, nz.langevin_noise(9, 4, seed=1, counter=0))
    np.testing.assert_array_equal(a[:2], nz.langevin_noise(9, 2, seed=1, counter=0))   # matrix c is addressed
    b = nz.langevin_noise(9, 4, seed=1, counter=1)
    c = nz.langevin_noise(9, 4, seed=2, counter=0)
    for x in (b, c):
        r = np.corrcoef(a.real.ravel(), x.real.ravel())[0, 1]
        assert abs(r) < 0.2


def test_noise_1x1_is_zero():
    """SU(1) has no generators: the traceless 1 x 1 noise vanishes."""
    assert np.abs(nz.langevin_noise(1, 5, seed=3)).max() == 0.0
