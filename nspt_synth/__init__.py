"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

This module only draws random numbers and builds input matrices.  It holds none
of the method's arithmetic (no star product, no transform, no twist phase, no
drift): both the CUDA path and the oracle receive the arrays built here and do
all of their own computing.

Distributions (the paper's ensembles are not public, so these stand in):

* order 0 of a coefficient series: Haar-random SU(N) (Mezzadri's QR recipe with
  the phase fix, then divided by det^(1/N));
* orders k >= 1: i.i.d. complex Gaussian entries of variance 1/N
  (real and imaginary parts each N(0, 1/(2N)));
* Langevin noise: a traceless Hermitian Gaussian matrix
  eta = sum_a xi_a T^a with orthonormal generators Tr(T^a T^b) = delta^{ab}
  and xi_a ~ N(0, 1), i.e. E|eta_ij|^2 = 1 off the diagonal;
* twist eaters Gamma_mu (the classical vacuum of the TEK model, Sec. 2, Eq. 1)
  built from L x L clock and shift matrices.
"""
from __future__ import annotations

import math

import numpy as np

SEED_BASE = 200102835


def rng(seed: int) -> np.random.Generator:
    """PCG64 generator; every input of a test or benchmark comes from one seed."""
    return np.random.Generator(np.random.PCG64(seed))


def haar_sun(g: np.random.Generator, N: int, count: int = 1) -> np.ndarray:
    """`count` Haar-random SU(N) matrices, shape (count, N, N), complex128."""
    Z = (g.standard_normal((count, N, N)) + 1j * g.standard_normal((count, N, N))) / math.sqrt(2.0)
    out = np.empty((count, N, N), np.complex128)
    for c in range(count):
        Q, R = np.linalg.qr(Z[c])
        d = np.diagonal(R)
        Q = Q * (d / np.abs(d))[None, :]
        det = np.linalg.det(Q)
        out[c] = Q / det ** (1.0 / N)
    return out


def gaussian(g: np.random.Generator, shape, var: float) -> np.ndarray:
    """Complex Gaussian entries with E|x|^2 = var (Re, Im each of variance var/2)."""
    s = math.sqrt(var / 2.0)
    return s * g.standard_normal(shape) + 1j * (s * g.standard_normal(shape))


def series_batch(g: np.random.Generator, N: int, T: int, batch: int) -> np.ndarray:
    """`batch` coefficient series, shape (batch, T+1, N, N): order 0 Haar SU(N),
    orders 1..T complex Gaussian with variance 1/N."""
    X = np.empty((batch, T + 1, N, N), np.complex128)
    X[:, 0] = haar_sun(g, N, batch)
    if T > 0:
        X[:, 1:] = gaussian(g, (batch, T, N, N), 1.0 / N)
    return X


def hermitian_noise(g: np.random.Generator, N: int, count: int) -> np.ndarray:
    """`count` traceless Hermitian Gaussian matrices, shape (count, N, N)."""
    G = gaussian(g, (count, N, N), 1.0)                  # off-diagonal E|.|^2 = 1
    H = np.triu(G, 1)
    H = H + np.conj(np.swapaxes(H, -1, -2))
    d = g.standard_normal((count, N))
    d = d - d.mean(axis=1, keepdims=True)                # traceless
    idx = np.arange(N)
    H[:, idx, idx] = d
    return H


def hermitian_traceless(g: np.random.Generator, N: int, count: int, scale: float = 1.0) -> np.ndarray:
    """Same distribution as `hermitian_noise`, multiplied by `scale`."""
    return scale * hermitian_noise(g, N, count)


def _clock_shift(L: int, omega: complex):
    P = np.diag(omega ** np.arange(L)).astype(np.complex128)
    Q = np.roll(np.eye(L, dtype=np.complex128), 1, axis=0)   # Q e_j = e_{j+1}
    return P, Q


def twist_eaters(L: int, flux: int) -> np.ndarray:
    """Four N x N unitary matrices (N = L^2), shape (4, N, N), such that for
    every mu < nu:  Gamma_mu Gamma_nu = exp(-2 pi i flux / L) Gamma_nu Gamma_mu.

    Built as (P^a Q^b) (x) (P^c Q^d) from the clock P = diag(omega^j) and the
    cyclic shift Q, with omega = exp(-2 pi i flux / L) and the four integer
    vectors (a,b,c,d) = (1,0,0,0), (0,1,0,0), (-1,1,1,0), (-1,1,0,1); their
    pairwise symplectic products are all 1, which gives the common phase.
    For odd L every factor has unit determinant, so each Gamma is in SU(N);
    for even L a global phase fixes the determinant.
    """
    if math.gcd(flux, L) != 1:
        raise ValueError("flux must be coprime to L")
    omega = np.exp(-2j * np.pi * flux / L)
    P, Q = _clock_shift(L, omega)
    vecs = [(1, 0, 0, 0), (0, 1, 0, 0), (-1, 1, 1, 0), (-1, 1, 0, 1)]
    mp = np.linalg.matrix_power
    out = []
    for a, b, c, d in vecs:
        X = mp(P, a % L) @ mp(Q, b % L)
        Y = mp(P, c % L) @ mp(Q, d % L)
        G = np.kron(X, Y)
        N = L * L
        det = np.linalg.det(G)
        G = G / det ** (1.0 / N)
        out.append(G)
    return np.stack(out)


def link_series(g: np.random.Generator, L: int, flux: int, T: int, streams: int) -> np.ndarray:
    """Link series for the Langevin step, shape (streams, 4, T+1, N, N):
    order 0 = twist eaters, orders 1..T complex Gaussian with variance 1/N."""
    N = L * L
    U = np.empty((streams, 4, T + 1, N, N), np.complex128)
    U[:, :, 0] = twist_eaters(L, flux)[None]
    if T > 0:
        U[:, :, 1:] = gaussian(g, (streams, 4, T, N, N), 1.0 / N)
    return U


def vacuum_links(L: int, flux: int, T: int, streams: int) -> np.ndarray:
    """The twisted vacuum as a link series, shape (streams, 4, T+1, N, N): the twist eaters at
    order 0, every higher order zero.  MD trajectories of the benchmark start here (the
    Gaussian orders of link_series are not a unitary series, and under MD their unphysical
    directions grow without bound at N >= 121)."""
    N = L * L
    U = np.zeros((streams, 4, T + 1, N, N), np.complex128)
    U[:, :, 0] = twist_eaters(L, flux)[None]
    return U


def md_momenta(g: np.random.Generator, N: int, streams: int) -> np.ndarray:
    """Order-1 momenta of an MD refresh, shape (streams, 4, N, N): traceless Hermitian Gaussian
    with E|P_ij|^2 = 1/N, the 't Hooft normalisation matching the 1/N variance of the series."""
    return hermitian_noise(g, N, 4 * streams).reshape(streams, 4, N, N) / np.sqrt(N)


def integer_series(g: np.random.Generator, N: int, T: int, batch: int, lo: int = -8, hi: int = 8) -> np.ndarray:
    """Series with small integer real and imaginary parts (for bit-exact tests)."""
    re = g.integers(lo, hi + 1, (batch, T + 1, N, N))
    im = g.integers(lo, hi + 1, (batch, T + 1, N, N))
    return (re + 1j * im).astype(np.complex128)


GROUP_N = (49, 121, 169, 225, 289)
GROUP_T = (15, 31, 63)


def uneven_group(count: int = 64, seed: int = SEED_BASE + 3):
    """The batched-uneven-products workload: `count` independent products with N drawn
    from GROUP_N and T from GROUP_T, each a batch of one pair (A, B) of series as in
    series_batch (Haar order 0, Gaussian orders >= 1), every pair from its own seed.
    Returns a list of (A, B)."""
    g = rng(seed)
    Ns = g.choice(GROUP_N, count)
    Ts = g.choice(GROUP_T, count)
    out = []
    for N, T in zip(Ns, Ts):
        gp = rng(int(g.integers(1 << 30)))
        out.append((series_batch(gp, int(N), int(T), 1), series_batch(gp, int(N), int(T), 1)))
    return out
