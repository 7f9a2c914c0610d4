"""Oracle for the seeded Langevin noise: traceless Hermitian Gaussian matrices
drawn from a counter-based generator.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The noise of the Langevin step (Eq. 3; the step's reading: eta = sum_a xi_a T^a
over orthonormal generators, Tr(T^a T^b) = delta^ab, xi_a ~ N(0, 1), so that
E|eta_ij|^2 = 1 off the diagonal) is an input of the step.  Where it is not
passed in, both this oracle and the library draw it from the same published
counter-based generator, Philox4x32-10 (Salmon, Moraes, Dror and Shaw,
"Parallel random numbers: as easy as 1, 2, 3", SC 2011), each side from its
definition:

* state: a counter of four 32-bit words and a key of two;
* one round: with the multipliers M0 = 0xD2511F53 and M1 = 0xCD9E8D57, the
  64-bit products M0 c0 and M1 c2 split into (hi, lo) halves, and the new
  counter is (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0));
* ten rounds, the key bumped by the Weyl constants (0x9E3779B9, 0xBB67AE85)
  after each round (modulo 2^32).

Mapping used here (fixed, so that every value has one address):

* key = (seed mod 2^32, seed div 2^32);
* matrix c of a call with counter t, block b: counter words (b, c, t mod 2^32,
  t div 2^32); each block gives two Gaussians, numbers 2b and 2b + 1 of the
  matrix's N^2 (row-major position g = i N + j);
* from the block's words (w0, w1, w2, w3): two 53-bit uniforms
  u1 = ((w0 >> 5) 2^26 + (w1 >> 6) + 1) 2^-53 in (0, 1] and
  u2 = ((w2 >> 5) 2^26 + (w3 >> 6)) 2^-53 in [0, 1); Box-Muller:
  r = sqrt(-2 ln u1), z_2b = r cos(2 pi u2), z_2b+1 = r sin(2 pi u2);
* the matrix: eta_ij = (z_{iN+j} + i z_{jN+i}) / sqrt(2) for i < j,
  eta_ji = conj(eta_ij), eta_ii = z_{iN+i} - (1/N) sum_k z_{kN+k}.
"""
from __future__ import annotations

import numpy as np

MASK32 = 0xFFFFFFFF
PHILOX_M0, PHILOX_M1 = 0xD2511F53, 0xCD9E8D57
PHILOX_W0, PHILOX_W1 = 0x9E3779B9, 0xBB67AE85


def philox4x32_10(ctr, key):
    """One Philox4x32-10 block: four 32-bit words from a counter of four and a key of two
    (plain Python integers, one block per call)."""
    c0, c1, c2, c3 = (int(x) & MASK32 for x in ctr)
    k0, k1 = (int(x) & MASK32 for x in key)
    for _ in range(10):
        p0 = PHILOX_M0 * c0
        p1 = PHILOX_M1 * c2
        c0, c1, c2, c3 = ((p1 >> 32) ^ c1 ^ k0, p1 & MASK32, (p0 >> 32) ^ c3 ^ k1, p0 & MASK32)
        k0 = (k0 + PHILOX_W0) & MASK32
        k1 = (k1 + PHILOX_W1) & MASK32
    return c0, c1, c2, c3


def philox4x32_10_array(c0, c1, c2, c3, k0, k1):
    """The same rounds on numpy uint64 arrays holding 32-bit words (elementwise; the
    64-bit products of two 32-bit words fit in uint64)."""
    c = [np.asarray(x, dtype=np.uint64) & np.uint64(MASK32) for x in (c0, c1, c2, c3)]
    k0 = np.uint64(int(k0) & MASK32)
    k1 = np.uint64(int(k1) & MASK32)
    m32 = np.uint64(MASK32)
    for _ in range(10):
        p0 = np.uint64(PHILOX_M0) * c[0]
        p1 = np.uint64(PHILOX_M1) * c[2]
        c = [(p1 >> np.uint64(32)) ^ c[1] ^ k0, p1 & m32, (p0 >> np.uint64(32)) ^ c[3] ^ k1, p0 & m32]
        k0 = (k0 + np.uint64(PHILOX_W0)) & m32
        k1 = (k1 + np.uint64(PHILOX_W1)) & m32
    return c


def gaussians(N: int, count: int, seed: int, counter: int) -> np.ndarray:
    """The N^2 Gaussians z of each of `count` matrices, shape (count, N * N), by the
    mapping of the module docstring."""
    nb = (N * N + 1) // 2
    b, c = np.meshgrid(np.arange(nb, dtype=np.uint64), np.arange(count, dtype=np.uint64))
    t = int(counter)
    w0, w1, w2, w3 = philox4x32_10_array(b, c, np.full_like(b, t & MASK32), np.full_like(b, t >> 32),
                                         int(seed) & MASK32, int(seed) >> 32)
    k1 = (w0 >> np.uint64(5)) * np.uint64(1 << 26) + (w1 >> np.uint64(6))
    k2 = (w2 >> np.uint64(5)) * np.uint64(1 << 26) + (w3 >> np.uint64(6))
    u1 = (k1.astype(np.float64) + 1.0) * 2.0 ** -53
    u2 = k2.astype(np.float64) * 2.0 ** -53
    r = np.sqrt(-2.0 * np.log(u1))
    z = np.empty((count, 2 * nb))
    z[:, 0::2] = r * np.cos(2.0 * np.pi * u2)
    z[:, 1::2] = r * np.sin(2.0 * np.pi * u2)
    return z[:, :N * N]


def langevin_noise(N: int, count: int, seed: int, counter: int = 0) -> np.ndarray:
    """`count` traceless Hermitian N x N matrices (complex128, shape (count, N, N)) from the
    Gaussians of `gaussians`, assembled as the module docstring states."""
    z = gaussians(N, count, seed, counter).reshape(count, N, N)
    eta = np.zeros((count, N, N), dtype=np.complex128)
    s = 1.0 / np.sqrt(2.0)
    for i in range(N):
        for j in range(i + 1, N):
            v = (z[:, i, j] + 1j * z[:, j, i]) * s
            eta[:, i, j] = v
            eta[:, j, i] = np.conj(v)
    d = np.array([z[:, i, i] for i in range(N)]).T          # (count, N)
    mean = d.sum(axis=1) / N
    for i in range(N):
        eta[:, i, i] = d[:, i] - mean
    return eta
