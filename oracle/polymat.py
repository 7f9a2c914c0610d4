"""Oracle for the star (convolution) product of truncated polynomial matrices.

TEST INFRASTRUCTURE ONLY (see the package docstring).

A series is an array of shape (..., T+1, N, N), complex128: axis -3 is the
perturbative order k, the last two axes an N x N coefficient matrix.
"""
from __future__ import annotations

import numpy as np

_PI_LD = np.longdouble("3.14159265358979323846264338327950288419716939937510")


def _as_series(X) -> np.ndarray:
    X = np.asarray(X)
    if X.ndim < 3 or X.shape[-1] != X.shape[-2]:
        raise ValueError("a series has shape (..., T+1, N, N)")
    return X


def star(A, B) -> np.ndarray:
    """(A star B)^(k) = sum_{l=0}^{k} A^(l) B^(k-l), k = 0..T  (Eq. 5).

    The matrix order inside each term is kept (A on the left).  Works for
    complex128 and for object arrays of exact numbers (Python ints, Fractions).
    """
    A = _as_series(A)
    B = _as_series(B)
    if A.shape[-3:] != B.shape[-3:]:
        raise ValueError("A and B need the same (T+1, N, N)")
    T = A.shape[-3] - 1
    shape = np.broadcast_shapes(A.shape, B.shape)
    dtype = np.result_type(A.dtype, B.dtype)
    C = np.zeros(shape, dtype=dtype)
    for k in range(T + 1):
        acc = np.zeros(shape[:-3] + shape[-2:], dtype=dtype)
        for l in range(k + 1):
            acc = acc + np.matmul(A[..., l, :, :], B[..., k - l, :, :])
        C[..., k, :, :] = acc
    return C


def default_fft_len(T: int) -> int:
    """Smallest power of two >= 2(T+1) (Sec. 2 uses 2 N_p with N_p = T+1 = 2^s)."""
    M = 1
    while M < 2 * (T + 1):
        M *= 2
    return M


def twiddle_powers(M: int) -> np.ndarray:
    """w^n for n = 0..M-1 with w = exp(2 pi i / M) (Sec. 2, Step 2), computed in
    extended precision and rounded once to complex128."""
    n = np.arange(M, dtype=np.longdouble)
    ang = (2 * _PI_LD) * n / np.longdouble(M)
    return (np.cos(ang).astype(np.float64) + 1j * np.sin(ang).astype(np.float64)).astype(np.complex128)


def dft_forward(A, M: int) -> np.ndarray:
    """Steps 1-2 of FFT-CONV (Sec. 2): pad the order axis with zeros to length M
    and return A~^(p) = sum_{k} A^(k) w^(kp), p = 0..M-1, w = exp(2 pi i/M),
    as a direct O(M^2) sum (no FFT)."""
    A = _as_series(A).astype(np.complex128)
    K = A.shape[-3]
    if M < K:
        raise ValueError("M must be >= T+1")
    w = twiddle_powers(M)
    k = np.arange(K)[None, :]
    p = np.arange(M)[:, None]
    W = w[(k * p) % M]                                      # (M, K)
    return np.tensordot(W, A, axes=([1], [A.ndim - 3])).transpose(
        tuple(range(1, A.ndim - 2)) + (0, A.ndim - 2, A.ndim - 1))


def dft_inverse(Ct, keep: int) -> np.ndarray:
    """Steps 4-5 of FFT-CONV: C^(k) = (1/M) sum_p C~^(p) w^(-kp), keeping
    k = 0..keep-1 and discarding the rest."""
    Ct = _as_series(Ct).astype(np.complex128)
    M = Ct.shape[-3]
    w = twiddle_powers(M)
    k = np.arange(keep)[:, None]
    p = np.arange(M)[None, :]
    Winv = np.conj(w[(k * p) % M]) / M                      # (keep, M)
    return np.tensordot(Winv, Ct, axes=([1], [Ct.ndim - 3])).transpose(
        tuple(range(1, Ct.ndim - 2)) + (0, Ct.ndim - 2, Ct.ndim - 1))


def star_dftconv(A, B, M: int | None = None) -> np.ndarray:
    """FFT-CONV, Steps 1-5 of Sec. 2, with direct DFTs of length M: transform
    both operands, multiply mode by mode (Step 3: C~^(p) = A~^(p) B~^(p)),
    transform back and keep orders 0..T.  Exact in exact arithmetic when
    M >= 2T+1."""
    A = _as_series(A)
    B = _as_series(B)
    T = A.shape[-3] - 1
    if M is None:
        M = default_fft_len(T)
    At = dft_forward(A, M)
    Bt = dft_forward(B, M)
    Ct = np.matmul(At, Bt)
    return dft_inverse(Ct, T + 1)


def dagger(A) -> np.ndarray:
    """Series conjugate: (A^dagger)^(k) = (A^(k))^H for real expansion parameter g."""
    A = _as_series(A)
    return np.conj(np.swapaxes(A, -1, -2))


def identity_series(N: int, T: int, lead=()) -> np.ndarray:
    """The unit of the star product: order 0 = identity, higher orders zero."""
    I = np.zeros(tuple(lead) + (T + 1, N, N), np.complex128)
    I[..., 0, :, :] = np.eye(N)
    return I


def star_backward(A, B, gC):
    """Backward of C = A star B for a real loss, with the convention
    grad = dL/dRe + i dL/dIm, so that dL = Re sum_k Tr(gC_k^H dC_k).

    Differentiating Eq. 5 gives the truncated correlations
        gA_j = sum_{k=j}^{T} gC_k (B_{k-j})^H,
        gB_j = sum_{k=j}^{T} (A_{k-j})^H gC_k,
    written here as explicit double sums.
    """
    A = _as_series(A).astype(np.complex128)
    B = _as_series(B).astype(np.complex128)
    gC = _as_series(gC).astype(np.complex128)
    T = A.shape[-3] - 1
    Ah = dagger(A)
    Bh = dagger(B)
    gA = np.zeros(np.broadcast_shapes(A.shape, gC.shape), np.complex128)
    gB = np.zeros(np.broadcast_shapes(B.shape, gC.shape), np.complex128)
    for j in range(T + 1):
        for k in range(j, T + 1):
            gA[..., j, :, :] += np.matmul(gC[..., k, :, :], Bh[..., k - j, :, :])
            gB[..., j, :, :] += np.matmul(Ah[..., k - j, :, :], gC[..., k, :, :])
    return gA, gB


def order_rel_error(X, ref) -> np.ndarray:
    """Per-order relative Frobenius error ||X_k - ref_k||_F / ||ref_k||_F."""
    X = np.asarray(X)
    ref = np.asarray(ref)
    num = np.sqrt(np.sum(np.abs(X - ref) ** 2, axis=(-1, -2)))
    den = np.sqrt(np.sum(np.abs(ref) ** 2, axis=(-1, -2)))
    return num / np.where(den == 0, 1.0, den)
