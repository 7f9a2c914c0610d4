"""GPU parity of the product path (FP64 form) against the FP64 oracle.

Tolerance: per-order relative Frobenius error <= 1e-12 (the FP64-form target);
integer-valued inputs: naive form bit-exact, FFT form exact after rounding.
Sizes span several 64x64 GEMM tiles and 32-entry FFT strips with ragged tails.
"""
import numpy as np
import pytest
import torch

import nspt_synth as syn
from oracle import polymat as pm

pytestmark = pytest.mark.gpu
TOL = 1e-12


@pytest.fixture(scope="module")
def nspt():
    import paper_2001_02835_b300 as n
    assert n.lib().nspt_init() == 0
    return n


from tests.gpu_util import dev, host, max_order_rel, order_errors, record  # noqa: E402


@pytest.mark.parametrize("N,T,M", [(1, 0, 2), (3, 2, 8), (9, 8, 32), (33, 15, 32), (70, 7, 64), (5, 63, 128),
                                   (4, 100, 256), (2, 200, 512)])
def test_order_fft_and_ifft_match_direct_dft(nspt, N, T, M):
    g = syn.rng(1000 + N * 7 + T)
    A = syn.series_batch(g, N, T, 3)
    At = host(nspt.order_fft(dev(A), M))
    ref = pm.dft_forward(A, M)
    assert np.abs(At - ref).max() <= 1e-13 * max(1.0, np.abs(ref).max())
    Ct = syn.gaussian(g, (3, M, N, N), 1.0)
    C = host(nspt.order_ifft(dev(Ct), T))
    refc = pm.dft_inverse(Ct, T + 1)
    assert np.abs(C - refc).max() <= 1e-14 * max(1.0, np.abs(Ct).max())


@pytest.mark.parametrize("algo", ["naive", "fft"])
@pytest.mark.parametrize("N,T,batch", [(1, 0, 1), (1, 5, 2), (2, 1, 3), (3, 2, 1), (9, 8, 4), (33, 7, 2),
                                       (65, 3, 2), (130, 2, 1), (9, 100, 1), (6, 200, 1)])
def test_mul_fp64_matches_oracle(nspt, algo, N, T, batch):
    g = syn.rng(2000 + N * 13 + T)
    A = syn.series_batch(g, N, T, batch)
    B = syn.series_batch(g, N, T, batch)
    C = host(nspt.polymat_mul(dev(A), dev(B), algo=algo))
    ref = pm.star(A, B)
    assert max_order_rel(C, ref) <= TOL


def test_mul_fft_lengths_and_naive_agree(nspt):
    g = syn.rng(2100)
    N, T = 17, 9
    A = syn.series_batch(g, N, T, 2)
    B = syn.series_batch(g, N, T, 2)
    ref = pm.star(A, B)
    for M in (20 + 12, 64, 128):
        C = host(nspt.polymat_mul(dev(A), dev(B), algo="fft", fft_len=M))
        assert max_order_rel(C, ref) <= TOL


def test_mul_integer_inputs_exact(nspt):
    g = syn.rng(2200)
    N, T = 11, 7
    A = syn.integer_series(g, N, T, 2)
    B = syn.integer_series(g, N, T, 2)
    ref = pm.star(A, B)                      # exact: all partial sums are small integers
    C = host(nspt.polymat_mul(dev(A), dev(B), algo="naive"))
    np.testing.assert_array_equal(C, ref)
    Cf = host(nspt.polymat_mul(dev(A), dev(B), algo="fft"))
    np.testing.assert_array_equal(np.round(Cf.real) + 1j * np.round(Cf.imag), ref)
    assert np.abs(Cf - ref).max() < 1e-9


def test_identity_series_is_unit(nspt):
    g = syn.rng(2300)
    N, T = 20, 6
    A = syn.series_batch(g, N, T, 2)
    I = pm.identity_series(N, T, (2,))
    for algo in ("naive", "fft"):
        np.testing.assert_array_equal(host(nspt.polymat_mul(dev(A), dev(I), algo=algo))[:, :, :, :].real.shape,
                                      A.shape)
        C = host(nspt.polymat_mul(dev(A), dev(I), algo=algo))
        assert np.abs(C - A).max() <= 1e-14


@pytest.mark.parametrize("algo", ["naive", "fft"])
@pytest.mark.parametrize("N,T,batch", [(1, 3, 1), (3, 2, 2), (9, 8, 2), (40, 5, 1)])
def test_backward_fp64_matches_oracle(nspt, algo, N, T, batch):
    g = syn.rng(3000 + N + T)
    A = syn.series_batch(g, N, T, batch)
    B = syn.series_batch(g, N, T, batch)
    W = syn.gaussian(g, A.shape, 1.0)
    gA, gB = nspt.polymat_mul_backward(dev(A), dev(B), dev(W), algo=algo)
    rA, rB = pm.star_backward(A, B, W)
    assert max_order_rel(host(gA), rA) <= TOL
    assert max_order_rel(host(gB), rB) <= TOL


def test_autograd_function_matches_oracle_and_fd(nspt):
    g = syn.rng(3100)
    N, T = 6, 4
    A = syn.series_batch(g, N, T, 1)
    B = syn.series_batch(g, N, T, 1)
    W = syn.gaussian(g, A.shape, 1.0)
    tA = dev(A).requires_grad_(True)
    tB = dev(B).requires_grad_(True)
    tW = dev(W)
    L = torch.real(torch.sum(torch.conj(tW) * nspt.star(tA, tB, algo="fft")))
    L.backward()
    rA, rB = pm.star_backward(A, B, W)
    assert max_order_rel(host(tA.grad), rA) <= TOL
    assert max_order_rel(host(tB.grad), rB) <= TOL
    # central finite differences through the GPU forward (h = 1e-6, FP64)
    h = 1e-6
    for idx in [(0, 0, 1, 2), (0, 3, 4, 0), (0, T, 5, 5)]:
        for d in (1.0, 1j):
            Ap, Am = A.copy(), A.copy()
            Ap[idx] += h * d
            Am[idx] -= h * d
            lp = float(np.real(np.vdot(W, host(nspt.polymat_mul(dev(Ap), dev(B), algo="fft")))))
            lm = float(np.real(np.vdot(W, host(nspt.polymat_mul(dev(Am), dev(B), algo="fft")))))
            fd = (lp - lm) / (2 * h)
            an = rA[idx].real if d == 1.0 else rA[idx].imag
            assert abs(fd - an) < 1e-7 * max(1.0, abs(an))


@pytest.mark.parametrize("T", [31])
def test_su225_fft_and_naive_full_oracle(nspt, T):
    """The paper's timing point SU(225), O(g^31), batch 4 (one per link), FP64 form: GPU
    FFT-CONV and GPU naive product against the oracle's Eq. 5 product, every entry of every
    order, within 1e-12 per order."""
    g = syn.rng(syn.SEED_BASE + 1)
    N, batch = 225, 4
    A = syn.series_batch(g, N, T, batch)
    B = syn.series_batch(g, N, T, batch)
    tA, tB = dev(A), dev(B)
    ref = pm.star(A, B)
    ef = order_errors(host(nspt.polymat_mul(tA, tB, algo="fft")), ref)
    en = order_errors(host(nspt.polymat_mul(tA, tB, algo="naive")), ref)
    record("su225_t31_fp64", per_order_fft=ef.max(0), per_order_naive=en.max(0))
    assert ef.max() <= TOL, ef.max()
    assert en.max() <= TOL, en.max()


def test_fp64_fft_per_order_rescale(nspt):
    """FFT-CONV mixes the orders in one spectrum: with orders growing like 4^k the low orders of
    the FP64 form drown (relative error far above 1e-12); the per-order rescale r = 1/4 (exact,
    undone on C) or the fitted one restores every order to FP64 accuracy."""
    g = syn.rng(4400)
    N, T = 16, 31
    A = syn.series_batch(g, N, T, 2)
    B = syn.series_batch(g, N, T, 2)
    s = (4.0 ** np.arange(T + 1))[None, :, None, None]
    A, B = A * s, B * s
    ref = pm.star(A, B)
    C0 = host(nspt.polymat_mul(dev(A), dev(B), algo="fft", prec="fp64", rescale_log2r=0))
    C2 = host(nspt.polymat_mul(dev(A), dev(B), algo="fft", prec="fp64", rescale_log2r=-2))
    Ca = host(nspt.polymat_mul(dev(A), dev(B), algo="fft", prec="fp64", rescale_log2r=nspt.RESCALE_AUTO))
    assert max_order_rel(C2, ref) <= 1e-12
    assert max_order_rel(Ca, ref) <= 1e-12
    assert max_order_rel(C0, ref) > 1e3 * max_order_rel(C2, ref)
