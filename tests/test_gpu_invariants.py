"""Invariants of the GPU path that hold at any size: associativity of the truncated
product, exp(gX) * exp(-gX) = 1 through order T, 1 x 1 series as scalar polynomials, and
unitarity of the link series through
the Langevin step and MD trajectories (exp_star(i X) is unitary for Hermitian X, i.e.
exp_star(iX) * exp_star(-iX) = 1 through order T), in every form."""
import numpy as np
import pytest
import torch

import nspt_synth as syn
from oracle import polymat as pm
from oracle import tek

from tests.gpu_util import dev, host, record, split_bound

pytestmark = pytest.mark.gpu

FORMS = [("naive", "fp64"), ("fft", "fp64"), ("fft", "split")]


@pytest.fixture(scope="module")
def nspt():
    import paper_2001_02835_b300 as n
    assert n.lib().nspt_init() == 0
    return n


@pytest.mark.parametrize("algo,prec", FORMS)
def test_product_is_associative(nspt, algo, prec):
    g = syn.rng(7500)
    N, T, batch = 33, 15, 2
    A, B, C = (dev(syn.series_batch(g, N, T, batch)) for _ in range(3))
    left = nspt.polymat_mul(nspt.polymat_mul(A, B, algo=algo, prec=prec), C, algo=algo, prec=prec)
    right = nspt.polymat_mul(A, nspt.polymat_mul(B, C, algo=algo, prec=prec), algo=algo, prec=prec)
    den = torch.linalg.matrix_norm(left).clamp_min(1e-300)
    err = (torch.linalg.matrix_norm(left - right) / den).max().item()
    record("associativity", algo=algo, prec=prec, err=err)
    # four products, each within the per-product bound
    assert err <= (1e-12 if prec == "fp64" else 4 * split_bound(6)), err


def _exp_series(X, T, sign):
    """the truncated series of exp(sign g X): coefficients (sign X)^k / k!, k = 0..T"""
    N = X.shape[0]
    out = np.empty((T + 1, N, N), dtype=np.complex128)
    out[0] = np.eye(N)
    for k in range(1, T + 1):
        out[k] = (sign * X) @ out[k - 1] / k
    return out


@pytest.mark.parametrize("algo,prec,cm", [("naive", "fp64", 4), ("fft", "fp64", 4), ("fft", "split", 4),
                                          ("fft", "split", 3)])
def test_exp_gx_times_exp_minus_gx_is_one(nspt, algo, prec, cm):
    """exp(gX) * exp(-gX) = 1 through order T: order 0 is the identity and every higher order
    vanishes.  The coefficients fall off factorially (1/31! ~ 1e-34 at ||X|| ~ 1), which no
    geometric rescale r^k flattens, so each order's error is measured on the scale FFT-CONV
    resolves it at: the naive form against sum_j ||A_j|| ||B_{k-j}|| (the size of order k's
    terms), the FFT forms (rescale r = 2^2) against r^-k (sum_j ||r^j A_j||)(sum_j ||r^j B_j||)
    / sqrt(M), the size of the rescaled spectra mapped back to order k.  The bound is
    log2(M) u, u = 2^-53 (FP64) or 2^-(8S-1) (S slices); the split forms with one slice fewer fail
    it."""
    g = syn.rng(7520)
    N, T, batch, log2r = 64, 31, 2, 2
    M = 64
    Xs = [syn.gaussian(g, (N, N), 1.0 / (4 * N)) for _ in range(batch)]     # ||X||_2 ~ 1
    A = np.stack([_exp_series(X, T, +1) for X in Xs])
    B = np.stack([_exp_series(X, T, -1) for X in Xs])
    kw = dict(algo=algo, prec=prec)
    if algo == "fft":
        kw["rescale_log2r"] = log2r
    if cm == 3:
        kw["complex_mode"] = 3
    dA, dB = dev(A), dev(B)

    def zero_order_errors(C):
        C = C.copy()
        C[:, 0] -= np.eye(N)
        return np.sqrt(np.sum(np.abs(C) ** 2, axis=(-1, -2)))

    e = zero_order_errors(host(nspt.polymat_mul(dA, dB, **kw)))
    na = np.sqrt(np.sum(np.abs(A) ** 2, axis=(-1, -2)))          # (batch, T+1)
    nb = np.sqrt(np.sum(np.abs(B) ** 2, axis=(-1, -2)))
    k = np.arange(T + 1)
    if algo == "naive":
        scale = np.stack([np.convolve(na[b], nb[b])[:T + 1] for b in range(batch)])
    else:
        r = 2.0 ** log2r
        sa = (na * r ** k).sum(axis=1, keepdims=True)
        sb = (nb * r ** k).sum(axis=1, keepdims=True)
        scale = sa * sb * r ** (-k) / np.sqrt(M)
    err = (e / scale).max()
    record("exp_identity", algo=algo, prec=prec, cm=cm, err=err)
    if prec == "fp64":
        assert err <= np.log2(M) * 2.0 ** -53, err
    else:
        assert err <= np.log2(M) * 2.0 ** -47, err
        e5 = zero_order_errors(host(nspt.polymat_mul(dA, dB, slices=5, **kw)))
        assert (e5 / scale).max() > np.log2(M) * 2.0 ** -47, (e5 / scale).max()


@pytest.mark.parametrize("algo,prec", FORMS)
def test_one_by_one_series_are_scalar_polynomials(nspt, algo, prec):
    g = syn.rng(7501)
    T, batch = 20, 3
    a = g.normal(size=(batch, T + 1)) + 1j * g.normal(size=(batch, T + 1))
    b = g.normal(size=(batch, T + 1)) + 1j * g.normal(size=(batch, T + 1))
    C = host(nspt.polymat_mul(dev(a.reshape(batch, T + 1, 1, 1).copy()), dev(b.reshape(batch, T + 1, 1, 1).copy()),
                              algo=algo, prec=prec)).reshape(batch, T + 1)
    for i in range(batch):
        ref = np.polynomial.polynomial.polymul(a[i], b[i])[:T + 1]
        err = np.abs(C[i] - ref).max() / np.abs(ref).max()
        record("one_by_one", algo=algo, prec=prec, err=err)
        assert err <= (1e-12 if prec == "fp64" else split_bound(6)), err


def _unitary_links(rg, L, k, T, streams):
    """U = exp_star(i H) * Gamma with Hermitian H (H^(0) = 0): a unitary series at every order."""
    N = L * L
    out = np.empty((streams, 4, T + 1, N, N), np.complex128)
    for s in range(streams):
        H = syn.gaussian(rg, (4, T + 1, N, N), 1.0 / N)
        H = 0.5 * (H + np.conj(np.swapaxes(H, -1, -2)))
        H[:, 0] = 0
        G = np.zeros((4, T + 1, N, N), np.complex128)
        G[:, 0] = syn.twist_eaters(L, k)
        out[s] = pm.star(tek.exp_star(1j * H), G)
    return out


def _unitarity_defect(nspt, U):
    s4 = U.shape[0] * 4
    Uf = U.reshape(s4, *U.shape[2:]).contiguous()
    P = nspt.polymat_mul(Uf, Uf.conj().transpose(-1, -2).contiguous(), algo="fft", prec="fp64")
    I = torch.zeros_like(P)
    I[:, 0] = torch.eye(U.shape[-1], dtype=P.dtype, device=P.device)
    return (P - I).abs().max().item()


@pytest.mark.parametrize("algo,prec", FORMS)
def test_langevin_and_md_keep_links_unitary(nspt, algo, prec):
    rg = syn.rng(7502)
    L, k, T, streams = 3, 1, 10, 2
    N = L * L
    U = dev(_unitary_links(rg, L, k, T, streams))
    assert _unitarity_defect(nspt, U) < 1e-12
    eta = dev(np.ascontiguousarray(syn.hermitian_noise(rg, N, 4 * streams).reshape(streams, 4, N, N)))
    tol = 1e-12 if prec == "fp64" else split_bound(6, "langevin", T)
    U1 = U.clone()
    nspt.tek_langevin_step(U1, eta, k, 0.05, algo=algo, prec=prec)
    d1 = _unitarity_defect(nspt, U1)
    record("unitarity_langevin", algo=algo, prec=prec, defect=d1)
    assert d1 < tol, d1
    assert (U1 - U).abs().max().item() > 1e-3
    P = torch.zeros_like(U)
    nspt.tek_md_trajectory(U1, P, k, 0.05, 5, eta=eta, algo=algo, prec=prec)
    d2 = _unitarity_defect(nspt, U1)
    record("unitarity_md", algo=algo, prec=prec, defect=d2)
    assert d2 < 5 * tol, d2
