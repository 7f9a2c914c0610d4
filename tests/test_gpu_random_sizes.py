"""Seeded random sizes through the product forms on the GPU: N from 1 to 300 (ragged tiles of
every kind), T from 0 to 100 (mode counts 2 to 256, T + 1 near and away from powers of two),
batch 1 to 3.  The FFT forms are checked against the naive FP64 form (Eq. 5, no order mixing),
whose own parity with the oracle the other tests pin."""
import math

import numpy as np
import pytest

import nspt_synth as syn

from tests.gpu_util import dev, host, max_order_rel, record, split_bound

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nspt():
    import paper_2001_02835_b300 as n
    assert n.lib().nspt_init() == 0
    return n


def _cases(count=20, seed=31337):
    g = np.random.default_rng(seed)
    out = []
    for i in range(count):
        N = int(g.integers(1, 21)) if i % 2 else int(g.integers(21, 301))
        T = int(g.integers(0, 101))
        # keep the naive reference quick: N^3 (T+1)(T+2)/2 below 1e10 multiply-adds
        while N ** 3 * (T + 1) * (T + 2) // 2 > 10_000_000_000:
            T //= 2
        out.append((N, T, int(g.integers(1, 4))))
    return out


@pytest.mark.parametrize("N,T,batch", _cases())
def test_random_sizes_fft_forms_match_naive(nspt, N, T, batch):
    g = syn.rng(8000 + N + 1000 * T)
    A = syn.series_batch(g, N, T, batch)
    B = syn.series_batch(g, N, T, batch)
    ref = host(nspt.polymat_mul(dev(A), dev(B), algo="naive", prec="fp64"))
    C64 = host(nspt.polymat_mul(dev(A), dev(B), algo="fft", prec="fp64"))
    assert max_order_rel(C64, ref) <= 1e-12
    Cs = host(nspt.polymat_mul(dev(A), dev(B), algo="fft", prec="split"))
    assert np.all(np.isfinite(Cs))
    err = max_order_rel(Cs, ref)
    record("random_sizes_product", N=N, T=T, err=err)
    assert err <= split_bound(6), err


def _tek_cases(count=12, seed=4242):
    g = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        L = int(g.choice([2, 3, 5, 7]))
        flux = int(g.choice([k for k in range(1, L) if math.gcd(k, L) == 1] or [1]))
        out.append((L, flux, int(g.integers(0, 71)), int(g.integers(1, 3))))
    return out


@pytest.mark.parametrize("L,flux,T,streams", _tek_cases())
def test_random_sizes_tek_split_matches_fp64(nspt, L, flux, T, streams):
    """One Langevin step and a 3-step MD trajectory at random (L, T): split form against the
    FP64 FFT form per order (T up to 70 crosses the orders where exp_star's 1/k! leaves the FP32
    normal range)."""
    import torch
    g = syn.rng(8800 + 10 * L + T)
    N = L * L
    U = syn.link_series(g, L, flux, T, streams)
    eta = dev(np.ascontiguousarray(syn.md_momenta(g, N, streams)))
    out = {}
    for prec in ("fp64", "split"):
        tU = dev(U)
        nspt.tek_langevin_step(tU, eta, flux, 0.01, algo="fft", prec=prec)
        tV, tP = dev(U), torch.zeros_like(dev(U))
        nspt.tek_md_trajectory(tV, tP, flux, 0.02, 3, eta=eta, algo="fft", prec=prec)
        out[prec] = (host(tU), host(tV))
    tol = split_bound(6, "langevin", T)
    for i in range(2):
        assert np.all(np.isfinite(out["split"][i]))
        if T > 0:
            err = max_order_rel(out["split"][i][:, :, 1:], out["fp64"][i][:, :, 1:])
            record("random_sizes_tek", L=L, T=T, which=("langevin", "md")[i], err=err)
            assert err <= tol, err


@pytest.mark.parametrize("N,T,batch", _cases(count=8, seed=777))
def test_random_sizes_backward_forms_match_naive(nspt, N, T, batch):
    """The backward (truncated correlations) at random sizes: FFT forms against the naive FP64
    form."""
    g = syn.rng(8500 + N + 1000 * T)
    A = syn.series_batch(g, N, T, batch)
    B = syn.series_batch(g, N, T, batch)
    W = syn.gaussian(g, A.shape, 1.0)
    rA, rB = (host(x) for x in nspt.polymat_mul_backward(dev(A), dev(B), dev(W), algo="naive", prec="fp64"))
    for prec, tol in (("fp64", 1e-12), ("split", split_bound(6, "backward"))):
        gA, gB = (host(x) for x in nspt.polymat_mul_backward(dev(A), dev(B), dev(W), algo="fft", prec=prec))
        err = max(max_order_rel(gA, rA), max_order_rel(gB, rB))
        record("random_sizes_backward", N=N, T=T, prec=prec, err=err)
        assert err <= tol, err
