"""GPU parity of the perturbative Wilson loops of the TEK links (the observable of
the NSPT runs) against the oracle, plus the twist-eater vacuum value."""
import numpy as np
import pytest
import torch

import nspt_synth as syn
from oracle import tek

from tests.gpu_util import dev, host, record, split_bound

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nspt():
    import paper_2001_02835_b300 as n
    assert n.lib().nspt_init() == 0
    return n


def split_tol(T, algo="fft"):
    return split_bound(6, "wilson", T, algo)


def per_order(got, ref):
    """max over orders k of max_(a,b) |W_k - ref_k| / max_(a,b) |ref_k| (the loops of one order
    share one scale; an order that vanishes is measured against the largest)."""
    num = np.abs(got - ref).max(axis=tuple(range(got.ndim - 1)))
    den = np.abs(ref).max(axis=tuple(range(ref.ndim - 1)))
    return float((num / np.where(den == 0, den.max(), den)).max())


@pytest.mark.parametrize("algo,prec", [("naive", "fp64"), ("fft", "fp64"), ("fft", "split"), ("naive", "split")])
@pytest.mark.parametrize("L,flux,T,batch,amax", [(3, 1, 4, 2, 2), (2, 1, 6, 1, 3), (5, 2, 3, 1, 2)])
def test_wilson_loops_match_oracle(nspt, algo, prec, L, flux, T, batch, amax):
    g = syn.rng(7300 + 10 * L + T)
    U = syn.link_series(g, L, flux, T, batch)
    ref = tek.wilson_loops(U, tek.twist_phases(L, flux), amax)
    got = host(nspt.tek_wilson_loops(dev(U), flux, amax, algo=algo, prec=prec))
    tol = 1e-12 if prec == "fp64" else split_tol(T, algo)
    err = per_order(got, ref)
    record("wilson", algo=algo, prec=prec, L=L, T=T, err=err)
    assert err <= tol, err


def test_wilson_loops_vacuum_is_one(nspt):
    L, flux, T = 5, 2, 3
    N = L * L
    U = np.zeros((1, 4, T + 1, N, N), np.complex128)
    U[0, :, 0] = syn.twist_eaters(L, flux)
    W = host(nspt.tek_wilson_loops(dev(U), flux, 3, algo="fft", prec="split"))
    np.testing.assert_allclose(W[0, :, :, 0], np.ones((3, 3)), atol=1e-12)
    assert np.abs(W[0, :, :, 1:]).max() < 1e-13


def test_wilson_loops_su121_split_vs_fp64(nspt):
    g = syn.rng(syn.SEED_BASE + 4)
    L, flux, T = 11, 3, 31
    U = dev(syn.link_series(g, L, flux, T, 2))
    W64 = host(nspt.tek_wilson_loops(U, flux, 2, algo="fft", prec="fp64"))
    Ws = host(nspt.tek_wilson_loops(U, flux, 2, algo="fft", prec="split"))
    W5 = host(nspt.tek_wilson_loops(U, flux, 2, algo="fft", prec="split", slices=5))
    # per order, relative to the largest loop coefficient of that order
    e6, e5 = per_order(Ws, W64), per_order(W5, W64)
    record("wilson_su121_split_vs_fp64", err_S6=e6, err_S5=e5)
    assert e6 <= split_tol(T), e6
    assert e5 > split_tol(T), e5
