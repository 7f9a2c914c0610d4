"""GPU parity of the perturbative Wilson loops of the TEK links (the observable of
the NSPT runs) against the oracle, plus the twist-eater vacuum value."""
import math

import numpy as np
import pytest
import torch

import nspt_synth as syn
from oracle import tek

from tests.gpu_util import dev, host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nspt():
    import paper_2001_02835_b300 as n
    assert n.lib().nspt_init() == 0
    return n


def split_tol(N):
    return 2.0 ** 10 * math.sqrt(N) * (2.0 ** -47 + 2.0 ** -44)


@pytest.mark.parametrize("algo,prec", [("naive", "fp64"), ("fft", "fp64"), ("fft", "split")])
@pytest.mark.parametrize("L,flux,T,batch,amax", [(3, 1, 4, 2, 2), (2, 1, 6, 1, 3), (5, 2, 3, 1, 2)])
def test_wilson_loops_match_oracle(nspt, algo, prec, L, flux, T, batch, amax):
    g = syn.rng(7300 + 10 * L + T)
    U = syn.link_series(g, L, flux, T, batch)
    ref = tek.wilson_loops(U, tek.twist_phases(L, flux), amax)
    got = host(nspt.tek_wilson_loops(dev(U), flux, amax, algo=algo, prec=prec))
    scale = np.abs(ref).max()
    tol = 1e-12 if prec == "fp64" else split_tol(L * L)
    assert np.abs(got - ref).max() <= tol * scale


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
    # per order, relative to the largest loop coefficient of that order
    den = np.abs(W64).max(axis=(0, 1, 2))
    assert (np.abs(Ws - W64).max(axis=(0, 1, 2)) / den).max() <= split_tol(L * L)
