"""GPU parity of the NSPT molecular dynamics (leapfrog with momentum refresh, the
paper's integrator) against the oracle, and its time reversibility."""
import math

import numpy as np
import pytest
import torch

import nspt_synth as syn
from oracle import tek

from tests.gpu_util import dev, host, max_order_rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nspt():
    import paper_2001_02835_b300 as n
    assert n.lib().nspt_init() == 0
    return n


def split_tol(N):
    return 2.0 ** 10 * math.sqrt(N) * (2.0 ** -47 + 2.0 ** -44)


@pytest.mark.parametrize("algo,prec", [("naive", "fp64"), ("fft", "fp64"), ("fft", "split")])
@pytest.mark.parametrize("L,flux,T,streams,nsteps", [(3, 1, 4, 2, 3), (2, 1, 6, 1, 2), (5, 2, 3, 1, 2)])
def test_md_trajectory_matches_oracle(nspt, algo, prec, L, flux, T, streams, nsteps):
    g = syn.rng(7000 + 10 * L + T)
    N = L * L
    U = syn.link_series(g, L, flux, T, streams)
    eta = np.ascontiguousarray(syn.hermitian_noise(g, N, streams * 4).reshape(streams, 4, N, N))
    z = tek.twist_phases(L, flux)
    eps = 0.05
    refU = np.empty_like(U)
    refP = np.empty_like(U)
    for s in range(streams):
        refU[s], refP[s] = tek.md_trajectory(U[s], eta[s], z, eps, nsteps)
    tU = dev(U)
    tP = torch.full_like(tU, float("nan"))   # refresh overwrites every order
    nspt.tek_md_trajectory(tU, tP, flux, eps, nsteps, eta=dev(eta), algo=algo, prec=prec)
    tol = 1e-12 if prec == "fp64" else split_tol(N)
    assert max_order_rel(host(tU)[:, :, 1:], refU[:, :, 1:]) <= tol
    gotP = host(tP)
    assert np.all(gotP[:, :, 0] == 0)
    assert max_order_rel(gotP[:, :, 1:], refP[:, :, 1:]) <= tol
    np.testing.assert_array_equal(host(tU)[:, :, 0], U[:, :, 0])


@pytest.mark.parametrize("prec", ["fp64", "split"])
def test_md_reversible_on_gpu(nspt, prec):
    g = syn.rng(7100)
    L, flux, T = 3, 1, 5
    N = L * L
    U = syn.link_series(g, L, flux, T, 2)
    eta = np.ascontiguousarray(syn.hermitian_noise(g, N, 8).reshape(2, 4, N, N))
    tU, tP = dev(U), torch.zeros_like(dev(U))
    nspt.tek_md_trajectory(tU, tP, flux, 0.04, 4, eta=dev(eta), algo="fft", prec=prec)
    tP.neg_()
    nspt.tek_md_trajectory(tU, tP, flux, 0.04, 4, algo="fft", prec=prec)
    tol = 1e-11 if prec == "fp64" else 1e3 * split_tol(N)
    assert np.abs(host(tU) - U).max() <= tol
    P0 = np.zeros_like(U)
    P0[:, :, 1] = eta
    assert np.abs(-host(tP) - P0).max() <= tol


def test_md_su121_split_vs_fp64(nspt):
    """40 leapfrog steps are the paper's trajectory length; here 4 steps at SU(121), O(g^31),
    8 streams: the split form against the FP64 form."""
    g = syn.rng(syn.SEED_BASE + 4)
    L, flux, T, streams = 11, 3, 31, 8
    N = L * L
    U = syn.link_series(g, L, flux, T, streams)
    eta = dev(np.ascontiguousarray(syn.hermitian_noise(g, N, streams * 4).reshape(streams, 4, N, N)))
    res = {}
    for prec in ("fp64", "split"):
        tU = dev(U)
        tP = torch.zeros_like(tU)
        nspt.tek_md_trajectory(tU, tP, flux, 0.02, 4, eta=eta, algo="fft", prec=prec)
        res[prec] = (host(tU), host(tP))
    tol = split_tol(N)
    assert max_order_rel(res["split"][0][:, :, 1:], res["fp64"][0][:, :, 1:]) <= tol
    assert max_order_rel(res["split"][1][:, :, 1:], res["fp64"][1][:, :, 1:]) <= tol
