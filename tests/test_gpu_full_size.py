"""Parity at the benchmarked sizes of the legs beside the headline product (the headline itself
is in test_gpu_split.py and test_gpu_polymat.py): the backward at SU(225), O(g^63), batch 4, and
one MD step of the benchmarked SU(225), O(g^31) configuration with the fitted rescale, every
entry of every order against the oracle."""
import numpy as np
import pytest

import nspt_synth as syn
from oracle import polymat as pm
from oracle import tek

from tests.gpu_util import dev, host, max_order_rel, record, split_bound

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nspt():
    import paper_2001_02835_b300 as n
    assert n.lib().nspt_init() == 0
    return n


def test_backward_su225_t63_full_oracle(nspt):
    g = syn.rng(syn.SEED_BASE + 9)
    N, T, batch = 225, 63, 4
    A = syn.series_batch(g, N, T, batch)
    B = syn.series_batch(g, N, T, batch)
    W = syn.gaussian(g, A.shape, 1.0)
    rA, rB = pm.star_backward(A, B, W)
    for prec, tol in (("fp64", 1e-12), ("split", split_bound(6, "backward"))):
        gA, gB = nspt.polymat_mul_backward(dev(A), dev(B), dev(W), algo="fft", prec=prec)
        err = max(max_order_rel(host(gA), rA), max_order_rel(host(gB), rB))
        record("backward_su225_t63", prec=prec, err=err)
        assert err <= tol, (prec, err)


def decaying_unitary_links(g, L, flux, T, rho):
    """exp_star(i H) * Gamma with traceless Hermitian H, H^(0) = 0 and order k scaled by rho^k:
    a unitary link series whose orders fall off geometrically, like links after thermalisation."""
    N = L * L
    H = syn.hermitian_traceless(g, N, 4 * (T + 1), 1.0 / N).reshape(4, T + 1, N, N)
    H = H * (rho ** np.arange(T + 1))[None, :, None, None]
    H[:, 0] = 0
    G = np.zeros((4, T + 1, N, N), np.complex128)
    G[:, 0] = syn.twist_eaters(L, flux)
    return pm.star(tek.exp_star(1j * H), G)


def test_md_step_su225_t31_full_oracle(nspt):
    """One leapfrog step with momentum refresh at SU(225), O(g^31), flux 1, eps 0.02 (the bench's
    MD configuration), the per-order rescale fitted on the device at every phase, both forms."""
    L, flux, T, eps = 15, 1, 31, 0.02
    N = L * L
    g = syn.rng(syn.SEED_BASE + 11)
    U = decaying_unitary_links(g, L, flux, T, 0.25)
    eta = syn.md_momenta(g, N, 1)[0]
    refU, refP = tek.md_trajectory(U, eta, tek.twist_phases(L, flux), eps, 1)
    for prec in ("fp64", "split"):
        tU = dev(U[None])
        tP = dev(np.zeros_like(U[None]))
        nspt.tek_md_trajectory(tU, tP, flux, eps, 1, eta=dev(eta[None]), algo="fft", prec=prec,
                               rescale_log2r=nspt.RESCALE_AUTO)
        eU = max_order_rel(host(tU)[0][:, 1:], refU[:, 1:])
        eP = max_order_rel(host(tP)[0][:, 1:], refP[:, 1:])
        record("md_su225_t31", prec=prec, errU=eU, errP=eP)
        tol = 1e-12 if prec == "fp64" else split_bound(6, "md", T)
        assert eU <= tol and eP <= tol, (prec, eU, eP)
