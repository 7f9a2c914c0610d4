"""GPU parity of the NSPT Langevin step (FP64 form) against the oracle."""
import numpy as np
import pytest

import nspt_synth as syn
from oracle import polymat as pm
from oracle import tek

from tests.gpu_util import dev, host, max_order_rel, record, split_bound

pytestmark = pytest.mark.gpu
TOL = 1e-12


@pytest.fixture(scope="module")
def nspt():
    import paper_2001_02835_b300 as n
    assert n.lib().nspt_init() == 0
    return n


@pytest.mark.parametrize("algo,prec", [("naive", "fp64"), ("fft", "fp64"), ("fft", "split")])
@pytest.mark.parametrize("L,flux,T,streams", [(3, 1, 8, 1), (3, 1, 2, 2), (2, 1, 5, 1), (5, 2, 4, 2),
                                               # exp_star blocks of 5 (T = 40) and 8 (T = 63) powers
                                               (2, 1, 40, 1), (2, 1, 63, 1)])
def test_langevin_step_matches_oracle(nspt, algo, prec, L, flux, T, streams):
    g = syn.rng(syn.SEED_BASE + 10 * L + T)
    N = L * L
    U = syn.link_series(g, L, flux, T, streams)
    eta = syn.hermitian_noise(g, N, streams * 4).reshape(streams, 4, N, N)
    eps = 0.01
    z = tek.twist_phases(L, flux)
    refU = np.empty_like(U)
    refF = np.empty_like(U)
    for s in range(streams):
        refU[s], refF[s] = tek.langevin_step(U[s], eta[s], z, eps)
    tU = dev(U)
    _, F = nspt.tek_langevin_step(tU, dev(eta), flux, eps, want_drift=True, algo=algo, prec=prec)
    gotU = host(tU)
    gotF = host(F)
    tol = TOL if prec == "fp64" else split_bound(6, "langevin", T)
    # F^(0) vanishes at the twist-eater vacuum (to rounding): it is compared against the
    # largest order's norm, every other order per order
    scaleF = np.sqrt(np.sum(np.abs(refF) ** 2, axis=(-1, -2))).max()
    e0 = np.sqrt(np.sum(np.abs(gotF[:, :, 0] - refF[:, :, 0]) ** 2, axis=(-1, -2))).max() / scaleF
    eF = max(max_order_rel(gotF[:, :, 1:], refF[:, :, 1:]), e0)
    eU = max_order_rel(gotU, refU)
    rec = {"algo": algo, "prec": prec, "N": N, "T": T, "errF": eF, "errU": eU}
    assert eF <= tol, eF
    assert eU <= tol, eU
    np.testing.assert_array_equal(gotU[:, :, 0], U[:, :, 0])
    if prec == "split" and N >= 9:
        # one slice fewer fails the bound
        tU5 = dev(U)
        _, F5 = nspt.tek_langevin_step(tU5, dev(eta), flux, eps, want_drift=True, algo=algo, prec=prec, slices=5)
        e5 = max(max_order_rel(host(F5)[:, :, 1:], refF[:, :, 1:]), max_order_rel(host(tU5), refU))
        rec["err_S5"] = e5
        assert e5 > tol, e5
    record("langevin_step", **rec)


def test_langevin_generic_vacuum_drift(nspt):
    """A non-vacuum order 0 (Haar links): the drift is nonzero at every order."""
    g = syn.rng(4100)
    L, flux, T = 3, 1, 4
    N = L * L
    U = syn.link_series(g, L, flux, T, 1)
    U[0, :, 0] = syn.haar_sun(g, N, 4)
    eta = syn.hermitian_noise(g, N, 4).reshape(1, 4, N, N)
    z = tek.twist_phases(L, flux)
    refU, refF = tek.langevin_step(U[0], eta[0], z, 0.02)
    tU = dev(U)
    _, F = nspt.tek_langevin_step(tU, dev(eta), flux, 0.02, want_drift=True, algo="fft")
    assert max_order_rel(host(F)[0], refF) <= TOL
    assert max_order_rel(host(tU)[0], refU) <= TOL


@pytest.mark.parametrize("T", [32, 40, 47, 63])
def test_split_langevin_high_orders_match_fp64(nspt, T):
    """O(g^40) and beyond: exp_star's coefficients 1/k! fall below the FP32 normal range
    (k >= 35), so spectrum rows whose entries are all subnormal reach the slicer; they must get
    an exponent bound, not the empty-row marker (which once scaled them by 2^254 into inf).
    The split Langevin step matches the FP64 form per order there too."""
    g = syn.rng(9100 + T)
    L, flux = 3, 1
    N = L * L
    U = syn.link_series(g, L, flux, T, 1)
    eta = dev(np.ascontiguousarray(syn.md_momenta(g, N, 1)))
    res = {}
    for prec in ("fp64", "split"):
        tU = dev(U)
        nspt.tek_langevin_step(tU, eta, flux, 0.01, algo="fft", prec=prec)
        res[prec] = host(tU)
    assert np.all(np.isfinite(res["split"]))
    err = max_order_rel(res["split"][:, :, 1:], res["fp64"][:, :, 1:])
    record("langevin_high_orders", T=T, err=err)
    assert err <= split_bound(6, "langevin", T), err
