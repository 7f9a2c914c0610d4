"""GPU parity of the unitarity projection (polar factor of a link series in the truncated
ring, order 0 kept) against the oracle, in every form: the projected series per order, a
unitary series left unchanged, and V^+ * V = 1 through order T."""
import numpy as np
import pytest
import torch

import nspt_synth as syn
from oracle import polymat as pm
from oracle import tek

from tests.gpu_util import dev, host, max_order_rel, record, split_bound

pytestmark = pytest.mark.gpu
FORMS = [("naive", "fp64"), ("fft", "fp64"), ("fft", "split"), ("naive", "split")]


@pytest.fixture(scope="module")
def nspt():
    import paper_2001_02835_b300 as n
    assert n.lib().nspt_init() == 0
    return n


def _tol(prec, T, algo="fft"):
    return 1e-12 if prec == "fp64" else split_bound(6, "unitarize", T, algo)


def near_unitary_links(g, L, flux, T, streams, delta=1e-2, h=0.25):
    """Links a projection is for: a unitary series exp_star(i H) * Gamma (H Hermitian, variance
    h/N per order, twist eaters at order 0) plus a non-unitary Gaussian drift of size delta at
    orders >= 1.  (A series far from unitary, e.g. Gaussian orders of variance 1/N, makes the
    projection ill-conditioned: its high orders come out of the cancellation of much larger
    terms, and any two exact evaluations differ far above rounding.)"""
    N = L * L
    out = np.empty((streams, 4, T + 1, N, N), np.complex128)
    for s in range(streams):
        H = syn.gaussian(g, (4, T + 1, N, N), h / N)
        H = 0.5 * (H + np.conj(np.swapaxes(H, -1, -2)))
        H[:, 0] = 0
        G = np.zeros((4, T + 1, N, N), np.complex128)
        G[:, 0] = syn.twist_eaters(L, flux)
        P = syn.gaussian(g, (4, T + 1, N, N), 1.0 / N)
        P[:, 0] = 0
        out[s] = pm.star(tek.exp_star(1j * H), G) + delta * P
    return out


@pytest.mark.parametrize("algo,prec", FORMS)
@pytest.mark.parametrize("L,flux,T,streams", [(3, 1, 6, 2), (2, 1, 0, 1), (2, 1, 1, 1), (5, 2, 15, 1),
                                               (11, 3, 31, 1)])
def test_unitarize_matches_oracle(nspt, algo, prec, L, flux, T, streams):
    if L == 11 and algo == "naive":
        pytest.skip("the naive form at SU(121), O(g^31) adds nothing over the FFT forms here")
    g = syn.rng(9300 + 10 * L + T)
    N = L * L
    U = near_unitary_links(g, L, flux, T, streams)
    ref = tek.unitarize(U)
    tU = dev(U)
    nspt.tek_unitarize(tU, algo=algo, prec=prec)
    got = host(tU)
    np.testing.assert_array_equal(got[:, :, 0], U[:, :, 0])
    err = max_order_rel(got, ref)
    rec = {"algo": algo, "prec": prec, "N": N, "T": T, "err": err}
    assert err <= _tol(prec, T, algo), err
    if prec == "split" and N >= 9:
        t5 = dev(U)
        nspt.tek_unitarize(t5, algo=algo, prec=prec, slices=5)
        rec["err_S5"] = max_order_rel(host(t5), ref)
        assert rec["err_S5"] > _tol(prec, T, algo), rec
    record("unitarize", **rec)


@pytest.mark.parametrize("algo,prec", FORMS)
def test_unitarize_keeps_unitary_series_and_makes_series_unitary(nspt, algo, prec):
    rg = syn.rng(9400)
    L, k, T = 3, 1, 8
    N = L * L
    H = syn.gaussian(rg, (4, T + 1, N, N), 1.0 / N)
    H = 0.5 * (H + np.conj(np.swapaxes(H, -1, -2)))
    H[:, 0] = 0
    G = np.zeros((4, T + 1, N, N), np.complex128)
    G[:, 0] = syn.twist_eaters(L, k)
    Uu = pm.star(tek.exp_star(1j * H), G)[None]           # a unitary series
    tU = dev(Uu)
    nspt.tek_unitarize(tU, algo=algo, prec=prec)
    e_fixed = max_order_rel(host(tU), Uu)
    # a non-unitary series becomes unitary: V^+ V = 1 through order T (checked with the oracle)
    U = near_unitary_links(rg, L, k, T, 1)
    tV = dev(U)
    nspt.tek_unitarize(tV, algo=algo, prec=prec)
    V = host(tV)[0]
    I = pm.identity_series(N, T, (4,))
    defect = np.abs(pm.star(pm.dagger(V), V) - I).max()
    record("unitarize_invariants", algo=algo, prec=prec, fixed=e_fixed, defect=defect)
    assert e_fixed <= _tol(prec, T, algo), e_fixed
    assert defect <= _tol(prec, T, algo), defect


def test_unitarize_argument_checks(nspt):
    import ctypes
    L = nspt.lib()
    o = nspt.make_opts(algo="fft", prec="fp64")
    x = torch.zeros((1, 3, 4, 4), dtype=torch.complex128, device="cuda")
    assert L.nspt_tek_unitarize(None, 4, 2, 1, 0, ctypes.byref(o), None) == -1
    assert L.nspt_tek_unitarize(x.data_ptr(), 4, 2, 1, 0, ctypes.byref(o), None) == -4   # no workspace
    ws = nspt._with_ws(nspt.OP_UNITARIZE, 4, 2, 1, o, x.device)  # noqa: F841
    assert L.nspt_tek_unitarize(x.data_ptr(), 4, 2, 1, 2, ctypes.byref(o), None) == -1   # special: 0 or 1
    # the fitted per-order rescale is allowed (one fit per product, on the device)
    tU = dev(near_unitary_links(syn.rng(9500), 2, 1, 6, 1))
    ref = tek.unitarize(host(tU))
    nspt.tek_unitarize(tU, algo="fft", prec="fp64", rescale_log2r=nspt.RESCALE_AUTO)
    assert max_order_rel(host(tU), ref) <= 1e-12


@pytest.mark.parametrize("algo,prec", FORMS)
@pytest.mark.parametrize("L,flux,T,streams", [(3, 1, 6, 2), (2, 1, 0, 1), (2, 1, 1, 1), (5, 2, 15, 1), (11, 3, 31, 1)])
def test_unitarize_special_matches_oracle(nspt, algo, prec, L, flux, T, streams):
    """The projection with the U(1) phase removed: every order against the oracle, and
    det V^(k) conditions through the oracle's det-preserving result (checked on the CPU)."""
    if L == 11 and algo == "naive":
        pytest.skip("the naive form at SU(121), O(g^31) adds nothing over the FFT forms here")
    g = syn.rng(9800 + 10 * L + T)
    N = L * L
    U = near_unitary_links(g, L, flux, T, streams)
    # a U(1) drift on top: every series times exp(i c g) with a seeded c per series
    c = g.normal(size=(streams, 4)) * 0.3
    ph = tek.scalar_exp(np.concatenate([np.zeros((streams, 4, 1)), 1j * c[..., None],
                                        np.zeros((streams, 4, T - 1))], axis=-1)) if T >= 1 else None
    if ph is not None:
        Ur = np.zeros_like(U)
        for k in range(T + 1):
            for j in range(k + 1):
                Ur[:, :, k] += U[:, :, j] * ph[:, :, k - j, None, None]
        U = Ur
    ref = tek.unitarize(U, special=True)
    res = {}
    for r in ([0, nspt.RESCALE_AUTO] if algo == "fft" else [0]):
        tU = dev(U)
        nspt.tek_unitarize(tU, special=True, algo=algo, prec=prec, rescale_log2r=r)
        got = host(tU)
        np.testing.assert_array_equal(got[:, :, 0], U[:, :, 0])
        res[r] = max_order_rel(got, ref)
    record("unitarize_special", algo=algo, prec=prec, N=N, T=T, err=res[0], err_auto=res.get(nspt.RESCALE_AUTO))
    assert res[0] <= _tol(prec, T, algo), res
