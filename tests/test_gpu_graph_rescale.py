"""The fitted per-order rescale (NSPT_RESCALE_AUTO) runs on the device: the Langevin step and
an MD trajectory with it can be captured in a CUDA graph, and a replay gives bit for bit the
eager result.  The inputs are series whose orders fall off from the twisted vacuum, so the
fit chooses a nonzero exponent (checked against the unscaled result)."""
import numpy as np
import pytest
import torch

import nspt_synth as syn

from tests.gpu_util import dev, host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nspt():
    import paper_2001_02835_b300 as n
    assert n.lib().nspt_init() == 0
    return n


def decaying_links(L, flux, T, streams, seed):
    """Twist eaters at order 0 and orders k >= 1 falling off like 8^-k (Gaussian, variance 1/N)."""
    g = syn.rng(seed)
    U = syn.link_series(g, L, flux, T, streams)
    U[:, :, 1:] *= (8.0 ** -np.arange(1, T + 1))[None, None, :, None, None]
    return U


@pytest.mark.parametrize("prec", ["fp64", "split"])
def test_langevin_step_with_fitted_rescale_replays_in_a_graph(nspt, prec):
    L, flux, T = 3, 1, 15
    N = L * L
    U0 = dev(decaying_links(L, flux, T, 2, 9600))
    eta = dev(np.ascontiguousarray(syn.md_momenta(syn.rng(9601), N, 2)))
    kw = dict(algo="fft", prec=prec, rescale_log2r=nspt.RESCALE_AUTO)
    Ue = U0.clone()
    nspt.tek_langevin_step(Ue, eta, flux, 0.01, **kw)
    U0r = U0.clone()
    nspt.tek_langevin_step(U0r, eta, flux, 0.01, algo="fft", prec=prec, rescale_log2r=0)
    assert not torch.equal(Ue, U0r)          # the fit picked a nonzero exponent
    Ug = U0.clone()
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        nspt.tek_langevin_step(Ug, eta, flux, 0.01, **kw)
    Ug.copy_(U0)
    graph.replay()
    torch.cuda.synchronize()
    np.testing.assert_array_equal(host(Ug), host(Ue))


@pytest.mark.parametrize("prec", ["fp64", "split"])
def test_md_trajectory_with_fitted_rescale_replays_in_a_graph(nspt, prec):
    L, flux, T, nsteps = 3, 1, 15, 3
    N = L * L
    U0 = dev(decaying_links(L, flux, T, 1, 9700))
    eta = dev(np.ascontiguousarray(syn.md_momenta(syn.rng(9701), N, 1)))
    kw = dict(algo="fft", prec=prec, rescale_log2r=nspt.RESCALE_AUTO)
    Ue, Pe = U0.clone(), torch.zeros_like(U0)
    nspt.tek_md_trajectory(Ue, Pe, flux, 0.02, nsteps, eta=eta, **kw)
    Ug, Pg = U0.clone(), torch.zeros_like(U0)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        nspt.tek_md_trajectory(Ug, Pg, flux, 0.02, nsteps, eta=eta, **kw)
    for _ in range(2):                       # replays from the same start give the same result
        Ug.copy_(U0)
        Pg.zero_()
        graph.replay()
        torch.cuda.synchronize()
        np.testing.assert_array_equal(host(Ug), host(Ue))
        np.testing.assert_array_equal(host(Pg), host(Pe))


@pytest.mark.parametrize("prec", ["fp64", "split"])
def test_fitted_rescale_degenerate_inputs(nspt, prec):
    """All-zero series, a single order (T = 0) and one nonzero order: the device fit has fewer
    than two orders to fit and keeps r = 1; the products stay exact zeros or match the
    fixed-rescale result bit for bit."""
    z = torch.zeros((2, 8, 5, 5), dtype=torch.complex128, device="cuda")
    C = nspt.polymat_mul(z, z, algo="fft", prec=prec, rescale_log2r=nspt.RESCALE_AUTO)
    assert torch.count_nonzero(C).item() == 0
    g = syn.rng(9900)
    for T in (0, 5):
        A = dev(syn.series_batch(g, 6, T, 2))
        B = dev(syn.series_batch(g, 6, T, 2))
        if T > 0:
            A[:, 1:] = 0          # only order 0 nonzero in A: one usable order
        ca = nspt.polymat_mul(A, B, algo="fft", prec=prec, rescale_log2r=nspt.RESCALE_AUTO)
        c0 = nspt.polymat_mul(A, B, algo="fft", prec=prec, rescale_log2r=0)
        np.testing.assert_array_equal(host(ca), host(c0))


@pytest.mark.parametrize("prec", ["fp64", "split"])
def test_wilson_loops_and_projection_with_fitted_rescale_replay_in_a_graph(nspt, prec):
    """Every product of the Wilson-loop measurement and of the unitarity projection (U(1) phase
    included) fits its rescale on the device, so both calls capture and replay bit for bit."""
    L, flux, T = 3, 1, 12
    U0 = dev(decaying_links(L, flux, T, 1, 9800))
    kw = dict(algo="fft", prec=prec, rescale_log2r=nspt.RESCALE_AUTO)
    We = nspt.tek_wilson_loops(U0, flux, 2, **kw)
    Ve = U0.clone()
    nspt.tek_unitarize(Ve, special=True, **kw)
    Ug = U0.clone()
    Vg = U0.clone()
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        Wg = nspt.tek_wilson_loops(Ug, flux, 2, **kw)
        nspt.tek_unitarize(Vg, special=True, **kw)
    Vg.copy_(U0)
    graph.replay()
    torch.cuda.synchronize()
    np.testing.assert_array_equal(host(Wg), host(We))
    np.testing.assert_array_equal(host(Vg), host(Ve))
