"""Products of host-resident series (nspt_polymat_mul_host): the pipelined copies and
products give the same C as the device-buffer product, for odd and even batches and
on calls in a row that reuse the device slots."""
import numpy as np
import pytest
import torch

import nspt_synth as syn
from oracle import polymat as pm

from tests.gpu_util import dev, host, max_order_rel, split_bound

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nspt():
    import paper_2001_02835_b300 as n
    assert n.lib().nspt_init() == 0
    return n


@pytest.mark.parametrize("prec", ["fp64", "split"])
@pytest.mark.parametrize("N,T,batch", [(9, 8, 1), (33, 15, 3), (40, 7, 5), (225, 15, 4)])
def test_host_product_equals_device_product(nspt, prec, N, T, batch):
    g = syn.rng(7400 + N + batch)
    outs = []
    for rep in range(2):   # two calls in a row through the same device slots
        A = syn.series_batch(g, N, T, batch)
        B = syn.series_batch(g, N, T, batch)
        hA = torch.from_numpy(A).pin_memory()
        hB = torch.from_numpy(B).pin_memory()
        hC = torch.full_like(hA, float("nan")).pin_memory()
        nspt.polymat_mul_host(hA, hB, hC, algo="fft", prec=prec)
        ref = host(nspt.polymat_mul(dev(A), dev(B), algo="fft", prec=prec))
        outs.append((hC, ref))
    torch.cuda.synchronize()
    for hC, ref in outs:
        if prec == "fp64":
            np.testing.assert_array_equal(hC.numpy(), ref)
        else:  # the tile width may differ between the batched and the per-element launch
            assert np.abs(hC.numpy() - ref).max() <= 1e-12 * np.abs(ref).max()


def test_host_product_with_fitted_rescale(nspt):
    """The fitted rescale in the host product is fitted per batch element on the device:
    a series whose orders grow as 4^k stays within the split bound per order."""
    g = syn.rng(2600)
    N, T, batch = 20, 15, 3
    w = 4.0 ** np.arange(T + 1)[None, :, None, None]
    A = syn.series_batch(g, N, T, batch) * w
    B = syn.series_batch(g, N, T, batch) * w
    for algo in ("fft", "naive"):
        C = nspt.polymat_mul_host(torch.from_numpy(A).pin_memory(), torch.from_numpy(B).pin_memory(), algo=algo,
                                  prec="split", rescale_log2r=nspt.RESCALE_AUTO)
        torch.cuda.synchronize()
        assert max_order_rel(C.numpy(), pm.star(A, B)) <= split_bound(6), algo


def test_host_product_3m_matches_device_product(nspt):
    """The host-memory product with three real products per complex product (3M)."""
    g = syn.rng(2700)
    N, T, batch = 33, 7, 3
    A = syn.series_batch(g, N, T, batch)
    B = syn.series_batch(g, N, T, batch)
    kw = dict(algo="fft", prec="split", complex_mode=3)
    C = nspt.polymat_mul_host(torch.from_numpy(A).pin_memory(), torch.from_numpy(B).pin_memory(), **kw)
    torch.cuda.synchronize()
    ref = host(nspt.polymat_mul(dev(A), dev(B), **kw))
    assert np.abs(C.numpy() - ref).max() <= 1e-12 * np.abs(ref).max()
    assert max_order_rel(C.numpy(), pm.star(A, B)) <= split_bound(6, "product3m")
