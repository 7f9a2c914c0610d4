"""GPU parity of the naive form (Eq. 5) on the split-precision tensor cores: every
order of A and B sliced once from FP64, one tcgen05 GEMM per pair (l, k - l),
summed over l in double-float, against the FP64 oracle.

Bound: the product bound of the split form (tests/gpu_util.py).  Each GEMM carries
its own operands' row and column exponents, so its error is relative to its own
pair's size, not to the largest order as in a mode product; the stated bound is
the same and, as there, the result with one slice fewer must fail it.
"""
import numpy as np
import pytest
import torch

import nspt_synth as syn
from oracle import polymat as pm

from tests.gpu_util import dev, host, max_order_rel, record, split_bound

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nspt():
    import paper_2001_02835_b300 as n
    assert n.lib().nspt_init() == 0
    return n


def naive_split(nspt, A, B, C=None, **kw):
    return nspt.polymat_mul(A, B, C, algo="naive", prec="split", **kw)


# (N, T, batch): ragged N against the 128 x 48 tile and the 16-wide K steps; T = 0 is the
# single pair; T = 15 has 136 pairs in 8 launches
NAIVE_CASES = [(1, 0, 1), (3, 2, 2), (9, 8, 4), (33, 15, 2), (48, 7, 1), (130, 5, 1), (225, 3, 1),
               (600, 1, 1),
               # the largest split size; the largest truncation order (129 launches); T = 63
               (1024, 1, 1), (3, 255, 1), (10, 63, 3)]


@pytest.mark.parametrize("N,T,batch", NAIVE_CASES)
def test_naive_split_matches_oracle(nspt, N, T, batch):
    g = syn.rng(8100 + N + 100 * T)
    A = syn.series_batch(g, N, T, batch)
    B = syn.series_batch(g, N, T, batch)
    tA, tB = dev(A), dev(B)
    ref = pm.star(A, B)
    errs = {}
    for S in (6, 5):
        errs[S] = max_order_rel(host(naive_split(nspt, tA, tB, slices=S)), ref)
    record("naive_split", N=N, T=T, batch=batch, err_S6=errs[6], err_S5=errs[5])
    assert errs[6] <= split_bound(6), errs
    assert errs[5] <= split_bound(5), errs
    if N >= 9:
        assert errs[5] > split_bound(6), errs      # one slice fewer fails the bound


def test_naive_split_integer_inputs_exact(nspt):
    """Small integer coefficients are one digit each and every partial sum is a small
    integer, so the split naive product is exact."""
    g = syn.rng(8200)
    N, T = 11, 7
    A = syn.integer_series(g, N, T, 2)
    B = syn.integer_series(g, N, T, 2)
    C = host(naive_split(nspt, dev(A), dev(B)))
    np.testing.assert_array_equal(C, pm.star(A, B))


def test_naive_split_rescale_is_an_exact_shift(nspt):
    """The per-order rescale of the naive split form only shifts the slices' exponents
    (order k by k log2r) and undoes it on the FP64 output: for a series whose products
    stay in the FP32 range every log2r gives the same bits, the fitted one included."""
    g = syn.rng(8300)
    N, T, batch = 17, 31, 2
    A = syn.series_batch(g, N, T, batch)
    B = syn.series_batch(g, N, T, batch)
    w = 2.0 ** np.arange(T + 1)[None, :, None, None]
    A, B = A * w, B / w ** 0.5
    tA, tB = dev(A), dev(B)
    C0 = host(naive_split(nspt, tA, tB, rescale_log2r=0))
    for lr in (-1, 3, nspt.RESCALE_AUTO):
        np.testing.assert_array_equal(host(naive_split(nspt, tA, tB, rescale_log2r=lr)), C0)
    assert max_order_rel(C0, pm.star(A, B)) <= split_bound(6)


def test_naive_split_fitted_rescale_beyond_fp32_range(nspt):
    """A_k, B_k ~ 8^k: C_31 ~ 2^186 is outside the FP32 range of the double-float
    accumulator unless the orders are rescaled; the fitted rescale brings it back."""
    g = syn.rng(8400)
    N, T = 13, 31
    A = syn.series_batch(g, N, T, 1)
    B = syn.series_batch(g, N, T, 1)
    w = 8.0 ** np.arange(T + 1)[None, :, None, None]
    A, B = A * w, B * w
    C = host(naive_split(nspt, dev(A), dev(B), rescale_log2r=nspt.RESCALE_AUTO))
    assert np.isfinite(C).all()
    assert max_order_rel(C, pm.star(A, B)) <= split_bound(6)


def test_naive_split_many_problems_per_launch(nspt):
    """batch 40: a launch gets 120 or 80 batched GEMMs, more than the 64 problems one launch takes."""
    g = syn.rng(8500)
    N, T, batch = 5, 3, 40
    A = syn.series_batch(g, N, T, batch)
    B = syn.series_batch(g, N, T, batch)
    C = host(naive_split(nspt, dev(A), dev(B)))
    assert max_order_rel(C, pm.star(A, B)) <= split_bound(6)


def test_naive_split_graph_replay_and_determinism(nspt):
    """Bit-reproducible, and bit for bit the same when replayed from a captured CUDA graph."""
    g = syn.rng(8600)
    N, T, batch = 40, 9, 2
    tA = dev(syn.series_batch(g, N, T, batch))
    tB = dev(syn.series_batch(g, N, T, batch))
    C1 = host(naive_split(nspt, tA, tB, rescale_log2r=nspt.RESCALE_AUTO))
    np.testing.assert_array_equal(host(naive_split(nspt, tA, tB, rescale_log2r=nspt.RESCALE_AUTO)), C1)
    Cg = torch.zeros_like(tA)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        naive_split(nspt, tA, tB, Cg, rescale_log2r=nspt.RESCALE_AUTO)
    graph.replay()
    np.testing.assert_array_equal(host(Cg), C1)


def test_naive_split_su225_t31_full_oracle(nspt):
    """SU(225), O(g^31), batch 4 (the FP64 timing point of the paper, here in the naive
    split form): every entry of every order against the oracle's DFT-CONV."""
    g = syn.rng(8700)
    N, T, batch = 225, 31, 4
    A = syn.series_batch(g, N, T, batch)
    B = syn.series_batch(g, N, T, batch)
    C = host(naive_split(nspt, dev(A), dev(B)))
    err = max_order_rel(C, pm.star_dftconv(A, B))
    record("naive_split_su225_t31", err=err)
    assert err <= split_bound(6), err


# ---- the backward (truncated correlations) of the naive split form ----

BWD_CASES = [(1, 0, 1), (3, 2, 2), (9, 8, 4), (33, 15, 2), (130, 5, 1), (10, 63, 2)]


@pytest.mark.parametrize("N,T,batch", BWD_CASES)
def test_naive_split_backward_matches_oracle(nspt, N, T, batch):
    g = syn.rng(8800 + N + 100 * T)
    A = syn.series_batch(g, N, T, batch)
    B = syn.series_batch(g, N, T, batch)
    G = syn.gaussian(g, A.shape, 1.0)
    rA, rB = pm.star_backward(A, B, G)
    tA, tB, tG = dev(A), dev(B), dev(G)
    errs = {}
    for S in (6, 5):
        gA, gB = nspt.polymat_mul_backward(tA, tB, tG, algo="naive", prec="split", slices=S)
        errs[S] = max(max_order_rel(host(gA), rA), max_order_rel(host(gB), rB))
    record("naive_split_backward", N=N, T=T, batch=batch, err_S6=errs[6], err_S5=errs[5])
    assert errs[6] <= split_bound(6, "backward"), errs
    if N >= 9:
        assert errs[5] > split_bound(6, "backward"), errs


def test_naive_split_backward_single_outputs_and_rescale_shift(nspt):
    """gA alone and gB alone equal the pair; a fixed rescale only shifts exponents, so every
    log2r gives the same bits."""
    g = syn.rng(8900)
    N, T, batch = 21, 15, 2
    A = syn.series_batch(g, N, T, batch)
    B = syn.series_batch(g, N, T, batch)
    G = syn.gaussian(g, A.shape, 1.0)
    tA, tB, tG = dev(A), dev(B), dev(G)
    kw = dict(algo="naive", prec="split")
    gA, gB = nspt.polymat_mul_backward(tA, tB, tG, **kw)
    assert torch.equal(nspt.polymat_mul_backward(tA, tB, tG, need_gB=False, **kw)[0], gA)
    assert torch.equal(nspt.polymat_mul_backward(tA, tB, tG, need_gA=False, **kw)[1], gB)
    for lr in (-2, 3):
        gA2, gB2 = nspt.polymat_mul_backward(tA, tB, tG, rescale_log2r=lr, **kw)
        assert torch.equal(gA2, gA) and torch.equal(gB2, gB)


def test_naive_split_backward_su225_t31_full_oracle(nspt):
    """SU(225), O(g^31), one pair: every entry of gA and gB against the oracle's sums."""
    g = syn.rng(9000)
    N, T = 225, 31
    A = syn.series_batch(g, N, T, 1)
    B = syn.series_batch(g, N, T, 1)
    G = syn.gaussian(g, A.shape, 1.0)
    gA, gB = nspt.polymat_mul_backward(dev(A), dev(B), dev(G), algo="naive", prec="split")
    rA, rB = pm.star_backward(A, B, G)
    err = max(max_order_rel(host(gA), rA), max_order_rel(host(gB), rB))
    record("naive_split_backward_su225_t31", err=err)
    assert err <= split_bound(6, "backward"), err


def test_naive_split_host_product(nspt):
    """The host-memory product (pinned series, device slots) in the naive split form."""
    g = syn.rng(9100)
    N, T, batch = 17, 9, 3
    A = syn.series_batch(g, N, T, batch)
    B = syn.series_batch(g, N, T, batch)
    hA = torch.from_numpy(A).pin_memory()
    hB = torch.from_numpy(B).pin_memory()
    C = nspt.polymat_mul_host(hA, hB, algo="naive", prec="split")
    torch.cuda.synchronize()
    assert max_order_rel(C.numpy(), pm.star(A, B)) <= split_bound(6)
