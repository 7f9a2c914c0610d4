"""Seeded random sizes through the product forms on the GPU: N from 1 to 300 (ragged tiles of
every kind), T from 0 to 100 (mode counts 2 to 256, T + 1 near and away from powers of two),
batch 1 to 3.  The FFT forms are checked against the naive FP64 form (Eq. 5, no order mixing),
whose own parity with the oracle the other tests pin."""
import math

import numpy as np
import pytest

import nspt_synth as syn

from tests.gpu_util import dev, host, max_order_rel

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
    assert max_order_rel(Cs, ref) <= 2.0 ** 10 * math.sqrt(N) * (2.0 ** -47 + 2.0 ** -44)
