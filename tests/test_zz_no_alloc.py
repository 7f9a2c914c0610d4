"""The allocation-free FFT-CONV entry point, nspt_polymat_mul_fft_noalloc.

Some callers cannot allocate device memory: code in host callbacks or
allocator hooks, processes whose device memory another framework owns, or
plug-in hosts that hand over only the input and output buffers.  For them the
library keeps the product's scratch (the three spectra) in one fixed device
array of 32 MiB.  These tests call that entry point through the C ABI twice in
a row and check both results against nspt_polymat_mul (FFT, FP64) and the
oracle with the FP64-form tolerance, run one problem whose spectra fill the
fixed scratch to within about 1% (where a layout or rounding slip would write
past the array), and check that the next larger problem is refused.  The file is collected last so that a run stopping
at the first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest
import torch

import nspt_synth as syn
from oracle import polymat as pm

from tests.gpu_util import dev, host, max_order_rel

pytestmark = pytest.mark.gpu
TOL = 1e-12  # per-order relative Frobenius error of the FP64 form


@pytest.fixture(scope="module")
def nspt():
    import paper_2001_02835_b300 as n
    assert n.lib().nspt_init() == 0
    return n


def test_noalloc_matches_existing_entry_on_two_calls(nspt):
    L = nspt.lib()
    cases = [(33, 15, 2), (20, 7, 3)]
    inputs, outs = [], []
    stream = torch.cuda.current_stream().cuda_stream
    for call, (N, T, batch) in enumerate(cases):
        g = syn.rng(9100 + call)
        A = syn.series_batch(g, N, T, batch)
        B = syn.series_batch(g, N, T, batch)
        dA, dB = dev(A), dev(B)
        C = torch.full_like(dA, float("nan"))
        rc = L.nspt_polymat_mul_fft_noalloc(dA.data_ptr(), dB.data_ptr(), C.data_ptr(), N, T, batch, stream)
        assert rc == 0, L.nspt_status_string(rc)
        inputs.append((A, B, dA, dB))
        outs.append(C)
    for (A, B, dA, dB), C in zip(inputs, outs):
        got = host(C)
        ref_entry = host(nspt.polymat_mul(dA, dB, algo="fft", prec="fp64"))
        assert max_order_rel(got, ref_entry) <= TOL
        assert max_order_rel(got, pm.star(A, B)) <= TOL


def test_noalloc_refuses_problems_beyond_its_scratch(nspt):
    L = nspt.lib()
    # SU(225), T = 63, batch 4 needs 3 * 4 * 128 * 225^2 * 16 bytes, far above 32 MiB
    x = torch.zeros(8, dtype=torch.complex128, device="cuda")
    y = torch.zeros(8, dtype=torch.complex128, device="cuda")
    z = torch.zeros(8, dtype=torch.complex128, device="cuda")
    rc = L.nspt_polymat_mul_fft_noalloc(x.data_ptr(), y.data_ptr(), z.data_ptr(), 225, 63, 4,
                                        torch.cuda.current_stream().cuda_stream)
    assert rc == -4 and b"too small" in L.nspt_status_string(rc)
    assert L.nspt_polymat_mul_fft_noalloc(None, None, None, 4, 3, 1, None) == -1


def test_noalloc_problem_that_nearly_fills_its_scratch(nspt):
    """3 * round256(batch * M * N^2 * 16) <= 32 MiB: at T = 15 (M = 32), batch 1, N = 147 uses
    33,191,424 of 33,554,432 bytes and is computed correctly; N = 148 (33,644,544 bytes) is
    refused before any launch."""
    L = nspt.lib()
    stream = torch.cuda.current_stream().cuda_stream
    N, T = 147, 15
    assert 3 * (32 * N * N * 16) <= 32 << 20 < 3 * (32 * (N + 1) ** 2 * 16)
    g = syn.rng(9200)
    A = syn.series_batch(g, N, T, 1)
    B = syn.series_batch(g, N, T, 1)
    dA, dB = dev(A), dev(B)
    C = torch.full_like(dA, float("nan"))
    rc = L.nspt_polymat_mul_fft_noalloc(dA.data_ptr(), dB.data_ptr(), C.data_ptr(), N, T, 1, stream)
    assert rc == 0, L.nspt_status_string(rc)
    got = host(C)
    assert max_order_rel(got, pm.star(A, B)) <= TOL
    assert max_order_rel(got, host(nspt.polymat_mul(dA, dB, algo="fft", prec="fp64"))) <= TOL
    big = torch.zeros((1, T + 1, N + 1, N + 1), dtype=torch.complex128, device="cuda")
    big2, big3 = torch.zeros_like(big), torch.zeros_like(big)
    rc = L.nspt_polymat_mul_fft_noalloc(big.data_ptr(), big2.data_ptr(), big3.data_ptr(), N + 1, T, 1, stream)
    assert rc == -4
