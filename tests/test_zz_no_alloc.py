"""The allocation-free FFT-CONV entry point, nspt_polymat_mul_fft_noalloc.

Some callers cannot allocate device memory: code in host callbacks or
allocator hooks, processes whose device memory another framework owns, or
plug-in hosts that hand over only the input and output buffers.  For them the
library keeps the product's scratch (the three spectra) in one fixed device
array of 32 MiB.  These tests call that entry point through the C ABI twice in
a row and check both results against nspt_polymat_mul (FFT, FP64) and the
oracle with the FP64-form tolerance, and check that a problem too large for the
fixed scratch is refused.  The file is collected last so that a run stopping
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
