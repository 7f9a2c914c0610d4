"""Failure detection without a GPU fault: the bounded device-side waits of the tensor
GEMMs give up (forced through the test hook), the launch exits cleanly, the host reads
NSPT_ERR_TIMEOUT, and the context stays usable; buffers in the wrong kind of memory are
refused on the host before any launch."""
import ctypes

import numpy as np
import pytest
import torch

import nspt_synth as syn
from oracle import polymat as pm

from tests.gpu_util import dev, host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nspt():
    import paper_2001_02835_b300 as n
    assert n.lib().nspt_init() == 0
    return n


def _split_call(nspt, A, B, C, opts):
    return nspt.lib().nspt_polymat_mul(A.data_ptr(), B.data_ptr(), C.data_ptr(), A.shape[-1], A.shape[1] - 1,
                                       A.shape[0], ctypes.byref(opts), nspt._stream_ptr(A.device))


def test_forced_wait_timeout_is_reported_and_the_context_survives(nspt):
    g = syn.rng(7600)
    A, B = syn.series_batch(g, 40, 7, 2), syn.series_batch(g, 40, 7, 2)
    tA, tB = dev(A), dev(B)
    C = torch.empty_like(tA)
    opts = nspt.make_opts(algo="fft", prec="split")
    ws = nspt._with_ws(nspt.OP_MUL, 40, 7, 2, opts, tA.device)  # noqa: F841
    L = nspt.lib()
    try:
        assert L.nspt_debug_wait_budget(-1) == 0
        assert _split_call(nspt, tA, tB, C, opts) == 0                 # enqueued
        assert L.nspt_device_status(ctypes.byref(opts), nspt._stream_ptr(tA.device)) == -6
    finally:
        L.nspt_debug_wait_budget(2_000_000_000)
    # the next call runs normally on the same context and workspace
    assert _split_call(nspt, tA, tB, C, opts) == 0
    assert L.nspt_device_status(ctypes.byref(opts), nspt._stream_ptr(tA.device)) == 0
    ref = pm.star(A, B)
    assert np.abs(host(C) - ref).max() <= 1e-11 * np.abs(ref).max()


def test_buffers_in_the_wrong_memory_are_refused(nspt):
    g = syn.rng(7601)
    A = syn.series_batch(g, 9, 3, 1)
    hA = torch.from_numpy(A)                      # host memory
    dA = dev(A)
    opts = nspt.make_opts(algo="naive")           # naive FP64: needs no workspace
    st = nspt._stream_ptr(dA.device)
    L = nspt.lib()
    dC = torch.empty_like(dA)
    # a host pointer where device memory is expected
    assert L.nspt_polymat_mul(hA.data_ptr(), dA.data_ptr(), dC.data_ptr(), 9, 3, 1, ctypes.byref(opts), st) == -1
    # a device pointer where host memory is expected
    fopts = nspt.make_opts(algo="fft")
    ws = torch.empty(L.nspt_workspace_size_host(9, 3, 1, ctypes.byref(fopts)), dtype=torch.uint8, device="cuda")
    fopts.workspace, fopts.workspace_bytes = ws.data_ptr(), ws.numel()
    hC = torch.empty_like(hA)
    assert L.nspt_polymat_mul_host(dA.data_ptr(), hA.data_ptr(), hC.data_ptr(), 9, 3, 1, ctypes.byref(fopts),
                                   st) == -1
    # the same calls with the right memory succeed
    assert L.nspt_polymat_mul(dA.data_ptr(), dA.data_ptr(), dC.data_ptr(), 9, 3, 1, ctypes.byref(opts), st) == 0
    torch.cuda.synchronize()
    np.testing.assert_allclose(host(dC), pm.star(A, A), atol=1e-12 * np.abs(A).max() ** 2 * 10)
