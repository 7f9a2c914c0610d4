"""Guard-region (canary) tests of every entry point: outputs, in-place series, inputs and
the workspace each sit inside one device allocation with 64 KiB of a fixed byte pattern
before and after them.  After the call the guards must be intact (no write outside a
buffer or past the workspace size the library asked for), the inputs unchanged, and the
outputs equal to those of a plain call (so every output entry was written).

Every access stays inside the allocations: a stray write lands in a guard, not in another
buffer, so these tests cannot fault the GPU.  Sizes are ragged against the tiles (N = 13,
130), small enough to run in seconds."""
import ctypes

import numpy as np
import pytest
import torch

import nspt_synth as syn

pytestmark = pytest.mark.gpu

GUARD = 1 << 16
PAT = 0xA5


@pytest.fixture(scope="module")
def nspt():
    import paper_2001_02835_b300 as n
    assert n.lib().nspt_init() == 0
    return n


class Guarded:
    """`nbytes` of device memory with GUARD pattern bytes on both sides."""

    def __init__(self, nbytes: int):
        self.n = int(nbytes)
        self.buf = torch.full((self.n + 2 * GUARD,), PAT, dtype=torch.uint8, device="cuda")

    @property
    def ptr(self) -> int:
        return self.buf.data_ptr() + GUARD

    def tensor(self, shape, dtype=torch.complex128) -> torch.Tensor:
        return self.buf[GUARD:GUARD + self.n].view(dtype).view(shape)

    def intact(self) -> bool:
        torch.cuda.synchronize()
        return bool((self.buf[:GUARD] == PAT).all()) and bool((self.buf[GUARD + self.n:] == PAT).all())


def guarded_copy(x: np.ndarray) -> Guarded:
    g = Guarded(x.nbytes)
    g.tensor(x.shape).copy_(torch.from_numpy(np.ascontiguousarray(x)))
    return g


def guarded_out(shape) -> Guarded:
    return Guarded(int(np.prod(shape)) * 16)


def guarded_ws(nspt, nbytes: int, opts):
    g = Guarded(max(int(nbytes), 1))
    opts.workspace = g.ptr
    opts.workspace_bytes = int(nbytes)
    return g


def check_inputs(pairs):
    for g, x in pairs:
        assert g.intact()
        np.testing.assert_array_equal(g.tensor(x.shape).cpu().numpy(), x)


PRODUCT_FORMS = [dict(algo="naive", prec="fp64"), dict(algo="fft", prec="fp64"),
                 dict(algo="naive", prec="split"), dict(algo="fft", prec="split"),
                 dict(algo="fft", prec="split", complex_mode=3)]


@pytest.mark.parametrize("N,T,batch", [(13, 5, 2), (130, 3, 1)])
@pytest.mark.parametrize("kw", PRODUCT_FORMS, ids=lambda k: "-".join(str(v) for v in k.values()))
def test_product_and_backward_stay_in_bounds(nspt, kw, N, T, batch):
    L = nspt.lib()
    g = syn.rng(9500 + N)
    A = syn.series_batch(g, N, T, batch)
    B = syn.series_batch(g, N, T, batch)
    gA_, gB_ = guarded_copy(A), guarded_copy(B)
    C = guarded_out(A.shape)
    opts = nspt.make_opts(**kw)
    ws = guarded_ws(nspt, L.nspt_workspace_size(nspt.OP_MUL, N, T, batch, ctypes.byref(opts)), opts)
    assert L.nspt_polymat_mul(gA_.ptr, gB_.ptr, C.ptr, N, T, batch, ctypes.byref(opts), None) == 0
    assert C.intact() and ws.intact()
    check_inputs([(gA_, A), (gB_, B)])
    ref = nspt.polymat_mul(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), **kw)
    assert torch.equal(C.tensor(A.shape), ref)
    if kw.get("complex_mode") == 3:
        return                                    # the 3M variant is for products only
    G = syn.gaussian(g, A.shape, 1.0)
    gG = guarded_copy(G)
    oA, oB = guarded_out(A.shape), guarded_out(A.shape)
    opts = nspt.make_opts(**kw)
    ws = guarded_ws(nspt, L.nspt_workspace_size(nspt.OP_MUL_BACKWARD, N, T, batch, ctypes.byref(opts)), opts)
    assert L.nspt_polymat_mul_backward(gA_.ptr, gB_.ptr, gG.ptr, oA.ptr, oB.ptr, N, T, batch,
                                       ctypes.byref(opts), None) == 0
    assert oA.intact() and oB.intact() and ws.intact()
    check_inputs([(gA_, A), (gB_, B), (gG, G)])
    rA, rB = nspt.polymat_mul_backward(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(),
                                       torch.from_numpy(G).cuda(), **kw)
    assert torch.equal(oA.tensor(A.shape), rA) and torch.equal(oB.tensor(A.shape), rB)


TEK_FORMS = [dict(algo="naive", prec="fp64"), dict(algo="fft", prec="fp64"), dict(algo="fft", prec="split")]


@pytest.mark.parametrize("kw", TEK_FORMS, ids=lambda k: "-".join(str(v) for v in k.values()))
def test_tek_entry_points_stay_in_bounds(nspt, kw):
    L = nspt.lib()
    Lx, flux, T, batch = 3, 1, 4, 2
    N = Lx * Lx
    g = syn.rng(9600)
    U = syn.link_series(g, Lx, flux, T, batch)
    eta = syn.hermitian_noise(g, N, batch * 4).reshape(batch, 4, N, N)
    # Langevin step: U in place, eta input, F output
    gU, gE, gF = guarded_copy(U), guarded_copy(eta), guarded_out(U.shape)
    opts = nspt.make_opts(**kw)
    ws = guarded_ws(nspt, L.nspt_workspace_size(nspt.OP_LANGEVIN, N, T, batch, ctypes.byref(opts)), opts)
    assert L.nspt_tek_langevin_step(gU.ptr, gE.ptr, gF.ptr, N, T, batch, flux, ctypes.c_double(0.01),
                                    ctypes.byref(opts), None) == 0
    assert gU.intact() and gF.intact() and ws.intact()
    check_inputs([(gE, eta)])
    rU, rF = nspt.tek_langevin_step(torch.from_numpy(U).cuda(), torch.from_numpy(eta).cuda(), flux, 0.01,
                                    want_drift=True, **kw)
    assert torch.equal(gU.tensor(U.shape), rU) and torch.equal(gF.tensor(U.shape), rF)
    # MD trajectory: U, P in place, eta (refresh) input
    gU, gP, gE = guarded_copy(U), guarded_out(U.shape), guarded_copy(eta)
    gP.tensor(U.shape).zero_()
    opts = nspt.make_opts(**kw)
    ws = guarded_ws(nspt, L.nspt_workspace_size(nspt.OP_MD, N, T, batch, ctypes.byref(opts)), opts)
    assert L.nspt_tek_md_trajectory(gU.ptr, gP.ptr, gE.ptr, N, T, batch, flux, ctypes.c_double(0.02), 2,
                                    ctypes.byref(opts), None) == 0
    assert gU.intact() and gP.intact() and ws.intact()
    check_inputs([(gE, eta)])
    # Wilson loops: U input, W output
    gU = guarded_copy(U)
    amax = 2
    W = Guarded(batch * amax * amax * (T + 1) * 16)
    opts = nspt.make_opts(**kw)
    ws = guarded_ws(nspt, L.nspt_workspace_size_wilson(N, T, batch, amax, ctypes.byref(opts)), opts)
    assert L.nspt_tek_wilson_loops(gU.ptr, N, T, batch, flux, amax, W.ptr, ctypes.byref(opts), None) == 0
    assert W.intact() and ws.intact()
    check_inputs([(gU, U)])
    rW = nspt.tek_wilson_loops(torch.from_numpy(U).cuda(), flux, amax, **kw)
    assert torch.equal(W.tensor(tuple(rW.shape)), rW)
    # unitarity projection with the U(1) phase: U in place
    gU = guarded_copy(U)
    opts = nspt.make_opts(**kw)
    ws = guarded_ws(nspt, L.nspt_workspace_size(nspt.OP_UNITARIZE, N, T, batch, ctypes.byref(opts)), opts)
    assert L.nspt_tek_unitarize(gU.ptr, N, T, batch, 1, ctypes.byref(opts), None) == 0
    assert gU.intact() and ws.intact()


def test_grouped_and_noise_stay_in_bounds(nspt):
    L = nspt.lib()
    g = syn.rng(9700)
    shapes = [(13, 5), (33, 2), (130, 3)]
    As = [syn.series_batch(g, N, T, 1) for N, T in shapes]
    Bs = [syn.series_batch(g, N, T, 1) for N, T in shapes]
    gAs, gBs = [guarded_copy(a) for a in As], [guarded_copy(b) for b in Bs]
    gCs = [guarded_out(a.shape) for a in As]
    arr = (nspt.PolymatDesc * len(As))()
    for i, (N, T) in enumerate(shapes):
        arr[i] = nspt.PolymatDesc(gAs[i].ptr, gBs[i].ptr, gCs[i].ptr, N, T, 1)
    opts = nspt.make_opts(algo="fft", prec="split")
    ws = guarded_ws(nspt, L.nspt_workspace_size_grouped(arr, len(As), ctypes.byref(opts)), opts)
    assert L.nspt_polymat_mul_grouped(arr, len(As), ctypes.byref(opts), None) == 0
    assert ws.intact() and all(c.intact() for c in gCs)
    check_inputs(list(zip(gAs, As)) + list(zip(gBs, Bs)))
    for i, (A, B) in enumerate(zip(As, Bs)):
        ref = nspt.polymat_mul(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), algo="fft", prec="split")
        assert torch.equal(gCs[i].tensor(A.shape), ref)
    # seeded noise: output and the device counter word
    N, count = 13, 5
    E = guarded_out((count, N, N))
    ctr = Guarded(8)
    ctr.tensor((1,), torch.int64).zero_()
    assert L.nspt_tek_noise(E.ptr, N, count, 3, 0, ctr.ptr, None) == 0
    assert E.intact() and ctr.intact()
    assert int(ctr.tensor((1,), torch.int64).item()) == 1
    assert torch.equal(E.tensor((count, N, N)), nspt.tek_noise(N, count, 3, 0))


def test_naive_split_wilson_and_projection_stay_in_bounds(nspt):
    """The Wilson loops and the unitarity projection on the naive split products."""
    L = nspt.lib()
    Lx, flux, T, batch, amax = 3, 1, 4, 2, 2
    N = Lx * Lx
    U = syn.link_series(syn.rng(9800), Lx, flux, T, batch)
    kw = dict(algo="naive", prec="split")
    gU = guarded_copy(U)
    W = Guarded(batch * amax * amax * (T + 1) * 16)
    opts = nspt.make_opts(**kw)
    ws = guarded_ws(nspt, L.nspt_workspace_size_wilson(N, T, batch, amax, ctypes.byref(opts)), opts)
    assert L.nspt_tek_wilson_loops(gU.ptr, N, T, batch, flux, amax, W.ptr, ctypes.byref(opts), None) == 0
    assert W.intact() and ws.intact()
    check_inputs([(gU, U)])
    rW = nspt.tek_wilson_loops(torch.from_numpy(U).cuda(), flux, amax, **kw)
    assert torch.equal(W.tensor(tuple(rW.shape)), rW)
    opts = nspt.make_opts(**kw)
    ws = guarded_ws(nspt, L.nspt_workspace_size(nspt.OP_UNITARIZE, N, T, batch, ctypes.byref(opts)), opts)
    assert L.nspt_tek_unitarize(gU.ptr, N, T, batch, 1, ctypes.byref(opts), None) == 0
    assert gU.intact() and ws.intact()
