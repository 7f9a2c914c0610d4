"""The C-ABI library loads and exports every symbol include/nspt.h declares;
host-side argument checks answer without touching a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    src = open(os.path.join(ROOT, "include", "nspt.h")).read()
    return sorted(set(re.findall(r"NSPT_API\s+[\w\s\*]+?\b(nspt_\w+)\s*\(", src)))


@pytest.fixture(scope="module")
def L():
    import paper_2001_02835_b300 as n
    return n.lib()


def test_every_declared_symbol_is_exported(L):
    syms = _declared_symbols()
    assert len(syms) >= 10
    for s in syms:
        assert hasattr(L, s), s


def test_status_strings(L):
    assert L.nspt_status_string(0) == b"ok"
    assert b"workspace" in L.nspt_status_string(-4)
    assert L.nspt_status_string(-99) == b"unknown status"


def test_argument_checks_need_no_gpu(L):
    import paper_2001_02835_b300 as n
    o = n.make_opts()
    # NULL pointers / bad sizes are rejected on the host before any CUDA call
    assert L.nspt_polymat_mul(None, None, None, 4, 3, 1, ctypes.byref(o), None) == -1
    assert L.nspt_polymat_mul(1 << 20, 2 << 20, 3 << 20, 0, 3, 1, ctypes.byref(o), None) == -1
    assert L.nspt_polymat_mul(1 << 20, 2 << 20, 3 << 20, 4, -1, 1, ctypes.byref(o), None) == -1
    # an empty batch is refused, not treated as a no-op
    assert L.nspt_polymat_mul(1 << 20, 2 << 20, 3 << 20, 4, 3, 0, ctypes.byref(o), None) == -1
    assert L.nspt_polymat_mul_backward(1 << 20, 2 << 20, 3 << 20, 4 << 20, 5 << 20, 4, 3, 0, ctypes.byref(o),
                                       None) == -1
    # output overlapping an input
    assert L.nspt_polymat_mul(1 << 20, 1 << 24, (1 << 20) + 16, 4, 3, 1, ctypes.byref(o), None) == -2
    # FFT length not a power of two / too short for wrap-free convolution
    o2 = n.make_opts(algo="fft", fft_len=12)
    assert L.nspt_polymat_mul(1 << 20, 1 << 24, 1 << 28, 4, 3, 1, ctypes.byref(o2), None) == -1
    o3 = n.make_opts(algo="fft", fft_len=4)
    assert L.nspt_polymat_mul(1 << 20, 1 << 24, 1 << 28, 4, 3, 1, ctypes.byref(o3), None) == -1
    # FFT form without a workspace
    o4 = n.make_opts(algo="fft")
    assert L.nspt_polymat_mul(1 << 20, 1 << 24, 1 << 28, 4, 3, 1, ctypes.byref(o4), None) == -4
    # split form beyond the slicers' shared-memory rows
    o5 = n.make_opts(algo="fft", prec="split")
    assert L.nspt_polymat_mul(1 << 20, 1 << 34, 1 << 36, 1025, 3, 1, ctypes.byref(o5), None) == -3
    # Langevin: N must be L^2 with gcd(flux, L) = 1, eps > 0
    assert L.nspt_tek_langevin_step(1 << 20, 1 << 30, None, 10, 2, 1, 1, 0.01, ctypes.byref(o), None) == -1
    assert L.nspt_tek_langevin_step(1 << 20, 1 << 30, None, 9, 2, 1, 3, 0.01, ctypes.byref(o), None) == -1
    assert L.nspt_tek_langevin_step(1 << 20, 1 << 30, None, 9, 2, 1, 1, -0.01, ctypes.byref(o), None) == -1


def test_workspace_sizes(L):
    import paper_2001_02835_b300 as n
    naive = n.make_opts(algo="naive")
    assert n.workspace_size(0, 225, 31, 4, naive) == 0
    fft = n.make_opts(algo="fft")
    spec = 4 * 64 * 225 * 225 * 16
    assert n.workspace_size(0, 225, 31, 4, fft) >= 3 * spec
    assert n.workspace_size(1, 225, 31, 4, fft) >= 4 * spec
    assert n.workspace_size(0, 225, 31, 4, n.make_opts(algo="fft", fft_len=128)) >= 6 * spec


def test_complex_mode_plans_need_no_gpu(L):
    """complex_mode = 3 (3M) is planned for the split-form product only: its workspace holds a
    third slice plane of the left operand; every other combination is refused on the host."""
    import paper_2001_02835_b300 as n
    N, T, b = 225, 31, 4
    m4 = n.workspace_size(n.OP_MUL, N, T, b, n.make_opts(algo="fft", prec="split"))
    m3 = n.workspace_size(n.OP_MUL, N, T, b, n.make_opts(algo="fft", prec="split", complex_mode=3))
    kp = (N + 7) & ~7
    assert m3 - m4 >= b * 64 * 6 * N * kp * 2          # one more BF16 plane per slice and mode
    for kw in (dict(prec="fp64"), dict(prec="split", slices=7), dict(prec="split", complex_mode=2)):
        kw.setdefault("complex_mode", 3)
        assert n.workspace_size(n.OP_MUL, N, T, b, n.make_opts(algo="fft", **kw)) == 0
    assert n.workspace_size(n.OP_MUL, 513, 3, 1, n.make_opts(algo="fft", prec="split", complex_mode=3)) == 0
    o3 = n.make_opts(algo="fft", prec="split", complex_mode=3)
    assert n.workspace_size(n.OP_MUL_BACKWARD, N, T, b, o3) == 0
    assert L.nspt_polymat_mul_backward(1 << 20, 2 << 20, 3 << 20, 4 << 20, 5 << 20, N, T, b, ctypes.byref(o3),
                                       None) == -3
    assert L.nspt_polymat_mul(1 << 20, 1 << 34, 1 << 36, 513, 3, 1, ctypes.byref(o3), None) == -3
    # a valid 3M request without its workspace: the workspace check, not the plan, refuses it
    assert L.nspt_polymat_mul(1 << 20, 1 << 34, 1 << 36, N, T, b, ctypes.byref(o3), None) == -4


def test_naive_split_plans_need_no_gpu(L):
    """The naive form of the split products is planned for nspt_polymat_mul, its backward, the
    unitarity projection and the Wilson loops: the product workspace holds the slices of every
    order of both operands (2 and 3 BF16 planes per digit) and two double-float accumulators;
    the Langevin step and MD, and 3M, refuse it."""
    import paper_2001_02835_b300 as n
    N, T, b, S = 225, 31, 4, 6
    kp = (N + 7) & ~7
    Q = b * (T + 1)
    need = Q * S * 5 * N * kp * 2 + 2 * Q * N * N * 16     # two accumulators
    ws = n.workspace_size(n.OP_MUL, N, T, b, n.make_opts(algo="naive", prec="split"))
    assert need <= ws <= need + 2 * Q * N * 4 + 8 * 256
    assert n.workspace_size(n.OP_MUL, N, T, b, n.make_opts(algo="naive", prec="fp64")) == 0
    # the backward reuses the product's layout (its two operands' slices, two accumulators)
    assert n.workspace_size(n.OP_MUL_BACKWARD, N, T, b, n.make_opts(algo="naive", prec="split")) == ws
    for op in (n.OP_LANGEVIN, n.OP_MD):
        assert n.workspace_size(op, N, T, b, n.make_opts(algo="naive", prec="split")) == 0
    # the unitarity projection and the Wilson loops run all their products through the product call
    assert n.workspace_size(n.OP_UNITARIZE, N, T, b, n.make_opts(algo="naive", prec="split")) > ws
    assert L.nspt_workspace_size_wilson(N, T, b, 2, ctypes.byref(n.make_opts(algo="naive", prec="split"))) > ws
    o3 = n.make_opts(algo="naive", prec="split", complex_mode=3)
    assert n.workspace_size(n.OP_MUL, N, T, b, o3) == 0
    assert L.nspt_polymat_mul(1 << 20, 1 << 34, 1 << 36, N, T, b, ctypes.byref(o3), None) == -3
    on = n.make_opts(algo="naive", prec="split")
    # valid requests without their workspace: the workspace check refuses them
    assert L.nspt_polymat_mul(1 << 20, 1 << 34, 1 << 36, N, T, b, ctypes.byref(on), None) == -4
    assert L.nspt_polymat_mul_backward(1 << 20, 1 << 34, 1 << 36, 1 << 38, 1 << 40, N, T, b, ctypes.byref(on),
                                       None) == -4


def test_noise_argument_checks_need_no_gpu(L):
    """nspt_tek_noise refuses a NULL output and empty or oversized shapes on the host."""
    assert L.nspt_tek_noise(None, 9, 4, 1, 0, None, None) == -1
    assert L.nspt_tek_noise(1 << 20, 0, 4, 1, 0, None, None) == -1
    assert L.nspt_tek_noise(1 << 20, 4097, 4, 1, 0, None, None) == -1
    assert L.nspt_tek_noise(1 << 20, 9, 0, 1, 0, None, None) == -1


def test_argument_checks_of_md_wilson_and_host_product(L):
    import paper_2001_02835_b300 as n
    o = n.make_opts()
    # MD: NULL links, N not a square, gcd(flux, L) != 1, eps <= 0, negative steps, momentum aliasing links
    assert L.nspt_tek_md_trajectory(None, 1 << 30, None, 9, 2, 1, 1, 0.02, 4, ctypes.byref(o), None) == -1
    assert L.nspt_tek_md_trajectory(1 << 20, 1 << 30, None, 10, 2, 1, 1, 0.02, 4, ctypes.byref(o), None) == -1
    assert L.nspt_tek_md_trajectory(1 << 20, 1 << 30, None, 9, 2, 1, 3, 0.02, 4, ctypes.byref(o), None) == -1
    assert L.nspt_tek_md_trajectory(1 << 20, 1 << 30, None, 9, 2, 1, 1, 0.0, 4, ctypes.byref(o), None) == -1
    assert L.nspt_tek_md_trajectory(1 << 20, 1 << 30, None, 9, 2, 1, 1, 0.02, -1, ctypes.byref(o), None) == -1
    assert L.nspt_tek_md_trajectory(1 << 20, (1 << 20) + 16, None, 9, 2, 1, 1, 0.02, 4, ctypes.byref(o), None) == -2
    # Wilson loops: extent out of range, N not a square, gcd(flux, L) != 1, output overlapping the links
    assert L.nspt_tek_wilson_loops(1 << 20, 9, 2, 1, 1, 0, 1 << 30, ctypes.byref(o), None) == -1
    assert L.nspt_tek_wilson_loops(1 << 20, 9, 2, 1, 1, 9, 1 << 30, ctypes.byref(o), None) == -1
    assert L.nspt_tek_wilson_loops(1 << 20, 10, 2, 1, 1, 2, 1 << 30, ctypes.byref(o), None) == -1
    assert L.nspt_tek_wilson_loops(1 << 20, 9, 2, 1, 3, 2, 1 << 30, ctypes.byref(o), None) == -1
    assert L.nspt_tek_wilson_loops(1 << 20, 9, 2, 1, 1, 2, (1 << 20) + 16, ctypes.byref(o), None) == -2
    assert L.nspt_workspace_size_wilson(9, 2, 1, 0, ctypes.byref(o)) == 0
    assert L.nspt_workspace_size_wilson(9, 2, 1, 2, ctypes.byref(o)) > 0
    # host product: NULL buffers, C overlapping A, missing workspace (also with the fitted rescale)
    assert L.nspt_polymat_mul_host(None, 1 << 24, 1 << 28, 4, 3, 2, ctypes.byref(o), None) == -1
    assert L.nspt_polymat_mul_host(1 << 20, 1 << 24, (1 << 20) + 16, 4, 3, 2, ctypes.byref(o), None) == -2
    assert L.nspt_polymat_mul_host(1 << 20, 1 << 24, 1 << 28, 4, 3, 2, ctypes.byref(o), None) == -4
    auto = n.make_opts(algo="fft", prec="split", rescale_log2r=n.RESCALE_AUTO)
    assert L.nspt_polymat_mul_host(1 << 20, 1 << 24, 1 << 28, 4, 3, 2, ctypes.byref(auto), None) == -4
    # two slots of three series of one element, plus the product workspace of one element
    ser = 4 * 4 * 16
    assert L.nspt_workspace_size_host(4, 3, 2, ctypes.byref(o)) >= 6 * ser
