"""Stored fixtures under tests/golden: the paper's benchmark parameters (Sec. 3,
Table "Parameters") and an exact integer product (Eq. 5) written from the oracle
by tests/golden/make_golden.py.  The stored product is pinned here by exact
Python-integer arithmetic, independent of the oracle."""
import ctypes
import os

import numpy as np
import pytest

from oracle import polymat as pm

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load_star_fixture(name="star_integer_N3_T5.txt"):
    rows = {}
    for line in open(os.path.join(GOLDEN, name)):
        if not line.strip() or line.startswith("#"):
            continue
        tag, k, i, *vals = line.split()
        rows[(tag, int(k), int(i))] = [int(v) for v in vals]
    T = max(k for (_, k, _) in rows)
    N = max(i for (_, _, i) in rows) + 1
    out = {}
    for tag in "ABC":
        X = np.zeros((T + 1, N, N), np.complex128)
        for k in range(T + 1):
            for i in range(N):
                v = rows[(tag, k, i)]
                X[k, i] = np.array(v[0::2], np.float64) + 1j * np.array(v[1::2], np.float64)
        out[tag] = X
    return out["A"], out["B"], out["C"]


def load_parameters():
    table = {}
    for line in open(os.path.join(GOLDEN, "paper_parameters.txt")):
        if not line.strip() or line.startswith("#"):
            continue
        name, steps, ns, ts = line.split()
        table[name] = (int(steps), [int(x) for x in ns.split(",")], [int(x) for x in ts.split(",")])
    return table


def test_stored_product_is_the_exact_integer_product():
    A, B, C = load_star_fixture()
    T1, N = A.shape[0], A.shape[1]
    ai = [[[(int(z.real), int(z.imag)) for z in row] for row in m] for m in A]
    bi = [[[(int(z.real), int(z.imag)) for z in row] for row in m] for m in B]
    for k in range(T1):
        for i in range(N):
            for j in range(N):
                re = im = 0
                for l in range(k + 1):
                    for m in range(N):
                        (p, q), (r, s) = ai[l][i][m], bi[k - l][m][j]
                        re += p * r - q * s
                        im += p * s + q * r
                assert (re, im) == (int(C[k, i, j].real), int(C[k, i, j].imag)), (k, i, j)


def test_oracle_forms_reproduce_the_stored_product():
    A, B, C = load_star_fixture()
    T = A.shape[0] - 1
    assert np.array_equal(pm.star(A, B), C)
    # the DFT-CONV steps at the paper's length 2(T+1) and at the shortest wrap-free length 2T+1
    for M in (2 * (T + 1), 2 * T + 1):
        D = pm.star_dftconv(A, B, M)
        assert np.abs(D - C).max() < 1e-9
        assert np.array_equal(np.round(D.real) + 1j * np.round(D.imag), C)
    # one order shorter than wrap-free folds order 2T onto order 0
    D = pm.star_dftconv(A, B, 2 * T)
    assert np.abs(D - C).max() > 0.5


def test_paper_parameter_table_axes():
    table = load_parameters()
    assert set(table) == {"CPU(Naive-CONV)", "CPU(FFT-CONV)", "GPU(FFT-CONV)"}
    for steps, ns, ts in table.values():
        assert steps == 40
        for t in ts:  # N_trunc = N_p - 1 with N_p a power of two; FFT length 2 N_p
            assert (t + 1) & t == 0
            assert pm.default_fft_len(t) == 2 * (t + 1)
        for n in ns:  # SU(N) with N = L^2 (the TEK lattice extent L)
            assert int(round(n ** 0.5)) ** 2 == n
    import sweep
    a = sweep.parser().parse_args([])
    steps, ns, ts = table["GPU(FFT-CONV)"]
    assert a.md_steps == steps
    assert [int(x) for x in a.N.split(",")] == ns and [int(x) for x in a.T.split(",")] == ts


def test_library_default_fft_length_is_twice_the_padded_series():
    import paper_2001_02835_b300 as n
    L = n.lib()
    table = load_parameters()
    for t in sorted({t for _, _, ts in table.values() for t in ts}):
        sizes = {}
        for M in (0, 2 * (t + 1), 4 * (t + 1)):
            o = n.make_opts(algo="fft", fft_len=M)
            sizes[M] = L.nspt_workspace_size(n.OP_MUL, 121, t, 1, ctypes.byref(o))
        assert sizes[0] == sizes[2 * (t + 1)] > 0
        assert sizes[4 * (t + 1)] > sizes[0]
