"""Writes the stored expected values of tests/golden from the FP64 oracle only.

star_integer_N3_T5.txt: a truncated product (Eq. 5) of Gaussian-integer
series, N = 3, T = 5, entries with real and imaginary parts in [-9, 9]
(seeded).  Every partial sum is an integer far below 2^53, so the oracle's
naive product is exact and the stored integers are the product itself.

Run from the repository root:  python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import polymat as pm  # noqa: E402

N, T, SEED, LIM = 3, 5, 2001028350, 9


def inputs():
    g = np.random.default_rng(SEED)
    shape = (T + 1, N, N)
    A = g.integers(-LIM, LIM + 1, shape) + 1j * g.integers(-LIM, LIM + 1, shape)
    B = g.integers(-LIM, LIM + 1, shape) + 1j * g.integers(-LIM, LIM + 1, shape)
    return A.astype(np.complex128), B.astype(np.complex128)


def _rows(name, X):
    out = []
    for k in range(X.shape[0]):
        for i in range(X.shape[1]):
            vals = " ".join("%d %d" % (int(v.real), int(v.imag)) for v in X[k, i])
            out.append("%s %d %d  %s" % (name, k, i, vals))
    return out


def main():
    A, B = inputs()
    C = pm.star(A, B)
    assert np.all(C == np.round(C))
    lines = ["# Truncated product C_k = sum_{j<=k} A_j B_{k-j} (Eq. 5) of Gaussian-integer",
             "# series, N = %d, T = %d; written by tests/golden/make_golden.py from the oracle's" % (N, T),
             "# naive product (exact: every partial sum is an integer below 2^53).",
             "# line: <A|B|C> <order k> <row i>  then (re im) for columns 0..N-1"]
    lines += _rows("A", A) + _rows("B", B) + _rows("C", C)
    with open(os.path.join(HERE, "star_integer_N3_T5.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
