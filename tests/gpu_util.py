"""Helpers shared by the GPU parity tests (no arithmetic of the method).

Error metric: per perturbative order k, ||X_k - ref_k||_F / ||ref_k||_F; an order whose
reference is exactly zero (order 0 of a drift at the twisted vacuum, say) is measured
against the largest order's norm instead.

Split-form bound.  With S digit slices every spectrum row (column) is carried to 8S - 1
bits below its largest entry, so a product's per-order relative error is
c * 2^-(8S-1), plus a floor f from the double-float transforms (about 45 bits: their sums
are formed on a common grid per butterfly, so each step's error is bounded relative to
the butterfly's largest input).  c and f were calibrated on B300 from the parity cases
themselves (every product case of the tests, the benchmarked SU(225), O(g^63) batch and the
64-product group, S = 2..8): the largest observed err / 2^-(8S-1) at S <= 6 was 84 (an
SU(6), O(g^200) product, M = 512), so C_OBS = 84, and the S = 7, 8 results, which the floor
dominates, stayed below F_OBS = 2^-44.  The stated bound takes four times both:
    split_bound(S) = 336 * 2^-(8S-1) + 2^-42      (2.4e-12 + 2.3e-13 = 2.6e-12 at S = 6),
1.3 units of the last digit with S - 1 slices: the result with one slice fewer (observed 6
to 60 such units at N >= 9) fails it.

Chained computations (the Langevin step, MD, the Wilson loops) mix the orders in every
product of the chain, and their error grows with the truncation order beyond T ~ 24 in
the FP64 FFT form as much as in the split form (the split/FP64 error ratio stays near
100 at every T); the bound for them is CHAIN[kind] * 2^max(0, (T - 24)/8) times the
product bound, with CHAIN at least four times the largest observed ratio to the product
bound times the growth (0.34 for the Langevin step at SU(121), O(g^31); 1.09 for one MD step
at SU(225), O(g^31) with the fitted rescale; 1.72 for the Wilson loops at SU(121), O(g^31);
0.21 for the backward; 0.14 for the unitarity projection).

The naive split form (one tensor-core GEMM per pair of orders, no transforms) makes each
pair's error relative to that pair's own size, so its chained computations (the unitarity
projection and the Wilson loops, whose products all go through the product call) neither mix
the orders nor grow with T: they take the product bound itself (CHAIN["naive_chain"] = 1, no
growth), over four times the largest observed ratio (0.07: the projection with the U(1) phase at
N = 25, T = 15; the Wilson loops stayed below 0.03); the projection with one slice fewer
exceeds it (4.6e-12 to 2.3e-11 for N = 9..121).

The 3M products (three real products per complex product, `complex_mode=3`) take the
product bound times CHAIN["product3m"]: their imaginary part P3 - P1 - P2 comes from the
digits of re + im, sliced at twice the row bound, and cancels; the largest observed ratio to
the product bound was 0.38 (the SU(225), O(g^63) batch), 1.3-2.2 times the 4M error of the
same product.
"""
import json
import os

import numpy as np
import torch

# calibration constants (see the module docstring)
C_OBS = 84.0                  # max err / 2^-(8S-1) over the product cases, S <= 6
F_OBS = 2.0 ** -44            # max err of the product cases at S = 7, 8
SPLIT_C = 4 * C_OBS
SPLIT_FLOOR = 4 * F_OBS
CHAIN = {"product": 1.0, "product3m": 2.0, "backward": 2.0, "langevin": 2.0, "md": 6.0, "wilson": 8.0,
         "unitarize": 2.0, "naive_chain": 1.0}


def dev(x: np.ndarray) -> torch.Tensor:
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda")


def host(t: torch.Tensor) -> np.ndarray:
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def order_errors(X, ref) -> np.ndarray:
    """Per-order relative Frobenius errors, shape (..., T+1) of the series' leading axes;
    orders whose reference is exactly zero are divided by the largest order's norm."""
    X = np.asarray(X)
    ref = np.asarray(ref)
    num = np.sqrt(np.sum(np.abs(X - ref) ** 2, axis=(-1, -2)))
    den = np.sqrt(np.sum(np.abs(ref) ** 2, axis=(-1, -2)))
    big = den.max() if den.size else 0.0
    return num / np.where(den == 0, big if big > 0 else 1.0, den)


def max_order_rel(X, ref) -> float:
    """max over batch and order of the per-order relative error (see order_errors)."""
    e = order_errors(X, ref)
    return float(e.max()) if e.size else 0.0


def split_bound(S: int, kind: str = "product", T: int = 0, algo: str = "fft") -> float:
    """Stated per-order bound of the split form with S slices (module docstring); T, the
    truncation order, matters for the chained kinds of FFT-CONV only; with algo="naive" the
    chained kinds take the naive form's bound ("naive_chain")."""
    if algo == "naive" and kind in ("langevin", "md", "wilson", "unitarize"):
        kind = "naive_chain"
    growth = 2.0 ** max(0.0, (T - 24) / 8.0) if kind in ("langevin", "md", "wilson", "unitarize") else 1.0
    return CHAIN[kind] * growth * (SPLIT_C * 2.0 ** -(8 * S - 1) + SPLIT_FLOOR)


def record(test: str, **kw):
    """Appends one JSON line of measured errors to $NSPT_ERR_LOG (when set), the data the
    calibration constants above were taken from."""
    path = os.environ.get("NSPT_ERR_LOG")
    if not path:
        return
    row = {"test": test}
    for k, v in kw.items():
        if isinstance(v, np.ndarray):
            v = v.tolist()
        elif isinstance(v, (np.floating, np.integer)):
            v = v.item()
        row[k] = v
    with open(path, "a") as f:
        f.write(json.dumps(row) + "\n")
