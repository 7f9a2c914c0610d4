"""Timing sweep over the axes of the paper's benchmark (the GPU rows of its parameter
table: SU(N) for N in {121, 169, 225, 289}, truncation orders 15, 31, 63, trajectories of
40 MD steps): for every point, one MD trajectory of one configuration (momentum refresh
plus 40 leapfrog steps, split form) split into its force and link-update phases, and the
split FFT-CONV product rate at batch 4.  Prints a markdown table.

    python sweep.py [--N 121,169,225,289] [--T 15,31,63] [--md-steps 40]
    python sweep.py --accuracy    # per-order accuracy from the vacuum

Each configuration starts at the twisted vacuum (twist eaters at order 0, higher orders
zero) with seeded momenta of variance 1/N; one untimed trajectory thermalises it, then the
next one is timed (CUDA events on the current stream).  The orders decay from the vacuum,
so every phase fits the per-order rescale of its order transforms.
"""
from __future__ import annotations

import argparse
import math
import os
import sys

import numpy as np
import torch

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import nspt_synth as syn  # noqa: E402
import paper_2001_02835_b300 as nspt  # noqa: E402


def _time(fn, reps=1):
    fn()
    torch.cuda.synchronize()
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.record()
    for _ in range(reps):
        fn()
    e.record()
    torch.cuda.synchronize()
    return s.elapsed_time(e) / reps


def flux_for(L):
    return next(k for k in (1, 2, 3, 4, 5) if math.gcd(k, L) == 1)


def md_point(N, T, steps, eps=0.02):
    L = int(round(math.sqrt(N)))
    flux = flux_for(L)
    g = syn.rng(syn.SEED_BASE + 5)
    U = torch.from_numpy(np.ascontiguousarray(syn.vacuum_links(L, flux, T, 1))).cuda()
    eta = torch.from_numpy(np.ascontiguousarray(syn.md_momenta(g, N, 1))).cuda()
    P = torch.zeros_like(U)
    nspt.profile_begin(400000)
    # _time runs one trajectory from the vacuum (thermalisation, untimed), then the timed one
    ms = _time(lambda: nspt.tek_md_trajectory(U, P, flux, eps, steps, eta=eta, algo="fft", prec="split",
                                              rescale_log2r=nspt.RESCALE_AUTO), 1)
    ph = nspt.profile_end()
    if not bool(torch.isfinite(torch.view_as_real(U)).all().item()):
        raise SystemExit("non-finite links after the trajectories at N=%d T=%d" % (N, T))
    # the profile holds the untimed and the timed trajectory: halve
    return ms, ph.get("md_force", (0.0, 0))[0] / 2, ph.get("md_link", (0.0, 0))[0] / 2


def product_point(N, T, batch=4):
    g = syn.rng(syn.SEED_BASE + 6)
    A = torch.from_numpy(syn.series_batch(g, N, T, batch)).cuda()
    B = torch.from_numpy(syn.series_batch(g, N, T, batch)).cuda()
    C = torch.empty_like(A)
    ms = _time(lambda: nspt.polymat_mul(A, B, C, algo="fft", prec="split"), 5)
    return batch / (ms * 1e-3)


def accuracy_table(L=11, T=15, flux=1, eps=0.02, steps=(1, 10, 40)):
    """Per-order error of MD trajectories from the twisted vacuum (momenta of variance 1/N)
    against the naive FP64 form, which computes every order on its own: the FFT-CONV forms
    (FP64 and split) with and without the per-order rescale fitted at every phase."""
    N = L * L
    g = syn.rng(syn.SEED_BASE + 9)
    U0 = syn.vacuum_links(L, flux, T, 1)
    eta = torch.from_numpy(np.ascontiguousarray(syn.md_momenta(g, N, 1))).cuda()

    def run(algo, prec, r, n):
        U = torch.from_numpy(U0).cuda()
        P = torch.zeros_like(U)
        nspt.tek_md_trajectory(U, P, flux, eps, n, eta=eta, algo=algo, prec=prec, rescale_log2r=r)
        return U.cpu().numpy()[0]

    ks = (1, T // 3, 2 * T // 3, T)
    print("| steps | form | rescale | %s | max over orders 1..%d |" % (" | ".join("order %d" % k for k in ks), T))
    print("|---|---|---|%s---|" % ("---|" * len(ks)))
    for n in steps:
        ref = run("naive", "fp64", 0, n)
        den = np.sqrt(np.sum(np.abs(ref) ** 2, axis=(0, 2, 3)))
        for prec in ("fp64", "split"):
            for r, name in ((0, "none"), (nspt.RESCALE_AUTO, "fitted per phase")):
                X = run("fft", prec, r, n)
                e = np.sqrt(np.sum(np.abs(X - ref) ** 2, axis=(0, 2, 3))) / np.where(den == 0, 1, den)
                print("| %d | FFT-CONV %s | %s | %s | %.1e |" % (n, prec, name, " | ".join("%.1e" % e[k] for k in ks),
                                                              e[1:].max()))
        mx = np.abs(ref).max(axis=(0, 2, 3))
        print("| %d | max abs U_k (naive) | | %s | |" % (n, " | ".join("%.1e" % mx[k] for k in ks)))
        sys.stdout.flush()


def parser():
    """Command line; the default axes are the GPU rows of the paper's benchmark parameters
    (Sec. 3, Table "Parameters": 40 MD steps, SU(121..289), N_trunc 15, 31, 63)."""
    ap = argparse.ArgumentParser()
    ap.add_argument("--N", default="121,169,225,289")
    ap.add_argument("--T", default="15,31,63")
    ap.add_argument("--md-steps", type=int, default=40)
    ap.add_argument("--accuracy", action="store_true",
                    help="print the per-order accuracy table of trajectories from the vacuum instead")
    return ap


def main(argv=None):
    a = parser().parse_args(argv)
    torch.cuda.set_device(0)
    if nspt.lib().nspt_init() != 0:
        raise SystemExit("nspt_init failed")
    if a.accuracy:
        accuracy_table()
        return
    Ns = [int(x) for x in a.N.split(",")]
    Ts = [int(x) for x in a.T.split(",")]
    print("| N | T | MD trajectory (%d steps) s | force s | link update s | 10 trajectories s | products/s |"
          % a.md_steps)
    print("|---|---|---|---|---|---|---|")
    for N in Ns:
        for T in Ts:
            ms, f, lk = md_point(N, T, a.md_steps)
            pps = product_point(N, T)
            print("| %d | %d | %.3f | %.3f | %.3f | %.1f | %.0f |" % (N, T, ms / 1e3, f / 1e3, lk / 1e3, ms / 100.0, pps))
            sys.stdout.flush()


if __name__ == "__main__":
    main()
