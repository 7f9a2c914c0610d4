"""Runs one library entry point repeatedly on synthetic inputs of a given size.

    python run_case.py --op mul --algo fft --prec split --N 225 --T 15 --batch 4 --reps 3

Used for profiling single calls (e.g. under ncu) and quick timing; every call
is a complete call of the entry point.  Prints the mean CUDA-event time per
call.
"""
from __future__ import annotations

import argparse
import os
import sys

import numpy as np
import torch

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import nspt_synth as syn  # noqa: E402
import paper_2001_02835_b300 as nspt  # noqa: E402


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--op", choices=["mul", "backward", "langevin", "md", "wilson", "unitarize"], default="mul")
    ap.add_argument("--algo", default="fft")
    ap.add_argument("--prec", default="split")
    ap.add_argument("--N", type=int, default=225)
    ap.add_argument("--T", type=int, default=15)
    ap.add_argument("--batch", type=int, default=4)
    ap.add_argument("--slices", type=int, default=0)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=1)
    ap.add_argument("--md-steps", type=int, default=40, help="leapfrog steps per call of --op md")
    ap.add_argument("--amax", type=int, default=2, help="largest loop extent of --op wilson")
    a = ap.parse_args(argv)
    torch.cuda.set_device(0)
    if nspt.lib().nspt_init() != 0:
        raise SystemExit("nspt_init failed")
    g = syn.rng(syn.SEED_BASE + 7)
    kw = dict(algo=a.algo, prec=a.prec, slices=a.slices)
    if a.op == "langevin":
        L = int(round(a.N ** 0.5))
        U = torch.from_numpy(np.ascontiguousarray(syn.link_series(g, L, 1, a.T, a.batch))).cuda()
        eta = torch.from_numpy(np.ascontiguousarray(syn.hermitian_noise(g, a.N, 4 * a.batch).reshape(a.batch, 4, a.N, a.N))).cuda()
        fn = lambda: nspt.tek_langevin_step(U, eta, 1, 0.01, **kw)  # noqa: E731
    elif a.op == "unitarize":
        # the projection with the U(1) phase removed, on links with Gaussian higher orders scaled
        # down to a small drift from unitarity, on a copy per call
        L = int(round(a.N ** 0.5))
        U0 = syn.link_series(g, L, 1, a.T, a.batch)
        U0[:, :, 1:] *= 1e-2
        U0 = torch.from_numpy(np.ascontiguousarray(U0)).cuda()
        U = torch.empty_like(U0)

        def fn():
            U.copy_(U0)
            nspt.tek_unitarize(U, special=True, **kw)
    elif a.op == "wilson":
        L = int(round(a.N ** 0.5))
        U = torch.from_numpy(np.ascontiguousarray(syn.link_series(g, L, 1, a.T, a.batch))).cuda()
        fn = lambda: nspt.tek_wilson_loops(U, 1, a.amax, **kw)  # noqa: E731
    elif a.op == "md":
        # from the twisted vacuum with momenta of variance 1/N, the rescale fitted per phase
        # (Gaussian link orders are not a unitary series and blow up under MD)
        L = int(round(a.N ** 0.5))
        U = torch.from_numpy(np.ascontiguousarray(syn.vacuum_links(L, 1, a.T, a.batch))).cuda()
        P = torch.zeros_like(U)
        eta = torch.from_numpy(np.ascontiguousarray(syn.md_momenta(g, a.N, a.batch))).cuda()
        if a.algo == "fft":
            kw["rescale_log2r"] = nspt.RESCALE_AUTO
        fn = lambda: nspt.tek_md_trajectory(U, P, 1, 0.02, a.md_steps, eta=eta, **kw)  # noqa: E731
    else:
        A = torch.from_numpy(syn.series_batch(g, a.N, a.T, a.batch)).cuda()
        B = torch.from_numpy(syn.series_batch(g, a.N, a.T, a.batch)).cuda()
        C = torch.empty_like(A)
        if a.op == "mul":
            fn = lambda: nspt.polymat_mul(A, B, C, **kw)  # noqa: E731
        else:
            G = torch.from_numpy(syn.gaussian(g, tuple(A.shape), 1.0)).cuda()
            fn = lambda: nspt.polymat_mul_backward(A, B, G, **kw)  # noqa: E731
    for _ in range(a.warmup):
        fn()
    torch.cuda.synchronize()
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.record()
    for _ in range(a.reps):
        fn()
    e.record()
    torch.cuda.synchronize()
    print("%s N=%d T=%d batch=%d %s/%s: %.3f ms per call" % (a.op, a.N, a.T, a.batch, a.algo, a.prec,
                                                            s.elapsed_time(e) / a.reps))


if __name__ == "__main__":
    main()
