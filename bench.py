#!/usr/bin/env python
"""Benchmark of the NSPT polynomial-matrix product on one B300 (or N replicas).

Metric: poly-matrix products/s (and effective TFLOP/s) at SU(225), O(g^63):
the truncated product C_k = sum_{l<=k} A_l B_{k-l}, k = 0..63, of two series of
225 x 225 complex matrices (Eq. 5), by FFT-CONV (Sec. 2, Steps 1-5) with M = 128,
batch 4 (one product per link direction).  One step = one call of
nspt_polymat_mul on a batch of 4 products with inputs resident in HBM; the
inputs (2 x 207 MB) and the spectra exceed the 126 MB L2, so no flush is needed.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

The end-to-end figure (`e2e`) is the same metric through nspt_polymat_mul_host
with pinned host buffers: every step copies A and B in and C out inside the
timed region (the copies of one batch element overlap the product of the next).
Unless --no-extras, the line also carries comparison legs: the FP64 form, the
O(g^31) timing point, the naive form, the backward, 64 uneven products in one
graph-captured launch, the Langevin step at SU(121), a 40-step MD trajectory at
SU(225), O(g^31) with its force / link-update split, and its Wilson loops.

Under torchrun (N > 1) every rank runs an independent replica on its own batch
(weak scaling; the products are independent, no data-path collective); rank 0
prints the JSON line with the max-over-ranks time.  `--impl reference` times the
FP64 CPU oracle (a deliberately slow, plain program) on a bounded sample.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import nspt_synth as syn  # noqa: E402

METRIC = "poly-matrix products/s at SU(225) O(g^63), FFT-CONV, batch 4"
N_DEF, T_DEF, BATCH = 225, 63, 4


def fft_flops(N, M):
    """Algorithmic FLOPs of one FFT-CONV product: M complex N^3 GEMMs plus three
    M-point radix-2 transforms over N^2 entries (5 M log2 M real flops each)."""
    return 8.0 * N ** 3 * M + 3 * 5.0 * N * N * M * math.log2(M)


def naive_flops(N, T):
    return 8.0 * N ** 3 * (T + 1) * (T + 2) / 2


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--prec", choices=["split", "fp64"], default=None)
    ap.add_argument("--T", type=int, default=T_DEF)
    ap.add_argument("--N", type=int, default=N_DEF)
    ap.add_argument("--no-extras", action="store_true", help="skip the comparison legs (FP64, T=31, MD, ...)")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def replica_seed(rank):
    """Each rank of an N-GPU run multiplies its own batch (independent products)."""
    return syn.SEED_BASE + 2 + 1000 * rank


def max_over_ranks(value, dist, device):
    """The slowest rank's time (the job finishes when the last replica does)."""
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, world, ms):
    """Units all ranks processed per second of the slowest rank's time."""
    return world * units_per_rank / (ms * 1e-3)


def inputs(N, T, batch, seed):
    g = syn.rng(seed)
    return syn.series_batch(g, N, T, batch), syn.series_batch(g, N, T, batch)


# --------------------------------------------------------------------------
# CPU oracle timing (the reference arm and cpu_baseline)
# --------------------------------------------------------------------------
def oracle_threads():
    try:
        from threadpoolctl import threadpool_info
        info = threadpool_info()
        n = [d.get("num_threads", 0) for d in info if d.get("user_api") == "blas"]
        return int(max(n)) if n else 1
    except Exception:  # pragma: no cover
        return os.cpu_count() or 1


def time_oracle_products(N, T, nprod, seed):
    """Wall time of the oracle's FFT-CONV (direct DFT, Sec. 2 Steps 1-5) on
    `nprod` products of the workload's shape."""
    from oracle import polymat as pm
    A, B = inputs(N, T, nprod, seed)
    t0 = time.perf_counter()
    pm.star_dftconv(A, B)
    return time.perf_counter() - t0


def time_oracle_naive(N, T, nprod, seed):
    """Wall time of the oracle's naive product (Eq. 5 loops) on `nprod` products."""
    from oracle import polymat as pm
    A, B = inputs(N, T, nprod, seed)
    t0 = time.perf_counter()
    pm.star(A, B)
    return time.perf_counter() - t0


def single_core_oracle_seconds(N, T):
    """The oracle's FFT-CONV of one product in a child process whose BLAS runs one thread
    (the thread count is fixed when numpy loads, so it cannot change in this process)."""
    env = dict(os.environ)
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS"):
        env[v] = "1"
    code = ("import sys; sys.path.insert(0, %r); import bench; "
            "print(bench.time_oracle_products(%d, %d, 1, %d))" % (ROOT, N, T, syn.SEED_BASE + 2))
    try:
        r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=300)
        return float(r.stdout.strip().split()[-1])
    except (subprocess.SubprocessError, ValueError, IndexError):
        return None


def cpu_baseline(N, T, M):
    """The oracle as it stands on the host cores, bounded samples: the workload's FFT-CONV on
    all cores (whole batches until about 10 s, at most 30 s) and on one core (one product),
    and the naive form (Eq. 5) at the correctness size SU(9), O(g^8), batch 4 and at the
    paper's timing point SU(225), O(g^31) (one product), on all cores."""
    done, tcpu = 0, 0.0
    while tcpu < 10.0 and done < 64:
        tcpu += time_oracle_products(N, T, BATCH, syn.SEED_BASE + 2)
        done += BATCH
        if tcpu > 30.0:
            break
    cores = oracle_threads()
    out = {"value": done / tcpu, "unit": "products/s", "cores": cores, "kind": "oracle",
           "sample": "%d products (N=%d, T=%d, M=%d) by the numpy FP64 oracle's direct-DFT FFT-CONV on %s"
                     % (done, N, T, M, cpu_model())}
    t1 = single_core_oracle_seconds(N, T)
    out["single_core"] = None if t1 is None else {
        "value": 1.0 / t1, "unit": "products/s", "cores": 1,
        "sample": "1 product (N=%d, T=%d), direct-DFT FFT-CONV, BLAS limited to one thread" % (N, T)}
    t0 = time_oracle_naive(9, 8, BATCH, syn.SEED_BASE)
    out["naive_su9_T8"] = {"value": BATCH / t0, "unit": "products/s", "cores": cores,
                           "sample": "batch of 4 products (N=9, T=8), Eq. 5 loops"}
    tn = time_oracle_naive(225, 31, 1, syn.SEED_BASE + 1)
    out["naive_su225_T31"] = {"value": 1.0 / tn, "unit": "products/s", "cores": cores,
                              "sample": "1 product (N=225, T=31), Eq. 5 loops"}
    tf = time_oracle_products(225, 31, BATCH, syn.SEED_BASE + 1)
    out["dftconv_su225_T31"] = {"value": BATCH / tf, "unit": "products/s", "cores": cores,
                                "sample": "batch of 4 products (N=225, T=31), direct-DFT FFT-CONV"}
    return out


def cpu_model():
    try:
        for line in open("/proc/cpuinfo"):
            if line.startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def arm_config(N, T, prec, ngpu, note, who="libnspt"):
    """The workload both arms report (the same sizes; `prec` and `who` say which arithmetic and
    which program ran it, `note` how)."""
    M = 1 << (2 * (T + 1) - 1).bit_length()
    return {"workload": "SU(%d) O(g^%d) FFT-CONV M=%d batch %d" % (N, T, M, BATCH),
            "N": N, "T": T, "M": M, "batch_per_gpu": BATCH, "prec": prec, "program": who,
            "parallelism": "replicas" if ngpu > 1 else "single", "l2": note}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    N, T = args.N, args.T
    nprod = BATCH
    for _ in range(args.warmup):
        time_oracle_products(N, T, nprod, syn.SEED_BASE + 2)
    times = [time_oracle_products(N, T, nprod, syn.SEED_BASE + 2) for _ in range(args.steps)]
    tot = sum(times)
    value = args.steps * nprod / tot
    cores = oracle_threads()
    line = {
        "impl": "reference",
        "metric": METRIC, "value": value, "unit": "products/s", "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "c128 (f64)", "data": "synthetic",
        "config": arm_config(N, T, "fp64", args.gpus,
                             "oracle's direct-DFT FFT-CONV in FP64 on the host cores, the whole batch per step",
                             who="numpy FP64 oracle"),
        "cpu_baseline": {"value": value, "unit": "products/s", "cores": cores, "kind": "oracle",
                         "sample": "batch of 4 products (N=%d, T=%d) per step, numpy FP64 oracle, %s"
                                   % (N, T, cpu_model())},
        "e2e": {"value": value, "unit": "products/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------------
# our arm
# --------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(prefix="nspt_clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if self.proc is None or not self.path:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                rows.append((float(p[1]), float(p[2]), float(p[3]), p[5], p[6], p[7], p[8]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        load = [r for r in rows if r[2] > 200.0] or rows
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in load for i, v in enumerate(r[3:7]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in load), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(load), "power_w_max": max(r[2] for r in rows)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d, "measured"
    return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "bf16_tflops_sustained": 1400.0}, "fallback"


def gemm_traffic_per_mode(N, slices):
    """DRAM bytes per mode of the tensor-core GEMM from the committed ncu record,
    or None when the kernel source changed since the capture (or sizes differ)."""
    import hashlib
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    rec = json.load(open(p)).get("gemm_tc")
    if not rec or rec.get("N") != N or rec.get("slices") != slices:
        return None
    src = os.path.join(ROOT, rec["source"])
    if not os.path.exists(src) or hashlib.sha256(open(src, "rb").read()).hexdigest()[:16] != rec["sha256_16"]:
        return None
    return rec["dram_bytes_per_mode"]


def fp64_peak_tflops(torch):
    """Measured FP64 denominator (the peaks file has none): cuBLAS DGEMM 4096^3, best of 5."""
    a = torch.randn(4096, 4096, dtype=torch.float64, device="cuda")
    b = torch.randn_like(a)
    c = a @ b
    torch.cuda.synchronize()
    best = 1e9
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(5):
        s.record()
        torch.matmul(a, b, out=c)
        e.record()
        e.synchronize()
        best = min(best, s.elapsed_time(e))
    del a, b, c
    return 2.0 * 4096 ** 3 / (best * 1e-3) / 1e12


def grouped_leg(torch, nspt, barrier, count=64, reps=5):
    """64 independent products, N from {49,121,169,225,289}, T from {15,31,63} (seeded),
    split form, tile width from the autotuner, one CUDA graph replayed per step."""
    pairs = syn.uneven_group(count)
    As = [torch.from_numpy(A).cuda() for A, _ in pairs]
    Bs = [torch.from_numpy(B).cuda() for _, B in pairs]
    Ns = [A.shape[-1] for A, _ in pairs]
    Ts = [A.shape[1] - 1 for A, _ in pairs]
    Cs = [torch.empty_like(A) for A in As]
    bn = nspt.autotune_grouped(As, Bs, cache_path=os.path.join(tempfile.gettempdir(), "nspt_tiles.txt"))
    nspt.polymat_mul_grouped(As, Bs, Cs, prec="split")
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        nspt.polymat_mul_grouped(As, Bs, Cs, prec="split")
    ms_graph = time_steps(torch, graph.replay, reps, 2, barrier) / reps
    ms_eager = time_steps(torch, lambda: nspt.polymat_mul_grouped(As, Bs, Cs, prec="split"), reps, 1, barrier) / reps
    flops = sum(fft_flops(int(N), 1 << math.ceil(math.log2(2 * (int(T) + 1)))) for N, T in zip(Ns, Ts))
    del graph, As, Bs, Cs
    return {"products": count, "tile_width": bn, "ms_per_group_graph": ms_graph, "ms_per_group_eager": ms_eager,
            "products_per_s": count / (ms_graph * 1e-3), "eff_tflops": flops / (ms_graph * 1e-3) / 1e12,
            "sizes": "N ~ U{49,121,169,225,289}, T ~ U{15,31,63}, seed 200102838"}


def langevin_leg(torch, nspt, barrier, L=11, T=31, streams=8, flux=3, eps=0.01):
    """One NSPT Langevin step of 8 streams x 4 links at SU(121), O(g^31), flux 3, both forms,
    with the oracle's step on one stream timed on the host cores beside it."""
    from oracle import tek
    g = syn.rng(syn.SEED_BASE + 4)
    N = L * L
    U = np.ascontiguousarray(syn.link_series(g, L, flux, T, streams))
    eta = np.ascontiguousarray(syn.hermitian_noise(g, N, streams * 4).reshape(streams, 4, N, N))
    tU0, tE = torch.from_numpy(U).cuda(), torch.from_numpy(eta).cuda()
    out = {}
    for p in ("split", "fp64"):
        tU = tU0.clone()
        reps = 5 if p == "split" else 1
        ms = time_steps(torch, lambda: nspt.tek_langevin_step(tU, tE, flux, eps, algo="fft", prec=p), reps, 1,
                        barrier) / reps
        out["%s_ms_per_step" % p] = ms
        out["%s_link_updates_per_s" % p] = streams * 4 / (ms * 1e-3)
    # the same split step with its noise drawn on the device each step (seeded generator,
    # device counter advanced by every draw)
    ctr = torch.zeros(1, dtype=torch.int64, device="cuda")
    tEs = torch.empty((streams * 4, N, N), dtype=torch.complex128, device="cuda")
    tU = tU0.clone()

    def seeded_step():
        nspt.tek_noise(N, streams * 4, syn.SEED_BASE + 4, 0, d_counter=ctr, out=tEs)
        nspt.tek_langevin_step(tU, tEs.view(streams, 4, N, N), flux, eps, algo="fft", prec="split")

    out["split_seeded_noise_ms_per_step"] = time_steps(torch, seeded_step, 5, 1, barrier) / 5
    t0 = time.perf_counter()
    tek.langevin_step(U[0], eta[0], tek.twist_phases(L, flux), eps)
    out["oracle_ms_per_stream"] = 1e3 * (time.perf_counter() - t0)
    out["oracle_cores"] = oracle_threads()
    del tU0, tE
    return out


def md_leg(torch, nspt, barrier, L=15, T=31, flux=1, eps=0.02, nsteps=40):
    """One MD trajectory of the paper's length (40 leapfrog steps, momentum refreshed at its
    start) of one SU(225) configuration at O(g^31) in the split form, with the time split
    into the force phase (drift plus momentum kicks) and the link-update phase, and the
    measurement of its Wilson loops up to 2 x 2 and the unitarity projection of its links.
    The configuration starts at the twisted vacuum and is thermalised by one untimed
    trajectory; the timed trajectory follows it with fresh momenta."""
    g = syn.rng(syn.SEED_BASE + 5)
    N = L * L
    tU = torch.from_numpy(np.ascontiguousarray(syn.vacuum_links(L, flux, T, 1))).cuda()
    tE0 = torch.from_numpy(np.ascontiguousarray(syn.md_momenta(g, N, 1))).cuda()
    tE = torch.from_numpy(np.ascontiguousarray(syn.md_momenta(g, N, 1))).cuda()
    tP = torch.zeros_like(tU)
    kw = dict(algo="fft", prec="split", rescale_log2r=nspt.RESCALE_AUTO)   # orders decay from the vacuum
    nspt.tek_md_trajectory(tU, tP, flux, eps, nsteps, eta=tE0, **kw)   # thermalisation
    nspt.profile_begin(200000)
    ms = time_steps(torch, lambda: nspt.tek_md_trajectory(tU, tP, flux, eps, nsteps, eta=tE, **kw), 1, 0, barrier)
    ph = nspt.profile_end()
    finite = bool(torch.isfinite(torch.view_as_real(tU)).all().item())
    umax = [float(x) for x in tU.abs()[0].amax(dim=(0, 2, 3)).cpu()]
    msw = time_steps(torch, lambda: nspt.tek_wilson_loops(tU, flux, 2, algo="fft", prec="split"), 2, 1, barrier) / 2
    # the unitarity projection of the evolved links (polar factor and U(1) phase), on a copy
    tW = tU.clone()
    msu = time_steps(torch, lambda: nspt.tek_unitarize(tW, special=True, algo="fft", prec="split"), 2, 1, barrier) / 2
    del tW
    out = {"ms_per_trajectory": ms, "md_steps": nsteps, "ms_per_md_step": ms / nsteps,
           "wilson_loops_amax2_ms": msw, "unitarity_projection_ms": msu,
           "force_ms": ph.get("md_force", (0.0, 0))[0], "link_update_ms": ph.get("md_link", (0.0, 0))[0],
           "kernel_stages_ms": {k: v[0] for k, v in ph.items() if k not in ("md_force", "md_link")},
           "links_finite": finite, "max_abs_link_order_0_8_16_24_31": [umax[k] for k in (0, 8, 16, 24, T)],
           "note": "one configuration (4 links) from the twisted vacuum after one thermalising trajectory, "
                   "momenta of variance 1/N, split form with the per-order rescale fitted at every phase; "
                   "10 trajectories = 10 x ms_per_trajectory"}
    del tU, tE, tE0, tP
    return out


def per_order_vs_oracle(torch, nspt, A, B, dA, dB, dC, T, barrier, extras):
    """Per-order relative errors of the split form (S = 5, 6; and 6 slices with three real
    products per complex product, 3M) and the FP64 form against the oracle's FFT-CONV (Sec. 2
    Steps 1-5, direct DFTs in FP64) on the bench's own inputs, and the split forms' speed."""
    from oracle import polymat as pm
    ref = pm.star_dftconv(A, B)
    den = np.sqrt(np.sum(np.abs(ref) ** 2, axis=(-1, -2)))

    def errs(C):
        num = np.sqrt(np.sum(np.abs(C - ref) ** 2, axis=(-1, -2)))
        return (num / np.where(den == 0, 1.0, den)).max(axis=0)

    out = {"oracle": "numpy FP64 direct-DFT FFT-CONV of the same batch",
           "fp64_form": [float("%.3g" % x) for x in errs(nspt.polymat_mul(dA, dB, algo="fft", prec="fp64").cpu().numpy())]}
    for S in (5, 6):
        kwS = dict(algo="fft", prec="split", slices=S)
        msS = time_steps(torch, lambda: nspt.polymat_mul(dA, dB, dC, **kwS), 5, 1, barrier) / 5
        e = errs(dC.cpu().numpy())
        out["split_S%d" % S] = [float("%.3g" % x) for x in e]
        extras["split_S%d_T%d" % (S, T)] = {"products_per_s": BATCH / (msS * 1e-3), "ms_per_step": msS,
                                            "max_per_order_rel_err_vs_oracle": float(e.max())}
    kw3 = dict(algo="fft", prec="split", complex_mode=3)
    ms3 = time_steps(torch, lambda: nspt.polymat_mul(dA, dB, dC, **kw3), 5, 1, barrier) / 5
    e = errs(dC.cpu().numpy())
    out["split_S6_3m"] = [float("%.3g" % x) for x in e]
    extras["split_S6_3m_T%d" % T] = {"products_per_s": BATCH / (ms3 * 1e-3), "ms_per_step": ms3,
                                     "max_per_order_rel_err_vs_oracle": float(e.max()),
                                     "note": "three real products per complex product (3M); 4M above"}
    kwn = dict(algo="naive", prec="split")
    msn = time_steps(torch, lambda: nspt.polymat_mul(dA, dB, dC, **kwn), 2, 1, barrier) / 2
    e = errs(dC.cpu().numpy())
    out["split_S6_naive"] = [float("%.3g" % x) for x in e]
    extras["split_S6_naive_T%d" % T] = {"products_per_s": BATCH / (msn * 1e-3), "ms_per_step": msn,
                                        "eff_tflops": naive_flops(A.shape[-1], T) * BATCH / (msn * 1e-3) / 1e12,
                                        "max_per_order_rel_err_vs_oracle": float(e.max()),
                                        "note": "naive form (Eq. 5): one tensor-core GEMM per pair of orders"}
    return out


def md_graph_leg(torch, nspt, barrier, L=11, T=15, flux=1, eps=0.02, nsteps=40):
    """One 40-step MD trajectory at SU(121), O(g^15) in the split form with the fitted rescale,
    enqueued eagerly and replayed as one captured CUDA graph (the fit runs on the device, so
    the whole trajectory captures): at this size the host's enqueue time of the ~300 launches
    per step is not hidden behind the GPU."""
    g = syn.rng(syn.SEED_BASE + 6)
    N = L * L
    U0 = torch.from_numpy(np.ascontiguousarray(syn.vacuum_links(L, flux, T, 1))).cuda()
    eta = torch.from_numpy(np.ascontiguousarray(syn.md_momenta(g, N, 1))).cuda()
    kw = dict(algo="fft", prec="split", rescale_log2r=nspt.RESCALE_AUTO)
    U, P = U0.clone(), torch.zeros_like(U0)
    nspt.tek_md_trajectory(U, P, flux, eps, nsteps, eta=eta, **kw)      # thermalisation
    Ut = U.clone()
    eager = time_steps(torch, lambda: nspt.tek_md_trajectory(U, P, flux, eps, nsteps, eta=eta, **kw), 2, 1, barrier) / 2
    Ug, Pg = Ut.clone(), torch.zeros_like(Ut)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        nspt.tek_md_trajectory(Ug, Pg, flux, eps, nsteps, eta=eta, **kw)
    replay = time_steps(torch, graph.replay, 2, 1, barrier) / 2
    del graph, U, P, Ug, Pg, U0, Ut, eta
    return {"ms_per_trajectory_eager": eager, "ms_per_trajectory_graph": replay, "md_steps": nsteps,
            "workload": "SU(%d), O(g^%d), one configuration, split form, fitted rescale" % (N, T)}


def time_steps(torch, fn, steps, warmup, barrier):
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    st = torch.cuda.current_stream()
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.record(st)
    for _ in range(steps):
        fn()
    e.record(st)
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    return s.elapsed_time(e)


def run_ours(args):
    import torch
    ws, rank, local = dist_env()
    dist = None
    if ws > 1:
        import torch.distributed as dist  # noqa: F811
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    import paper_2001_02835_b300 as nspt
    if nspt.lib().nspt_init() != 0:
        raise SystemExit("libnspt: nspt_init failed (not an sm_103 device?)")

    def barrier():
        if dist is not None:
            dist.barrier()

    N, T = args.N, args.T
    M = 1 << math.ceil(math.log2(2 * (T + 1)))
    prec = args.prec or "split"
    A, B = inputs(N, T, BATCH, replica_seed(rank))
    dA = torch.from_numpy(A).cuda()
    dB = torch.from_numpy(B).cuda()
    dC = torch.empty_like(dA)
    kw = dict(algo="fft", prec=prec)
    fn = lambda: nspt.polymat_mul(dA, dB, dC, **kw)  # noqa: E731

    # timed region (stage events on, clocks sampled)
    for _ in range(args.warmup):
        fn()
    torch.cuda.synchronize()
    l0 = nspt.launch_count()
    nspt.profile_begin(100000)
    with ClockSampler(torch.cuda.current_device()) as clk:
        ms = time_steps(torch, fn, args.steps, 0, barrier)
    stages = nspt.profile_end()
    launches = nspt.launch_count() - l0
    clocks = clk.summary()
    ms = max_over_ranks(ms, dist, "cuda")
    ms_step = ms / args.steps
    value = whole_job_rate(BATCH * args.steps, ws, ms)

    # end to end through the C ABI with host buffers (pinned): nspt_polymat_mul_host copies
    # A and B in and C out for every step inside the timed region, overlapping the copies of
    # one batch element with the product of the next
    hA = torch.from_numpy(A).pin_memory()
    hB = torch.from_numpy(B).pin_memory()
    hC = torch.empty_like(hA).pin_memory()

    def e2e_step():
        nspt.polymat_mul_host(hA, hB, hC, **kw)

    e2e_steps = max(3, args.steps // 2)
    ms_e2e = time_steps(torch, e2e_step, e2e_steps, 1, barrier)
    e2e_value = whole_job_rate(BATCH * e2e_steps, ws, max_over_ranks(ms_e2e, dist, "cuda"))
    nbytes = A.nbytes

    peaks, peak_kind = measured_peaks()
    # dominant kernel of the step
    dom = max(stages.items(), key=lambda kv: kv[1][0])
    dom_name, (dom_ms, dom_n) = dom
    per_launch_ms = dom_ms / max(dom_n, 1)
    if dom_name == "gemm_tc":
        slices = 6
        pairs = slices * (slices + 1) // 2
        launches_per_step = max(1, dom_n // args.steps)
        modes = M * BATCH / launches_per_step
        # algorithmic work of the method (Step 3): one complex N x N x N product per mode,
        # 8 N^3 flops; the split's slice pairs and the tile padding are overhead, not work
        flops = 8.0 * N ** 3 * modes
        achieved = flops / (per_launch_ms * 1e-3) / 1e12
        # what the tensor cores issue: per mode S(S+1)/2 slice pairs x 4 real products of
        # 2 N^3 flops (unpadded N), the issued-MMA efficiency of the kernel
        issued = pairs * 4 * 2.0 * N ** 3 * modes / (per_launch_ms * 1e-3) / 1e12
        peak = peaks["bf16_tflops_sustained"]
        tpm = gemm_traffic_per_mode(N, slices)
        roof = {"kernel": dom_name, "bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": (tpm * modes if tpm else None),
                "work": "8 N^3 per mode (Step 3), N=%d, %d modes per launch" % (N, int(modes)),
                "traffic_source": "profiles/traffic.json (small-case capture scaled per mode)" if tpm else None,
                "peak_source": "%s bf16_tflops_sustained (of %s)" % (peak_kind, peak_kind),
                "frac_of_burst": achieved / peaks["bf16_tflops"],
                "issued_mma": {"tflops": issued, "frac_of_sustained": issued / peak,
                               "frac_of_burst": issued / peaks["bf16_tflops"],
                               "work": "S(S+1)/2 = %d slice pairs x 4 real products x 2 N^3 per mode" % pairs}}
    elif dom_name in ("gemm_mode", "gemm_conv"):
        f64 = fp64_peak_tflops(torch)
        flops = 8.0 * N ** 3 * M * BATCH / max(1, dom_n // args.steps)
        achieved = flops / (per_launch_ms * 1e-3) / 1e12
        roof = {"kernel": dom_name, "bound": "alu", "achieved": achieved, "peak": f64, "unit": "TFLOP/s",
                "frac": achieved / f64, "traffic": None,
                "peak_source": "measured cuBLAS DGEMM 4096^3 in this run (FP64 pipe)"}
    else:
        byts = (T + 1 + M) * N * N * 16.0 * BATCH
        achieved = byts / (per_launch_ms * 1e-3) / 1e9
        roof = {"kernel": dom_name, "bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / peaks["hbm_gbs"], "traffic": None, "peak_source": "%s hbm_gbs" % peak_kind}

    extras = {}
    if not args.no_extras and ws == 1:
        # FP64 form at the same workload, and the paper's timing point T = 31
        if prec != "fp64":
            kw64 = dict(algo="fft", prec="fp64")
            ms64 = time_steps(torch, lambda: nspt.polymat_mul(dA, dB, dC, **kw64), 3, 1, barrier)
            extras["fp64_fft_T%d" % T] = {"products_per_s": BATCH * 3 / (ms64 * 1e-3), "ms_per_step": ms64 / 3}
            # accuracy against speed: the split form with 5 and 6 slices and the FP64 form,
            # per-order relative error (Frobenius, max over the batch) against the FP64 oracle's
            # FFT-CONV of the same inputs, computed on the host cores
            extras["per_order_err_vs_oracle"] = per_order_vs_oracle(torch, nspt, A, B, dA, dB, dC, T, barrier,
                                                                    extras)
        A31, B31 = inputs(N, 31, BATCH, syn.SEED_BASE + 1)
        a31, b31 = torch.from_numpy(A31).cuda(), torch.from_numpy(B31).cuda()
        c31 = torch.empty_like(a31)
        for p in ([prec] if prec == "fp64" else [prec, "fp64"]):
            ms31 = time_steps(torch, lambda: nspt.polymat_mul(a31, b31, c31, algo="fft", prec=p), 3, 1, barrier)
            extras["%s_fft_T31" % p] = {"products_per_s": BATCH * 3 / (ms31 * 1e-3), "ms_per_step": ms31 / 3,
                                        "eff_tflops": fft_flops(N, 64) * BATCH * 3 / (ms31 * 1e-3) / 1e12}
        extras["grouped_64_uneven"] = grouped_leg(torch, nspt, barrier)
        gC = torch.from_numpy(syn.gaussian(syn.rng(syn.SEED_BASE + 9), A.shape, 1.0)).cuda()
        for p in ("split", "fp64"):
            reps = 5 if p == "split" else 2
            msb = time_steps(torch, lambda: nspt.polymat_mul_backward(dA, dB, gC, algo="fft", prec=p), reps, 1,
                             barrier) / reps
            extras["backward_%s_T%d" % (p, T)] = {"ms_per_batch": msb, "products_per_s": BATCH / (msb * 1e-3)}
        del gC
        extras["langevin_su121_T31_8streams"] = langevin_leg(torch, nspt, barrier)
        extras["md_trajectory_su225_T31"] = md_leg(torch, nspt, barrier)
        extras["md_trajectory_su121_T15_graph"] = md_graph_leg(torch, nspt, barrier)
        msn = time_steps(torch, lambda: nspt.polymat_mul(a31, b31, c31, algo="naive"), 1, 1, barrier)
        extras["fp64_naive_T31"] = {"products_per_s": BATCH / (msn * 1e-3), "ms_per_step": msn,
                                    "eff_tflops": naive_flops(N, 31) * BATCH / (msn * 1e-3) / 1e12}
        msn = time_steps(torch, lambda: nspt.polymat_mul(a31, b31, c31, algo="naive", prec="split"), 3, 1,
                         barrier) / 3
        extras["split_naive_T31"] = {"products_per_s": BATCH / (msn * 1e-3), "ms_per_step": msn,
                                     "eff_tflops": naive_flops(N, 31) * BATCH / (msn * 1e-3) / 1e12}
        g31 = torch.from_numpy(syn.gaussian(syn.rng(syn.SEED_BASE + 10), A31.shape, 1.0)).cuda()
        msb = time_steps(torch, lambda: nspt.polymat_mul_backward(a31, b31, g31, algo="naive", prec="split"), 2, 1,
                         barrier) / 2
        extras["backward_split_naive_T31"] = {"ms_per_batch": msb, "products_per_s": BATCH / (msb * 1e-3),
                                              "note": "gA and gB, one tensor-core GEMM per pair of orders each"}
        del g31
        del a31, b31, c31

    cpu = None
    if rank == 0:
        cpu = cpu_baseline(N, T, M)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "products/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None,
            "dtype": "c128 in/out; " + ("double-float (f32 pair) order transforms, bf16 digit slices x6, "
                                        "fp32 exact digit-group partials" if prec == "split" else "f64"),
            "data": "synthetic (Haar SU(N) order 0, Gaussian var 1/N orders >= 1, seed 200102837)",
            "config": arm_config(N, T, prec, ws, "inputs 2 x %.0f MB > 126 MB L2, no flush" % (nbytes / 1e6)),
            "eff_tflops": fft_flops(N, M) * value / 1e12,
            "roofline": roof,
            "stages_ms_per_step": {k: v[0] / args.steps for k, v in stages.items()},
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": "products/s", "h2d_bytes_per_step": 2 * nbytes,
                    "d2h_bytes_per_step": nbytes},
            "gpu_launches": launches,
            "clocks": clocks,
            "extras": extras,
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
