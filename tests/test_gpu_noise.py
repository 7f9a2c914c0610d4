"""GPU parity of the seeded Langevin noise (nspt_tek_noise, Philox4x32-10 on the device)
against the oracle's restatement of the same generator (oracle/noise.py).

The generator's words are integers and map to the Gaussians by the same FP64 steps
on both sides; only the transcendental functions differ (CUDA's log, sqrt and
sincospi against numpy's log, sqrt, cos and sin of 2 pi u), by a few units of the
last place: |z| < 8.6, so the entries agree to 1e-13 absolute, while a single wrong
word of the generator moves an entry by O(1)."""
import numpy as np
import pytest
import torch

import nspt_synth as syn
from oracle import noise as nz
from oracle import tek

from tests.gpu_util import dev, host, max_order_rel

pytestmark = pytest.mark.gpu

ABS = 1e-13


@pytest.fixture(scope="module")
def nspt():
    import paper_2001_02835_b300 as n
    assert n.lib().nspt_init() == 0
    return n


@pytest.mark.parametrize("N,count,seed,counter", [(1, 3, 5, 0), (2, 5, 1, 7), (9, 16, 2001, 0),
                                                  (33, 7, (3 << 32) | 99, (1 << 32) + 5), (121, 4, 42, 123),
                                                  (225, 2, 7, 0), (1024, 1, 11, 3)])
def test_noise_matches_oracle(nspt, N, count, seed, counter):
    eta = host(nspt.tek_noise(N, count, seed, counter))
    ref = nz.langevin_noise(N, count, seed, counter)
    assert np.abs(eta - ref).max() <= ABS
    np.testing.assert_array_equal(eta, np.conj(np.swapaxes(eta, -1, -2)))      # Hermitian bit for bit
    assert np.abs(np.trace(eta, axis1=1, axis2=2)).max() <= 1e-12


def test_device_counter_advances_and_graph_replays_draw_fresh_noise(nspt):
    N, count, seed, base = 12, 4, 77, 1000
    ctr = torch.zeros(1, dtype=torch.int64, device="cuda")
    for k in range(3):
        eta = host(nspt.tek_noise(N, count, seed, base, d_counter=ctr))
        assert np.abs(eta - nz.langevin_noise(N, count, seed, base + k)).max() <= ABS
    assert int(ctr.item()) == 3
    out = torch.empty((count, N, N), dtype=torch.complex128, device="cuda")
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        nspt.tek_noise(N, count, seed, base, d_counter=ctr, out=out)
    # capture enqueues without running: the counter is still 3
    for k in range(3, 6):
        graph.replay()
        assert np.abs(host(out) - nz.langevin_noise(N, count, seed, base + k)).max() <= ABS
    assert int(ctr.item()) == 6


def test_noise_statistics_at_su121(nspt):
    """The device draw has the step's distribution: E|eta_ij|^2 = 1 off the diagonal,
    diagonal variance 1 - 1/N (8 streams x 4 links at SU(121))."""
    N, count = 121, 32
    eta = host(nspt.tek_noise(N, count, seed=9, counter=0))
    off = ~np.eye(N, dtype=bool)
    n_off = count * N * (N - 1) // 2
    assert abs(np.mean(np.abs(eta[:, off]) ** 2) - 1.0) < 4 / np.sqrt(n_off)
    d = np.real(np.diagonal(eta, axis1=1, axis2=2))
    assert abs(np.mean(d ** 2) - (1 - 1 / N)) < 4 * np.sqrt(2.0 / (count * N))


def test_seeded_langevin_step_matches_oracle(nspt):
    """SU(9), O(g^8), 4 streams (the correctness size of the paper's product), flux 1,
    eps = 0.01: noise drawn on the device, then the FP64 step, against the oracle's step
    with the oracle's draw of the same noise."""
    L, flux, T, streams, eps, seed = 3, 1, 8, 4, 0.01, 2001
    N = L * L
    U = syn.link_series(syn.rng(syn.SEED_BASE), L, flux, T, streams)
    tU = dev(U)
    eta = nspt.tek_noise(N, streams * 4, seed, 0).reshape(streams, 4, N, N)
    nspt.tek_langevin_step(tU, eta, flux, eps, algo="naive", prec="fp64")
    ref_eta = nz.langevin_noise(N, streams * 4, seed, 0).reshape(streams, 4, N, N)
    z = tek.twist_phases(L, flux)
    ref = np.stack([tek.langevin_step(U[s], ref_eta[s], z, eps)[0] for s in range(streams)])
    assert max_order_rel(host(tU), ref) <= 1e-12
