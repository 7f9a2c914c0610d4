"""Drift from the backward kernel: the NSPT drift of the Langevin step equals the
derivative of the order-truncated TEK action (Eqs. 1-3), with the derivative
taken by the autograd Function over nspt_polymat_mul / nspt_polymat_mul_backward.

S~^(k) = 12 N delta_k0 - sum_{mu != nu} Tr[z (U_mu U_nu U_mu^+ U_nu^+)^(k)] depends on
U^(j) only through the g^j factor of U(g), so one backward pass of
L = Re S~^(T) gives dS~^(T)/dU^(j) = D^(T-j), every coefficient of the action's
derivative series D.  With Y = i U * D^+ (star product), the drift of every
order is F^(k) = -[(Y^(k) + Y^(k)^H)/2]_traceless.  At SU(121), T = 31, flux 3,
8 streams (the configuration this module is built around) the test checks that
drift against the library's staple-based drift, against the oracle's drift on
one stream, against central finite differences (h = 1e-6) through the GPU
forward, and then runs a full Langevin step composed from library products on
the backward-derived drift against nspt_tek_langevin_step.  The library's step
itself (FP64 and split forms) is compared with the oracle's step on one stream.

Orders are compared one by one (relative Frobenius error); the drift's order 0,
zero to rounding at the twisted vacuum, is compared against the largest order.
"""
import math

import numpy as np
import pytest
import torch

import nspt_synth as syn
from oracle import tek

from tests.gpu_util import dev, host, max_order_rel, record, split_bound

pytestmark = pytest.mark.gpu
L_SIDE, FLUX, T, STREAMS, EPS = 11, 3, 31, 8, 0.01
N = L_SIDE * L_SIDE


@pytest.fixture(scope="module")
def nspt():
    import paper_2001_02835_b300 as n
    assert n.lib().nspt_init() == 0
    return n


def dag(X):
    return X.conj().transpose(-1, -2).contiguous()


def action_series(nspt, U, z):
    """(streams, T+1) complex series of the truncated action, differentiable in U."""
    S_, T1 = U.shape[0], U.shape[2]
    tot = torch.zeros((S_, T1), dtype=torch.complex128, device=U.device)
    for mu in range(4):
        for nu in range(4):
            if mu == nu:
                continue
            Um, Un = U[:, mu], U[:, nu]
            P = nspt.star(nspt.star(nspt.star(Um, Un, algo="fft"), dag(Um), algo="fft"), dag(Un), algo="fft")
            tot = tot - complex(z[mu, nu]) * torch.diagonal(P, dim1=-2, dim2=-1).sum(-1)
    corr = torch.zeros_like(tot)
    corr[:, 0] = 12 * U.shape[-1]
    return tot + corr


def drift_from_backward(nspt, U, z):
    Ug = U.clone().requires_grad_(True)
    S = action_series(nspt, Ug, z)
    loss = S[:, -1].real.sum()
    loss.backward()
    G = Ug.grad.detach()
    D = torch.flip(G, dims=[2])                       # D^(m) = dS^(T)/dU^(T-m)
    s4 = U.shape[0] * 4
    Uf = U.reshape(s4, *U.shape[2:]).contiguous()
    Df = D.reshape(s4, *D.shape[2:]).contiguous()
    Y = 1j * nspt.polymat_mul(Uf, dag(Df), algo="fft")
    Fb = -(Y + dag(Y)) / 2
    tr = torch.diagonal(Fb, dim1=-2, dim2=-1).sum(-1) / U.shape[-1]
    Fb = Fb - tr[..., None, None] * torch.eye(U.shape[-1], dtype=Fb.dtype, device=Fb.device)
    return Fb.reshape(U.shape), S.detach()


def per_order_err(A, B):
    """max over (stream, link, order >= 1) of ||A - B||_F / ||B||_F, and for order 0 (zero to
    rounding at the vacuum) ||A - B||_F over the largest order's ||B||_F."""
    A = A.cpu().numpy() if torch.is_tensor(A) else np.asarray(A)
    B = B.cpu().numpy() if torch.is_tensor(B) else np.asarray(B)
    scale = np.sqrt(np.sum(np.abs(B) ** 2, axis=(-1, -2))).max()
    e0 = np.sqrt(np.sum(np.abs(A[..., 0, :, :] - B[..., 0, :, :]) ** 2, axis=(-1, -2))).max() / scale
    return max(max_order_rel(A[..., 1:, :, :], B[..., 1:, :, :]), float(e0))


@pytest.fixture(scope="module")
def c4(nspt):
    g = syn.rng(syn.SEED_BASE + 4)
    U = syn.link_series(g, L_SIDE, FLUX, T, STREAMS)
    eta = syn.hermitian_noise(g, N, STREAMS * 4).reshape(STREAMS, 4, N, N)
    z = tek.twist_phases(L_SIDE, FLUX)
    tU = dev(U)
    Fb, S = drift_from_backward(nspt, tU, z)
    return dict(U=U, eta=eta, z=z, tU=tU, Fb=Fb, S=S)


def test_action_is_real_and_vacuum_order_vanishes(c4):
    S = c4["S"]
    assert torch.abs(S.imag).max().item() <= 1e-9 * max(1.0, torch.abs(S).max().item())
    assert abs(S[:, 0].real).max().item() <= 1e-9          # twist-eater vacuum: S~^(0) = 0


def test_backward_drift_equals_library_drift(nspt, c4):
    U1 = c4["tU"].clone()
    _, F = nspt.tek_langevin_step(U1, dev(c4["eta"]), FLUX, EPS, want_drift=True, algo="fft")
    assert per_order_err(c4["Fb"], F) <= 1e-10
    # F^(0) = 0 at the vacuum
    assert torch.abs(F[:, :, 0]).max().item() <= 1e-10


def test_backward_drift_equals_oracle_drift_one_stream(c4):
    Fo = tek.drift(c4["U"][0], c4["z"])
    err = per_order_err(c4["Fb"][0], torch.from_numpy(Fo).to(c4["Fb"].device))
    assert err <= 1e-10


def test_action_gradient_central_differences(nspt, c4):
    """autograd gradient of L = Re S~^(T) (stream 0) vs central differences, h = 1e-6, FP64."""
    z = c4["z"]
    U0 = c4["tU"][:1].clone()
    Ug = U0.clone().requires_grad_(True)
    action_series(nspt, Ug, z)[:, -1].real.sum().backward()
    G = Ug.grad
    h = 1e-6
    rs = np.random.default_rng(3)
    for _ in range(3):
        mu, j, a, b = int(rs.integers(4)), int(rs.integers(T + 1)), int(rs.integers(N)), int(rs.integers(N))
        for d in (1.0, 1j):
            Up, Um = U0.clone(), U0.clone()
            Up[0, mu, j, a, b] += h * d
            Um[0, mu, j, a, b] -= h * d
            lp = action_series(nspt, Up, z)[:, -1].real.sum().item()
            lm = action_series(nspt, Um, z)[:, -1].real.sum().item()
            fd = (lp - lm) / (2 * h)
            an = G[0, mu, j, a, b].real.item() if d == 1.0 else G[0, mu, j, a, b].imag.item()
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (mu, j, a, b, d, fd, an)


def _oracle_action_fftconv(U, z):
    """The truncated action (Eq. 1, beta stripped) of one stream by the oracle, with its
    FFT-CONV product (direct DFTs, pinned against Eq. 5 on the CPU) for speed."""
    from oracle import polymat as pm
    N = U.shape[-1]
    S = np.zeros(U.shape[-3], np.complex128)
    for mu in range(4):
        for nu in range(4):
            if mu == nu:
                continue
            Um, Un = U[mu], U[nu]
            P = pm.star_dftconv(pm.star_dftconv(pm.star_dftconv(Um, Un), pm.dagger(Um)), pm.dagger(Un))
            S -= z[mu, nu] * np.trace(P, axis1=-2, axis2=-1)
    S[0] += 12 * N
    return S


def test_weighted_action_gradient_vs_oracle_central_differences(nspt, c4):
    """Loss = sum_k w_k Re S~^(k) with seeded w_k ~ N(0, 1) on stream 0 (every order of the
    action, so every order of the backward's correlations): the autograd gradient through the
    library's forward and backward kernels against central differences (h = 1e-6, FP64) of the
    oracle's action at sampled link entries."""
    z = c4["z"]
    w = np.random.default_rng(41).normal(size=T + 1)
    U0 = c4["tU"][:1].clone().requires_grad_(True)
    S = action_series(nspt, U0, z)[0]
    (S.real * torch.from_numpy(w).to(S.device)).sum().backward()
    G = U0.grad[0]
    Uh = c4["U"][0]
    h = 1e-6
    rs = np.random.default_rng(42)
    for _ in range(2):
        mu, j, a, b = int(rs.integers(4)), int(rs.integers(T + 1)), int(rs.integers(N)), int(rs.integers(N))
        for d in (1.0, 1j):
            Up, Um = Uh.copy(), Uh.copy()
            Up[mu, j, a, b] += h * d
            Um[mu, j, a, b] -= h * d
            lp = float(np.dot(w, _oracle_action_fftconv(Up, z).real))
            lm = float(np.dot(w, _oracle_action_fftconv(Um, z).real))
            fd = (lp - lm) / (2 * h)
            an = G[mu, j, a, b].real.item() if d == 1.0 else G[mu, j, a, b].imag.item()
            record("c4_weighted_grad_fd", fd=fd, an=an)
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (mu, j, a, b, d, fd, an)


def test_langevin_step_with_backward_drift(nspt, c4):
    """U' = exp_star(i X) * U with X from the backward-derived drift, composed from
    library products (Horner with shrinking truncation), equals the library's step."""
    tU, Fb = c4["tU"], c4["Fb"]
    eta = dev(c4["eta"])
    X = EPS * Fb.clone()
    X[:, :, 0] = 0
    X[:, :, 1] += math.sqrt(2 * EPS) * eta
    s4 = STREAMS * 4
    Y = (1j * X).reshape(s4, T + 1, N, N).contiguous()
    I = torch.zeros_like(Y)
    I[:, 0] = torch.eye(N, dtype=Y.dtype, device=Y.device)
    R = I.clone()
    for n in range(T, 0, -1):
        R = I + nspt.polymat_mul(Y, R, algo="fft") / n
    Uf = tU.reshape(s4, T + 1, N, N).contiguous()
    Uc = nspt.polymat_mul(R, Uf, algo="fft").reshape(tU.shape)
    U1 = tU.clone()
    nspt.tek_langevin_step(U1, eta, FLUX, EPS, algo="fft")
    assert max_order_rel(host(Uc), host(U1)) <= 1e-10
    assert torch.equal(U1[:, :, 0], tU[:, :, 0])


def test_split_langevin_step_matches_fp64_form(nspt, c4):
    """The split-precision Langevin step (tensor-core staples and exp_star) against the FP64
    form at SU(121), O(g^31), 8 streams, within the stated split bound; 5 slices fail it."""
    eta = dev(c4["eta"])
    U64, Us, U5 = c4["tU"].clone(), c4["tU"].clone(), c4["tU"].clone()
    _, F64 = nspt.tek_langevin_step(U64, eta, FLUX, EPS, want_drift=True, algo="fft", prec="fp64")
    _, Fs = nspt.tek_langevin_step(Us, eta, FLUX, EPS, want_drift=True, algo="fft", prec="split")
    _, F5 = nspt.tek_langevin_step(U5, eta, FLUX, EPS, want_drift=True, algo="fft", prec="split", slices=5)
    tol = split_bound(6, "langevin", T)
    eF, eU = per_order_err(Fs, F64), max_order_rel(host(Us), host(U64))
    e5 = max(per_order_err(F5, F64), max_order_rel(host(U5), host(U64)))
    record("c4_split_vs_fp64", errF=eF, errU=eU, err_S5=e5)
    assert eF <= tol, eF
    assert eU <= tol, eU
    assert e5 > tol, e5
    assert torch.equal(Us[:, :, 0], c4["tU"][:, :, 0])


@pytest.mark.parametrize("prec", ["fp64", "split"])
def test_langevin_step_matches_oracle_one_stream(nspt, c4, prec):
    """The library's Langevin step at SU(121), O(g^31), flux 3 against the oracle's step
    (Eqs. 1-3, Taylor exp_star, Eq. 5 products) on stream 0: updated links and drift per
    order, within 1e-12 (FP64 form) or the stated split bound."""
    ref = c4.get("oracle_step")
    if ref is None:
        ref = tek.langevin_step(c4["U"][0], c4["eta"][0], c4["z"], EPS)
        c4["oracle_step"] = ref
    refU, refF = ref
    tU = c4["tU"][:1].clone()
    _, F = nspt.tek_langevin_step(tU, dev(c4["eta"][:1]), FLUX, EPS, want_drift=True, algo="fft", prec=prec)
    eU = max_order_rel(host(tU)[0], refU)
    eF = per_order_err(host(F)[0], refF)
    record("c4_vs_oracle", prec=prec, errU=eU, errF=eF)
    tol = 1e-12 if prec == "fp64" else split_bound(6, "langevin", T)
    assert eU <= tol, eU
    assert eF <= tol, eF
    np.testing.assert_array_equal(host(tU)[0][:, 0], c4["U"][0][:, 0])
