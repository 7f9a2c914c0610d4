"""Pins of the FP64 oracle against what the paper and mathematics fix.

Each test compares the oracle with something other than itself: a library
routine on a special case, exact integer arithmetic, closed forms, evaluation of
the truncated series at a small coupling against plain matrix functions, or a
finite-difference derivative of an independently written function.  A planted
mistake (a dropped term, a wrong sign, a transposed operand) fails at least one.
"""
import math
from fractions import Fraction

import numpy as np
import numpy.polynomial.polynomial as npoly
import pytest
import scipy.linalg as sla

import nspt_synth as syn
from oracle import polymat as pm
from oracle import tek

# ----------------------------------------------------------------------------
# star product (Eq. 5)
# ----------------------------------------------------------------------------


@pytest.mark.parametrize("T", [0, 1, 4, 9])
def test_star_1x1_is_scalar_polynomial_product(T):
    g = syn.rng(11 + T)
    a = syn.gaussian(g, T + 1, 1.0)
    b = syn.gaussian(g, T + 1, 1.0)
    C = pm.star(a.reshape(T + 1, 1, 1), b.reshape(T + 1, 1, 1))[:, 0, 0]
    ref = npoly.polymul(a, b)[: T + 1]
    np.testing.assert_allclose(C, ref, rtol=0, atol=1e-14)


def _exact_star(Ai, Bi):
    """Brute force over Python integers (Gaussian integers as (re, im) pairs)."""
    T1, N = Ai.shape[0], Ai.shape[1]
    out = [[[(0, 0)] * N for _ in range(N)] for _ in range(T1)]
    for k in range(T1):
        for i in range(N):
            for j in range(N):
                re = im = 0
                for l in range(k + 1):
                    for m in range(N):
                        ar, ai = int(Ai[l, i, m].real), int(Ai[l, i, m].imag)
                        br, bi = int(Bi[k - l, m, j].real), int(Bi[k - l, m, j].imag)
                        re += ar * br - ai * bi
                        im += ar * bi + ai * br
                out[k][i][j] = (re, im)
    return out


def test_star_integer_inputs_bit_exact():
    g = syn.rng(5)
    A = syn.integer_series(g, 3, 5, 1)[0]
    B = syn.integer_series(g, 3, 5, 1)[0]
    C = pm.star(A, B)
    ex = _exact_star(A, B)
    for k in range(6):
        for i in range(3):
            for j in range(3):
                assert C[k, i, j].real == ex[k][i][j][0]
                assert C[k, i, j].imag == ex[k][i][j][1]


def test_star_exact_fractions_object_arrays():
    A = np.empty((3, 2, 2), dtype=object)
    B = np.empty((3, 2, 2), dtype=object)
    vals = [Fraction(n, d) for n, d in [(1, 3), (2, 7), (-5, 11), (3, 2)]]
    for k in range(3):
        for i in range(2):
            for j in range(2):
                A[k, i, j] = vals[(k + i + 2 * j) % 4] * (k + 1)
                B[k, i, j] = vals[(2 * k + j + i) % 4] - k
    C = pm.star(A, B)
    # C_2 = A_0 B_2 + A_1 B_1 + A_2 B_0, written out entry by entry
    for i in range(2):
        for j in range(2):
            s = Fraction(0)
            for l in range(3):
                for m in range(2):
                    s += A[l, i, m] * B[2 - l, m, j]
            assert C[2, i, j] == s


def test_identity_and_shift():
    g = syn.rng(7)
    N, T = 4, 6
    A = syn.series_batch(g, N, T, 2)
    I = pm.identity_series(N, T, (2,))
    np.testing.assert_array_equal(pm.star(A, I), A)
    np.testing.assert_array_equal(pm.star(I, A), A)
    S = np.zeros_like(I)
    S[:, 1] = np.eye(N)                     # the series g * 1
    C = pm.star(A, S)
    assert np.all(C[:, 0] == 0)
    np.testing.assert_array_equal(C[:, 1:], A[:, :-1])


def test_diagonal_inputs_are_independent_scalar_products():
    g = syn.rng(8)
    N, T = 3, 5
    a = syn.gaussian(g, (T + 1, N), 1.0)
    b = syn.gaussian(g, (T + 1, N), 1.0)
    A = np.zeros((T + 1, N, N), np.complex128)
    B = np.zeros_like(A)
    for i in range(N):
        A[:, i, i] = a[:, i]
        B[:, i, i] = b[:, i]
    C = pm.star(A, B)
    for i in range(N):
        np.testing.assert_allclose(C[:, i, i], npoly.polymul(a[:, i], b[:, i])[: T + 1], atol=1e-14)
    off = C.copy()
    for i in range(N):
        off[:, i, i] = 0
    assert np.all(off == 0)


def test_star_keeps_matrix_order():
    g = syn.rng(9)
    A = syn.series_batch(g, 3, 2, 1)[0]
    B = syn.series_batch(g, 3, 2, 1)[0]
    C = pm.star(A, B)
    np.testing.assert_allclose(C[1], A[0] @ B[1] + A[1] @ B[0], atol=1e-15)
    assert np.abs(C[1] - (B[0] @ A[1] + B[1] @ A[0])).max() > 1e-3


def test_truncated_series_evaluates_to_matrix_product():
    # sum_k g^k C_k = A(g) B(g) + O(g^{T+1})
    rg = syn.rng(10)
    N, T = 4, 3
    A = syn.series_batch(rg, N, T, 1)[0]
    B = syn.series_batch(rg, N, T, 1)[0]
    C = pm.star(A, B)
    errs = []
    for gc in (1e-2, 2e-2):
        pw = gc ** np.arange(T + 1)
        Ag = np.tensordot(pw, A, 1)
        Bg = np.tensordot(pw, B, 1)
        Cg = np.tensordot(pw, C, 1)
        errs.append(np.abs(Ag @ Bg - Cg).max())
    assert errs[0] < 1e-7
    assert 2 ** (T + 1) * 0.6 < errs[1] / errs[0] < 2 ** (T + 1) * 1.6


def test_associativity_bilinearity_and_dagger():
    g = syn.rng(12)
    N, T = 4, 5
    A, B, C = (syn.series_batch(g, N, T, 1)[0] for _ in range(3))
    np.testing.assert_allclose(pm.star(pm.star(A, B), C), pm.star(A, pm.star(B, C)), atol=1e-13)
    a, b = 0.3 - 1.2j, 2.5 + 0.1j
    np.testing.assert_allclose(pm.star(a * A + b * C, B), a * pm.star(A, B) + b * pm.star(C, B), atol=1e-13)
    np.testing.assert_allclose(pm.dagger(pm.star(A, B)), pm.star(pm.dagger(B), pm.dagger(A)), atol=1e-14)


# ----------------------------------------------------------------------------
# FFT-CONV by direct DFT (Sec. 2, Steps 1-5)
# ----------------------------------------------------------------------------


def test_forward_dft_matches_library_special_case():
    # with w = exp(+2 pi i/M) and no normalisation, Step 2 equals M * numpy's ifft
    g = syn.rng(13)
    T, M = 5, 16
    A = syn.series_batch(g, 3, T, 2)
    At = pm.dft_forward(A, M)
    pad = np.zeros((2, M, 3, 3), np.complex128)
    pad[:, : T + 1] = A
    np.testing.assert_allclose(At, M * np.fft.ifft(pad, axis=1), atol=1e-13)
    back = pm.dft_inverse(At, M)
    np.testing.assert_allclose(back, np.fft.fft(At, axis=1) / M, atol=1e-14)
    np.testing.assert_allclose(back[:, : T + 1], A, atol=1e-14)


def test_twiddles_against_long_double_definition():
    for M in (2, 3, 32, 64, 128):
        w = pm.twiddle_powers(M)
        assert w[0] == 1
        np.testing.assert_allclose(np.abs(w), 1, atol=2e-16)
        np.testing.assert_allclose(w ** M, 1, atol=1e-13)
        np.testing.assert_allclose(w, np.exp(2j * np.pi * np.arange(M) / M), atol=1e-15)


@pytest.mark.parametrize("N,T", [(1, 0), (2, 1), (3, 2), (4, 7), (2, 8)])
def test_dftconv_equals_naive_bruteforce(N, T):
    g = syn.rng(100 + 10 * N + T)
    A = syn.series_batch(g, N, T, 2)
    B = syn.series_batch(g, N, T, 2)
    ref = pm.star(A, B)
    for M in {2 * T + 1, pm.default_fft_len(T), 2 * T + 3}:
        C = pm.star_dftconv(A, B, M)
        np.testing.assert_allclose(C, ref, atol=1e-13, rtol=0)


def test_dftconv_aliases_below_the_bound():
    # M = 2T wraps order 2T onto order 0: C_0 picks up A_T B_T
    g = syn.rng(21)
    N, T = 3, 4
    A = syn.series_batch(g, N, T, 1)[0]
    B = syn.series_batch(g, N, T, 1)[0]
    ref = pm.star(A, B)
    C = pm.star_dftconv(A, B, 2 * T)
    np.testing.assert_allclose(C[0], ref[0] + A[T] @ B[T], atol=1e-13)
    assert np.abs(C[0] - ref[0]).max() > 1e-2


def test_dftconv_integer_inputs_round_to_exact():
    g = syn.rng(22)
    A = syn.integer_series(g, 4, 7, 1)[0]
    B = syn.integer_series(g, 4, 7, 1)[0]
    C = pm.star_dftconv(A, B)
    ex = _exact_star(A, B)
    assert np.abs(C - np.round(C.real) - 1j * np.round(C.imag)).max() < 1e-9
    for k in range(8):
        for i in range(4):
            for j in range(4):
                assert round(C[k, i, j].real) == ex[k][i][j][0]
                assert round(C[k, i, j].imag) == ex[k][i][j][1]


# ----------------------------------------------------------------------------
# backward (truncated correlation)
# ----------------------------------------------------------------------------


def _loss(A, B, W):
    return float(np.real(np.sum(np.conj(W) * pm.star(A, B))))


def test_backward_central_finite_differences():
    g = syn.rng(31)
    N, T = 3, 4
    A = syn.series_batch(g, N, T, 1)[0]
    B = syn.series_batch(g, N, T, 1)[0]
    W = syn.gaussian(g, A.shape, 1.0)
    gA, gB = pm.star_backward(A, B, W)
    h = 1e-6
    for (X, gX, which) in ((A, gA, 0), (B, gB, 1)):
        for idx in [(0, 0, 1), (2, 1, 2), (T, 2, 0), (1, 1, 1)]:
            for d, part in ((1.0, "re"), (1j, "im")):
                Xp = X.copy()
                Xm = X.copy()
                Xp[idx] += h * d
                Xm[idx] -= h * d
                if which == 0:
                    fd = (_loss(Xp, B, W) - _loss(Xm, B, W)) / (2 * h)
                else:
                    fd = (_loss(A, Xp, W) - _loss(A, Xm, W)) / (2 * h)
                an = gX[idx].real if part == "re" else gX[idx].imag
                assert abs(fd - an) < 1e-8 * max(1.0, abs(an))


def test_backward_adjoint_identity():
    g = syn.rng(32)
    N, T = 4, 6
    A = syn.series_batch(g, N, T, 2)
    B = syn.series_batch(g, N, T, 2)
    W = syn.gaussian(g, A.shape, 1.0)
    gA, gB = pm.star_backward(A, B, W)
    lhs = np.real(np.vdot(W, pm.star(A, B)))
    # the loss is linear in each operand separately
    assert abs(lhs - np.real(np.vdot(gA, A))) < 1e-11 * abs(lhs) + 1e-12
    assert abs(lhs - np.real(np.vdot(gB, B))) < 1e-11 * abs(lhs) + 1e-12


def test_backward_1x1_is_scalar_correlation():
    g = syn.rng(33)
    T = 6
    a, b, w = (syn.gaussian(g, T + 1, 1.0) for _ in range(3))
    gA, gB = pm.star_backward(a.reshape(-1, 1, 1), b.reshape(-1, 1, 1), w.reshape(-1, 1, 1))
    # gA_j = sum_k w_k conj(b_{k-j}): numpy.correlate(w, b, 'full') at lag j
    full = np.correlate(w, b, "full")          # c[n] = sum_m w[m+n-(T)] conj(b[m])
    np.testing.assert_allclose(gA[:, 0, 0], full[T:], atol=1e-14)
    full2 = np.correlate(w, a, "full")
    np.testing.assert_allclose(gB[:, 0, 0], full2[T:], atol=1e-14)


# ----------------------------------------------------------------------------
# exp_star
# ----------------------------------------------------------------------------


def test_exp_star_single_order_closed_form():
    g = syn.rng(41)
    N, T = 3, 6
    X = syn.gaussian(g, (N, N), 1.0 / N)
    Y = np.zeros((T + 1, N, N), np.complex128)
    Y[1] = X
    E = tek.exp_star(Y)
    for k in range(T + 1):
        np.testing.assert_allclose(E[k], np.linalg.matrix_power(X, k) / math.factorial(k), atol=1e-14)


def test_exp_star_inverse_and_expm_evaluation():
    rg = syn.rng(42)
    N, T = 3, 4
    Y = syn.gaussian(rg, (T + 1, N, N), 1.0 / N)
    Y[0] = 0
    E = tek.exp_star(Y)
    Einv = tek.exp_star(-Y)
    I = pm.identity_series(N, T)
    np.testing.assert_allclose(pm.star(E, Einv), I, atol=1e-14)
    errs = []
    for gc in (1e-2, 2e-2):
        pw = gc ** np.arange(T + 1)
        ref = sla.expm(np.tensordot(pw, Y, 1))
        errs.append(np.abs(np.tensordot(pw, E, 1) - ref).max())
    assert errs[0] < 1e-9
    assert 2 ** (T + 1) * 0.5 < errs[1] / errs[0] < 2 ** (T + 1) * 1.7


# ----------------------------------------------------------------------------
# TEK: twist, action, drift, Langevin
# ----------------------------------------------------------------------------


@pytest.mark.parametrize("L,k", [(3, 1), (5, 2), (11, 3)])
def test_twist_eaters_satisfy_twisted_vacuum(L, k):
    G = syn.twist_eaters(L, k)
    z = tek.twist_phases(L, k)
    N = L * L
    for mu in range(4):
        np.testing.assert_allclose(G[mu] @ G[mu].conj().T, np.eye(N), atol=1e-12)
        assert abs(np.linalg.det(G[mu]) - 1) < 1e-10
        for nu in range(4):
            if mu == nu:
                continue
            P = z[mu, nu] * G[mu] @ G[nu] @ G[mu].conj().T @ G[nu].conj().T
            np.testing.assert_allclose(P, np.eye(N), atol=1e-12)
            assert z[nu, mu] == np.conj(z[mu, nu])


def test_vacuum_has_zero_action_and_force():
    L, k, T = 3, 1, 3
    N = L * L
    U = np.zeros((4, T + 1, N, N), np.complex128)
    U[:, 0] = syn.twist_eaters(L, k)
    z = tek.twist_phases(L, k)
    S = tek.action(U, z)
    assert np.abs(S).max() < 1e-12
    F = tek.drift(U, z)
    assert np.abs(F).max() < 1e-12


def test_action_is_real_and_drift_hermitian_traceless():
    g = syn.rng(51)
    U = syn.link_series(g, 3, 1, 3, 1)[0]
    z = tek.twist_phases(3, 1)
    S = tek.action(U, z)
    assert np.abs(S.imag).max() < 1e-12 * max(1, np.abs(S).max())
    F = tek.drift(U, z)
    np.testing.assert_allclose(F, np.conj(np.swapaxes(F, -1, -2)), atol=1e-13)
    assert np.abs(np.trace(F, axis1=-2, axis2=-1)).max() < 1e-13


def _staple_minus_sign(U, z):
    """The staple with the second term's sign as printed in Eqs. 2-3 (minus):
    a planted alternative that the finite-difference test must reject."""
    out = np.zeros_like(U)
    for mu in range(4):
        Um = U[mu]
        Umd = pm.dagger(Um)
        inner = np.zeros_like(Um)
        for nu in range(4):
            if nu == mu:
                continue
            Un, Und = U[nu], pm.dagger(U[nu])
            inner += z[mu, nu] * pm.star(pm.star(Un, Umd), Und)
            inner -= np.conj(z[mu, nu]) * pm.star(pm.star(Und, Umd), Un)
        out[mu] = pm.star(Um, inner)
    return out


def _fd_drift_check(U, z, F, mu, X, h=1e-5):
    """Returns max_k |dS~^(k)/de - (-Tr[X F^(k)])| and the scale."""
    Up, Um = U.copy(), U.copy()
    Ep, Em = sla.expm(1j * h * X), sla.expm(-1j * h * X)
    Up[mu] = Ep[None] @ U[mu]
    Um[mu] = Em[None] @ U[mu]
    dS = (tek.action(Up, z) - tek.action(Um, z)) / (2 * h)
    pred = -np.einsum("ij,kji->k", X, F[mu])
    return np.abs(dS - pred).max(), np.abs(pred).max()


def test_drift_is_minus_gradient_of_truncated_action():
    g = syn.rng(52)
    L, k, T = 3, 1, 3
    U = syn.link_series(g, L, k, T, 1)[0]
    # a non-vacuum order 0 so that every order has a nonzero drift
    U[:, 0] = syn.haar_sun(g, L * L, 4)
    z = tek.twist_phases(L, k)
    F = tek.drift(U, z)
    X = syn.hermitian_traceless(g, L * L, 1)[0]
    for mu in range(4):
        err, scale = _fd_drift_check(U, z, F, mu, X)
        assert err < 1e-7 * scale, (mu, err, scale)
    # planted mistake: the minus-sign staple violates the identity
    S_bad = _staple_minus_sign(U, z)
    N = L * L
    D = S_bad - np.conj(np.swapaxes(S_bad, -1, -2))
    D = D - (np.trace(D, axis1=-2, axis2=-1) / N)[..., None, None] * np.eye(N)
    F_bad = 1j * D
    err, scale = _fd_drift_check(U, z, F_bad, 0, X)
    assert err > 1e-3 * scale


def _nonpert_staple(Ug, z):
    S = []
    for mu in range(4):
        Um = Ug[mu]
        acc = np.zeros_like(Um)
        for nu in range(4):
            if nu == mu:
                continue
            Un = Ug[nu]
            acc += z[mu, nu] * Un @ Um.conj().T @ Un.conj().T
            acc += np.conj(z[mu, nu]) * Un.conj().T @ Um.conj().T @ Un
        S.append(Um @ acc)
    return np.stack(S)


def test_langevin_step_matches_nonperturbative_update():
    # sum_k g^k U'^(k) = expm(i X(g)) U(g) + O(g^{T+1}) with
    # X(g) = eps (F(g) - F^(0)) + g sqrt(2 eps) eta and F(g) from plain products
    rg = syn.rng(53)
    L, k, T, eps = 3, 1, 3, 0.05
    N = L * L
    U = syn.link_series(rg, L, k, T, 1)[0]
    U[:, 0] = syn.haar_sun(rg, N, 4)           # generic order 0: F^(0) != 0
    eta = syn.hermitian_noise(rg, N, 4)
    z = tek.twist_phases(L, k)
    Unew, F = tek.langevin_step(U, eta, z, eps)
    errs = []
    for gc in (5e-3, 1e-2):
        pw = gc ** np.arange(T + 1)
        Ug = np.einsum("k,mkij->mij", pw, U)
        S = _nonpert_staple(Ug, z)
        D = S - np.conj(np.swapaxes(S, -1, -2))
        D = D - (np.trace(D, axis1=-2, axis2=-1) / N)[:, None, None] * np.eye(N)
        Fg = 1j * D
        ref = []
        for mu in range(4):
            Xg = eps * (Fg[mu] - F[mu, 0]) + gc * math.sqrt(2 * eps) * eta[mu]
            ref.append(sla.expm(1j * Xg) @ Ug[mu])
        ref = np.stack(ref)
        got = np.einsum("k,mkij->mij", pw, Unew)
        errs.append(np.abs(got - ref).max())
    assert errs[0] < 1e-8
    assert 2 ** (T + 1) * 0.5 < errs[1] / errs[0] < 2 ** (T + 1) * 1.7


def _unitary_series(rg, L, k, T):
    N = L * L
    H = syn.gaussian(rg, (4, T + 1, N, N), 1.0 / N)
    H = 0.5 * (H + np.conj(np.swapaxes(H, -1, -2)))
    H[:, 0] = 0
    E = tek.exp_star(1j * H)
    G = np.zeros((4, T + 1, N, N), np.complex128)
    G[:, 0] = syn.twist_eaters(L, k)
    return pm.star(E, G)


def test_langevin_step_preserves_unitary_series():
    rg = syn.rng(54)
    L, k, T = 3, 1, 4
    N = L * L
    U = _unitary_series(rg, L, k, T)
    I = pm.identity_series(N, T, (4,))
    np.testing.assert_allclose(pm.star(U, pm.dagger(U)), I, atol=1e-13)
    eta = syn.hermitian_noise(rg, N, 4)
    Unew, F = tek.langevin_step(U, eta, tek.twist_phases(L, k), 0.01)
    np.testing.assert_allclose(pm.star(Unew, pm.dagger(Unew)), I, atol=1e-13)
    np.testing.assert_array_equal(Unew[:, 0], U[:, 0])
    assert np.abs(Unew - U).max() > 1e-3


def test_langevin_small_eps_first_order():
    rg = syn.rng(55)
    L, k, T = 3, 1, 3
    U = syn.link_series(rg, L, k, T, 1)[0]
    z = tek.twist_phases(L, k)
    eta = np.zeros((4, 9, 9), np.complex128)
    d = []
    for eps in (1e-4, 2e-4):
        Unew, F = tek.langevin_step(U, eta, z, eps)
        X = F.copy()
        X[:, 0] = 0
        lin = 1j * pm.star(X, U)
        d.append(np.abs((Unew - U) / eps - lin).max())
        scale = np.abs(lin).max()
    assert d[0] < 1e-3 * scale
    assert 1.6 < d[1] / d[0] < 2.4


# ----------------------------------------------------------------------------
# molecular dynamics (leapfrog with momentum refresh)
# ----------------------------------------------------------------------------


def test_md_step_is_time_reversible():
    """Leapfrog is reversible: step, flip the momentum, step again -> back to the start
    (exact in the truncated ring, so up to rounding)."""
    rg = syn.rng(61)
    L, k, T = 3, 1, 4
    N = L * L
    U = syn.link_series(rg, L, k, T, 1)[0]
    P = np.zeros_like(U)
    P[:, 1] = syn.hermitian_noise(rg, N, 4)
    P[:, 2:] = 0.3 * syn.hermitian_traceless(rg, N, 4 * (T - 1)).reshape(4, T - 1, N, N)
    z = tek.twist_phases(L, k)
    U1, P1 = tek.md_step(U, P, z, 0.05)
    U2, P2 = tek.md_step(U1, -P1, z, 0.05)
    np.testing.assert_allclose(U2, U, atol=1e-12)
    np.testing.assert_allclose(-P2, P, atol=1e-12)
    assert np.abs(U1 - U).max() > 1e-3


def test_md_step_matches_nonperturbative_leapfrog():
    """sum_k g^k of the series step equals the leapfrog of the matrix equations
    U' = exp(i eps Ph(g)) U(g), Ph = P(g) + eps/2 (F(g) - F^(0)) ... to O(g^{T+1})."""
    rg = syn.rng(62)
    L, k, T, eps = 3, 1, 3, 0.07
    N = L * L
    U = syn.link_series(rg, L, k, T, 1)[0]
    U[:, 0] = syn.haar_sun(rg, N, 4)           # generic order 0: F^(0) != 0 is dropped
    P = np.zeros_like(U)
    P[:, 1] = syn.hermitian_noise(rg, N, 4)
    z = tek.twist_phases(L, k)
    U1, P1 = tek.md_step(U, P, z, eps)

    def force(Ug):
        S = _nonpert_staple(Ug, z)
        D = S - np.conj(np.swapaxes(S, -1, -2))
        D = D - (np.trace(D, axis1=-2, axis2=-1) / N)[:, None, None] * np.eye(N)
        return 1j * D

    F0 = tek.drift(U, z)[:, 0]                  # order-0 parts removed at both force evaluations
    errs = []
    for gc in (5e-3, 1e-2):
        pw = gc ** np.arange(T + 1)
        Ug = np.einsum("k,mkij->mij", pw, U)
        Pg = np.einsum("k,mkij->mij", pw, P)
        Ph = Pg + 0.5 * eps * (force(Ug) - F0)
        U1g = np.stack([sla.expm(1j * eps * Ph[m]) @ Ug[m] for m in range(4)])
        F0b = tek.drift(U1, z)[:, 0]
        P1g = Ph + 0.5 * eps * (force(U1g) - F0b)
        errs.append(max(np.abs(np.einsum("k,mkij->mij", pw, U1) - U1g).max(),
                        np.abs(np.einsum("k,mkij->mij", pw, P1) - P1g).max()))
    assert errs[0] < 1e-8
    assert 2 ** (T + 1) * 0.5 < errs[1] / errs[0] < 2 ** (T + 1) * 1.7


def test_md_trajectory_refresh_and_vacuum():
    rg = syn.rng(63)
    L, k, T = 3, 1, 3
    N = L * L
    U = np.zeros((4, T + 1, N, N), np.complex128)
    U[:, 0] = syn.twist_eaters(L, k)
    z = tek.twist_phases(L, k)
    # the vacuum with zero momentum is a fixed point of the dynamics
    U0, P0 = tek.md_trajectory(U, np.zeros((4, N, N)), z, 0.1, 3)
    assert np.abs(U0 - U).max() < 1e-13 and np.abs(P0).max() < 1e-13
    # with refreshed momentum the links move, order 0 never does, and P^(0) stays 0
    eta = syn.hermitian_noise(rg, N, 4)
    U1, P1 = tek.md_trajectory(U, eta, z, 0.1, 3)
    np.testing.assert_array_equal(U1[:, 0], U[:, 0])
    assert np.all(P1[:, 0] == 0)
    assert np.abs(U1[:, 1]).max() > 1e-2
    # momentum and drift stay Hermitian and traceless order by order
    np.testing.assert_allclose(P1, np.conj(np.swapaxes(P1, -1, -2)), atol=1e-13)
    assert np.abs(np.trace(P1, axis1=-2, axis2=-1)).max() < 1e-12


# ---------------------------------------------------------------------------
# Wilson loops (the measured observable)
# ---------------------------------------------------------------------------
def test_wilson_loops_twist_eater_vacuum_is_one():
    """Gamma_mu Gamma_nu = conj(z_{mu nu}) Gamma_nu Gamma_mu gives
    Gamma_mu^a Gamma_nu^b Gamma_mu^-a Gamma_nu^-b = conj(z)^(ab): every loop is 1 at order 0
    and vanishes at higher orders of the pure vacuum."""
    for L, k in ((3, 1), (5, 2)):
        N = L * L
        U = np.zeros((4, 4, N, N), np.complex128)
        U[:, 0] = syn.twist_eaters(L, k)
        W = tek.wilson_loops(U, tek.twist_phases(L, k), 3)
        np.testing.assert_allclose(W[..., 0], np.ones((3, 3)), atol=1e-12)
        assert np.abs(W[..., 1:]).max() < 1e-13


def test_wilson_loops_match_nonperturbative_loops():
    """sum_k g^k W(a,b)^(k) equals the matrix Wilson loop of U(g) = sum_k g^k U^(k)
    (real g) up to O(g^{T+1})."""
    rg = syn.rng(71)
    L, k, T, amax = 3, 1, 3, 2
    N = L * L
    U = syn.link_series(rg, L, k, T, 1)[0]
    z = tek.twist_phases(L, k)
    W = tek.wilson_loops(U, z, amax)
    errs = []
    for gc in (5e-3, 1e-2):
        pw = gc ** np.arange(T + 1)
        Ug = np.einsum("k,mkij->mij", pw, U)
        ref = np.zeros((amax, amax), np.complex128)
        for mu in range(4):
            for nu in range(4):
                if mu == nu:
                    continue
                for a in range(1, amax + 1):
                    for b in range(1, amax + 1):
                        A = np.linalg.matrix_power(Ug[mu], a)
                        B = np.linalg.matrix_power(Ug[nu], b)
                        ref[a - 1, b - 1] += z[mu, nu] ** (a * b) * np.trace(A @ B @ A.conj().T @ B.conj().T)
        ref /= 12 * N
        got = np.einsum("k,abk->ab", pw, W)
        errs.append(np.abs(got - ref).max())
    assert errs[0] < 1e-8
    assert 2 ** (T + 1) * 0.5 < errs[1] / errs[0] < 2 ** (T + 1) * 1.7


def test_wilson_1x1_is_the_plaquette_of_the_action():
    rg = syn.rng(72)
    L, k, T = 3, 1, 4
    N = L * L
    U = syn.link_series(rg, L, k, T, 2)
    z = tek.twist_phases(L, k)
    W = tek.wilson_loops(U, z, 1)
    S = tek.action(U, z)
    expect = -S / (12 * N)
    expect[..., 0] += 1.0
    np.testing.assert_allclose(W[..., 0, 0, :], expect, atol=1e-12)


def test_wilson_loops_conjugation_symmetry():
    """The (nu, mu) plane with extents (b, a) is the dagger of the (mu, nu) plane with (a, b),
    and z_{nu mu} = conj(z_{mu nu}), so W(a, b) = conj(W(b, a)) order by order."""
    rg = syn.rng(73)
    U = syn.link_series(rg, 3, 1, 3, 1)[0]
    W = tek.wilson_loops(U, tek.twist_phases(3, 1), 3)
    np.testing.assert_allclose(W, np.conj(np.swapaxes(W, 0, 1)), atol=1e-12)


# ----------------------------------------------------------------------------
# unitarity projection (polar factor in the truncated ring)
# ----------------------------------------------------------------------------
def test_binomial_coefficients_are_the_inverse_square_root_series():
    # (1 + x)^(-1/2) by numpy's polynomial powers: the coefficients square to 1/(1 + x)
    c = np.array([tek.binom_minus_half(n) for n in range(12)])
    sq = np.polynomial.polynomial.polymul(c, c)[:12]
    inv = np.array([(-1.0) ** n for n in range(12)])
    np.testing.assert_allclose(sq, inv, atol=1e-12)
    assert [tek.binom_minus_half(n) for n in range(4)] == [1.0, -0.5, 0.375, -0.3125]


def test_unitarize_leaves_a_unitary_series_unchanged():
    rg = syn.rng(70)
    U = _unitary_series(rg, 3, 1, 5)
    V = tek.unitarize(U)
    np.testing.assert_allclose(V, U, atol=1e-13)
    np.testing.assert_array_equal(V[:, 0], U[:, 0])


def test_unitarize_output_is_unitary_and_idempotent():
    rg = syn.rng(71)
    L, k, T = 3, 1, 6
    N = L * L
    U = syn.link_series(rg, L, k, T, 1)[0]          # Gaussian higher orders: not unitary
    I = pm.identity_series(N, T, (4,))
    assert np.abs(pm.star(pm.dagger(U), U) - I).max() > 1e-2
    V = tek.unitarize(U)
    np.testing.assert_allclose(pm.star(pm.dagger(V), V), I, atol=1e-13)
    np.testing.assert_allclose(pm.star(V, pm.dagger(V)), I, atol=1e-13)
    np.testing.assert_allclose(tek.unitarize(V), V, atol=1e-13)
    np.testing.assert_array_equal(V[:, 0], U[:, 0])


def test_unitarize_matches_nonperturbative_polar_factor():
    # sum_k g^k V^(k) = polar factor of U(g) (scipy) + O(g^{T+1})
    rg = syn.rng(72)
    L, k, T = 3, 1, 3
    N = L * L
    U = syn.link_series(rg, L, k, T, 1)[0]
    U[:, 0] = syn.haar_sun(rg, N, 4)
    V = tek.unitarize(U)
    errs = []
    for gc in (5e-3, 1e-2):
        pw = gc ** np.arange(T + 1)
        Ug = np.einsum("k,mkij->mij", pw, U)
        ref = np.stack([sla.polar(Ug[m])[0] for m in range(4)])
        got = np.einsum("k,mkij->mij", pw, V)
        errs.append(np.abs(got - ref).max())
    assert errs[0] < 1e-8
    assert 2 ** (T + 1) * 0.5 < errs[1] / errs[0] < 2 ** (T + 1) * 1.7


def test_unitarize_1x1_is_the_phase_of_a_scalar_series():
    # a scalar series u(g) with |u0| = 1: v(g) = u(g) / |u(g)|, Taylor coefficients by exact
    # rational arithmetic on u(g) = u0 (1 + a g) for real a: v = u0 (1 + a g)/|1 + a g| = u0
    # (sign of 1 + a g) = u0 for small g, so every order above 0 vanishes
    T = 6
    u = np.zeros((T + 1, 1, 1), np.complex128)
    u[0] = np.exp(0.3j)
    u[1] = 0.7 * np.exp(0.3j)
    v = tek.unitarize(u)
    np.testing.assert_allclose(v[1:], 0, atol=1e-15)
    # a purely imaginary first order, u = u0 (1 + i b g): v = u0 (1 + i b g) / sqrt(1 + b^2 g^2)
    b = 0.4
    u[1] = 1j * b * np.exp(0.3j)
    v = tek.unitarize(u)[:, 0, 0] / np.exp(0.3j)
    ref = np.zeros(T + 1, np.complex128)
    from scipy.special import binom
    for n in range(T // 2 + 1):       # (1 + b^2 g^2)^(-1/2) = sum_n binom(-1/2, n) b^(2n) g^(2n)
        c = binom(-0.5, n) * b ** (2 * n)
        ref[2 * n] += c
        if 2 * n + 1 <= T:
            ref[2 * n + 1] += 1j * b * c
    np.testing.assert_allclose(v, ref, atol=1e-15)


def test_log_star_and_scalar_exp_special_cases():
    # scalar series: log(1 + d) and exp(b) against numpy polynomial arithmetic
    T = 7
    rg = np.random.default_rng(73)
    d = np.zeros(T + 1, np.complex128)
    d[1:] = rg.normal(size=T) + 1j * rg.normal(size=T)
    L = tek.log_star_unit(d.reshape(T + 1, 1, 1))[:, 0, 0]
    # exp of the log series gives back 1 + d (truncated)
    np.testing.assert_allclose(tek.scalar_exp(L), np.r_[1.0, d[1:]], atol=1e-12)
    # exp(b) for b = c g: c^k / k!
    b = np.zeros(T + 1, np.complex128)
    b[1] = 0.3 - 0.2j
    ref = np.array([b[1] ** k / math.factorial(k) for k in range(T + 1)])
    np.testing.assert_allclose(tek.scalar_exp(b), ref, atol=1e-15)
    # log of a commuting (diagonal) matrix series: entrywise scalar logs
    D = np.zeros((T + 1, 2, 2), np.complex128)
    D[1:, 0, 0] = d[1:]
    D[1:, 1, 1] = np.conj(d[1:])
    LD = tek.log_star_unit(D)
    np.testing.assert_allclose(LD[:, 0, 0], L, atol=1e-13)
    np.testing.assert_allclose(LD[:, 1, 1], tek.log_star_unit(np.conj(d).reshape(T + 1, 1, 1))[:, 0, 0], atol=1e-13)


def test_u1_phase_removal_fixes_the_determinant_nonperturbatively():
    # sum_k g^k W^(k) = polar(U(g)) * (det U0 / det polar(U(g)))^(1/N) + O(g^{T+1})
    rg = syn.rng(74)
    L, k, T = 3, 1, 3
    N = L * L
    U = syn.link_series(rg, L, k, T, 1)[0]
    U[:, 0] = syn.haar_sun(rg, N, 4)
    W = tek.unitarize(U, special=True)
    errs, dets = [], []
    for gc in (5e-3, 1e-2):
        pw = gc ** np.arange(T + 1)
        Ug = np.einsum("k,mkij->mij", pw, U)
        ref = []
        for m in range(4):
            P = sla.polar(Ug[m])[0]
            ratio = np.linalg.det(U[m, 0]) / np.linalg.det(P)
            ref.append(P * ratio ** (1.0 / N))
        got = np.einsum("k,mkij->mij", pw, W)
        errs.append(np.abs(got - np.stack(ref)).max())
        dets.append(max(abs(np.linalg.det(got[m]) - np.linalg.det(U[m, 0])) for m in range(4)))
    assert errs[0] < 1e-8
    assert 2 ** (T + 1) * 0.5 < errs[1] / errs[0] < 2 ** (T + 1) * 1.7
    assert dets[0] < 1e-8 and 2 ** (T + 1) * 0.5 < dets[1] / dets[0] < 2 ** (T + 1) * 1.7


def test_u1_phase_removal_keeps_special_unitary_series():
    # an SU(N)-type series exp_star(i H) * Gamma with traceless H has no U(1) phase to remove
    rg = syn.rng(75)
    L, k, T = 3, 1, 5
    N = L * L
    H = syn.gaussian(rg, (4, T + 1, N, N), 1.0 / N)
    H = 0.5 * (H + np.conj(np.swapaxes(H, -1, -2)))
    H = H - (np.trace(H, axis1=-2, axis2=-1) / N)[..., None, None] * np.eye(N)
    H[:, 0] = 0
    G = np.zeros((4, T + 1, N, N), np.complex128)
    G[:, 0] = syn.twist_eaters(L, k)
    U = pm.star(tek.exp_star(1j * H), G)
    np.testing.assert_allclose(tek.unitarize(U, special=True), U, atol=1e-13)
    # a phase-rotated one gets its phase removed: U * exp(i c g) (scalar) -> U
    c = 0.37
    ph = tek.scalar_exp(np.r_[0.0, 1j * c, np.zeros(T - 1)])
    Ur = np.zeros_like(U)
    for kk in range(T + 1):
        for j in range(kk + 1):
            Ur[:, kk] += U[:, j] * ph[kk - j]
    np.testing.assert_allclose(tek.unitarize(Ur, special=True), U, atol=1e-12)


def test_u1_phase_from_jacobis_formula_equals_the_log_definition():
    # for a unitary series V: Im Tr log(V0^+ V)_k = Im Tr(V^+ * V')_(k-1) / k, V'_j = (j+1) V_(j+1)
    rg = syn.rng(76)
    L, k, T = 3, 1, 8
    U = tek.unitarize(syn.link_series(rg, L, k, T, 1)[0])
    V0h = np.zeros_like(U)
    V0h[:, 0] = np.conj(np.swapaxes(U[:, 0], -1, -2))
    D = pm.star(V0h, U)
    D[:, 0] = 0
    a_log = np.imag(np.trace(tek.log_star_unit(D), axis1=-2, axis2=-1))
    Vp = np.zeros_like(U)
    Vp[:, :T] = U[:, 1:] * np.arange(1, T + 1)[None, :, None, None]
    t = np.imag(np.trace(pm.star(pm.dagger(U), Vp), axis1=-2, axis2=-1))
    a_jac = np.zeros_like(a_log)
    a_jac[:, 1:] = t[:, :T] / np.arange(1, T + 1)[None, :]
    np.testing.assert_allclose(a_jac, a_log, atol=1e-11 * np.abs(a_log).max())
    assert np.abs(a_log[:, 1:]).max() > 1e-3
