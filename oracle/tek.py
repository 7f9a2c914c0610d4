"""Oracle for the twisted Eguchi-Kawai (TEK) pieces of one NSPT Langevin step.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Links are series U of shape (..., 4, T+1, N, N) with N = L^2.  All products
are the oracle star product of ``polymat``.  Readings of the paper that these
functions fix (each pinned by a test):

* twist: z_{mu nu} = exp(2 pi i k eps_{mu nu} / L) with eps = +1 for mu < nu and
  -1 for mu > nu, so z_{nu mu} = conj(z_{mu nu}) (Eq. 1, antisymmetric exponent);
* staple: the second term of S_mu enters with a PLUS sign,
  S_mu = U_mu star sum_{nu != mu} [ z_{mu nu} U_nu U_mu^+ U_nu^+
                                   + conj(z_{mu nu}) U_nu^+ U_mu^+ U_nu ],
  which is what differentiating the action of Eq. 1 gives (Eqs. 2-3 print a
  minus; the finite-difference drift test fails for the minus sign);
* drift: F^(k) = i [S^(k) - S^(k)^H - Tr(S^(k) - S^(k)^H)/N], with beta
  absorbed by the rescaled time of Eq. 3;
* Langevin step (Euler-Maruyama in the rescaled time):
  X^(0) = 0, X^(1) = eps F^(1) + sqrt(2 eps) eta, X^(k>=2) = eps F^(k),
  U' = exp_star(i X) star U; order 0 of U is left unchanged;
* unitarity projection (the paper names a unitarity projection among the NSPT
  steps but prints no algorithm): the polar factor of the series in the
  truncated ring, V = U * (U^+ * U)^(-1/2), with order 0 (unitary) kept as it is;
  optionally followed by the removal of the U(1) (trace, zero-mode) phase, so that
  det V = det U^(0) through order T; see ``unitarize``;
* Wilson loops: W(a, b) = 1/(12 N) sum over ordered planes of
  z_{mu nu}^(ab) Tr[U_mu^a U_nu^b (U_mu^a)^+ (U_nu^b)^+] (the paper measures Wilson
  loops but does not restate their definition; the z^(ab) factor makes the
  twist-eater vacuum value exactly 1).
"""
from __future__ import annotations

import math

import numpy as np

from . import polymat as pm


def twist_phases(L: int, flux: int) -> np.ndarray:
    """4 x 4 complex array z[mu, nu] = exp(2 pi i flux eps_{mu nu} / L); the
    diagonal (never used) is set to 0."""
    z = np.zeros((4, 4), np.complex128)
    for mu in range(4):
        for nu in range(4):
            if mu == nu:
                continue
            eps = 1 if mu < nu else -1
            z[mu, nu] = np.exp(2j * np.pi * flux * eps / L)
    return z


def plaquette(U, z, mu: int, nu: int):
    """Series of z_{mu nu} U_mu U_nu U_mu^+ U_nu^+ (the Eq. 1 plaquette)."""
    Um, Un = U[..., mu, :, :, :], U[..., nu, :, :, :]
    P = pm.star(pm.star(pm.star(Um, Un), pm.dagger(Um)), pm.dagger(Un))
    return z[mu, nu] * P


def action(U, z) -> np.ndarray:
    """Order-truncated TEK action with beta stripped (Eq. 1):
    S~^(k) = 12 N delta_{k0} - sum_{mu != nu} Tr[ (z U_mu U_nu U_mu^+ U_nu^+)^(k) ].
    Returns shape (..., T+1), complex (real up to rounding)."""
    U = np.asarray(U)
    N = U.shape[-1]
    T = U.shape[-3] - 1
    S = np.zeros(U.shape[:-4] + (T + 1,), np.complex128)
    for mu in range(4):
        for nu in range(4):
            if mu == nu:
                continue
            P = plaquette(U, z, mu, nu)
            S = S - np.trace(P, axis1=-2, axis2=-1)
    S[..., 0] += 12 * N
    return S


def staple(U, z) -> np.ndarray:
    """S_mu^(k) of Eq. 3 (plus sign on the second term, see the module
    docstring), for mu = 0..3.  Shape (..., 4, T+1, N, N)."""
    U = np.asarray(U)
    out = np.zeros_like(U, dtype=np.complex128)
    for mu in range(4):
        Um = U[..., mu, :, :, :]
        Umd = pm.dagger(Um)
        inner = np.zeros_like(Um, dtype=np.complex128)
        for nu in range(4):
            if nu == mu:
                continue
            Un = U[..., nu, :, :, :]
            Und = pm.dagger(Un)
            inner = inner + z[mu, nu] * pm.star(pm.star(Un, Umd), Und)
            inner = inner + np.conj(z[mu, nu]) * pm.star(pm.star(Und, Umd), Un)
        out[..., mu, :, :, :] = pm.star(Um, inner)
    return out


def drift(U, z) -> np.ndarray:
    """F_mu^(k) = i [S^(k) - S^(k)^H - Tr(S^(k) - S^(k)^H)/N] (Eqs. 2-3, beta
    absorbed).  Hermitian and traceless order by order."""
    S = staple(U, z)
    N = S.shape[-1]
    D = S - np.conj(np.swapaxes(S, -1, -2))
    tr = np.trace(D, axis1=-2, axis2=-1)
    D = D - (tr / N)[..., None, None] * np.eye(N)
    return 1j * D


def exp_star(Y) -> np.ndarray:
    """exp_star(Y) = sum_{n=0}^{T} Y^{star n} / n! for a series with Y^(0) = 0
    (then Y^{star n} starts at order n and the sum is exact through order T)."""
    Y = np.asarray(Y, np.complex128)
    if np.any(Y[..., 0, :, :] != 0):
        raise ValueError("exp_star needs Y^(0) = 0")
    T = Y.shape[-3] - 1
    N = Y.shape[-1]
    E = pm.identity_series(N, T, Y.shape[:-3])
    P = E.copy()
    for n in range(1, T + 1):
        P = pm.star(P, Y) / n
        E = E + P
    return E


def langevin_step(U, eta, z, eps: float):
    """One NSPT Langevin step of all four links (Eq. 3 in rescaled time).

    U   : (..., 4, T+1, N, N) link series
    eta : (..., 4, N, N) traceless Hermitian Gaussian noise (order g^1)
    Returns (U_new, F) with F the drift of the input links.
    """
    U = np.asarray(U, np.complex128)
    eta = np.asarray(eta, np.complex128)
    F = drift(U, z)
    X = eps * F
    X[..., :, 0, :, :] = 0.0
    if X.shape[-3] > 1:
        X[..., :, 1, :, :] += math.sqrt(2.0 * eps) * eta
    Unew = pm.star(exp_star(1j * X), U)
    return Unew, F


def md_step(U, P, z, eps: float):
    """One leapfrog step of the NSPT molecular dynamics (Eq. 3 with beta absorbed by the
    rescaled time): the momentum series P~ = sum_{k>=1} g^k P^(k) (stored with P^(0) = 0),
    dU^(k)/dt = i (P~ * U)^(k), dP^(k)/dt = F^(k) for k >= 1 (order 0 of F is dropped:
    the momentum has no order g^0):
        P_half = P + eps/2 F(U);  U' = exp_star(i eps P_half) * U;  P' = P_half + eps/2 F(U').
    Returns (U', P')."""
    U = np.asarray(U, np.complex128)
    P = np.array(P, np.complex128)
    P[..., :, 0, :, :] = 0.0
    F = drift(U, z)
    F[..., :, 0, :, :] = 0.0
    Ph = P + 0.5 * eps * F
    Unew = pm.star(exp_star(1j * eps * Ph), U)
    F2 = drift(Unew, z)
    F2[..., :, 0, :, :] = 0.0
    return Unew, Ph + 0.5 * eps * F2


def md_trajectory(U, eta, z, eps: float, nsteps: int):
    """Momentum refresh (P^(1) = eta, higher orders 0) followed by `nsteps` leapfrog steps."""
    U = np.asarray(U, np.complex128)
    P = np.zeros_like(U)
    P[..., :, 1, :, :] = eta
    for _ in range(nsteps):
        U, P = md_step(U, P, z, eps)
    return U, P


def wilson_loops(U, z, amax: int) -> np.ndarray:
    """Perturbative coefficients of the plane-averaged a x b Wilson loops of the TEK
    model (the observables the NSPT runs measure, Sec. 1):
        W(a, b)^(k) = 1/(12 N) sum_{mu != nu} z_{mu nu}^(a b) Tr[(U_mu^a U_nu^b (U_mu^a)^+ (U_nu^b)^+)^(k)],
    powers and products being star products of the link series.  Returns shape
    (..., amax, amax, T+1) with [a-1, b-1, k]; W(1, 1) is the plaquette of Eq. 1."""
    U = np.asarray(U, np.complex128)
    N = U.shape[-1]
    T = U.shape[-3] - 1
    powers = []
    for mu in range(4):
        pw = [None, U[..., mu, :, :, :]]
        for _ in range(2, amax + 1):
            pw.append(pm.star(pw[-1], U[..., mu, :, :, :]))
        powers.append(pw)
    W = np.zeros(U.shape[:-4] + (amax, amax, T + 1), np.complex128)
    for mu in range(4):
        for nu in range(4):
            if mu == nu:
                continue
            for a in range(1, amax + 1):
                for b in range(1, amax + 1):
                    A, B = powers[mu][a], powers[nu][b]
                    X = pm.star(pm.star(pm.star(A, B), pm.dagger(A)), pm.dagger(B))
                    W[..., a - 1, b - 1, :] += z[mu, nu] ** (a * b) * np.trace(X, axis1=-2, axis2=-1)
    return W / (12 * N)


def binom_minus_half(n: int) -> float:
    """Coefficient of x^n in (1 + x)^(-1/2): (-1)^n (2n)! / (4^n (n!)^2)."""
    return (-1) ** n * math.comb(2 * n, n) / 4.0 ** n


def log_star_unit(D) -> np.ndarray:
    """log_star(1 + D) = sum_{n=1}^{T} (-1)^(n+1) D^{star n} / n for a series with D^(0) = 0
    (exact through order T)."""
    D = np.asarray(D, np.complex128)
    if np.any(D[..., 0, :, :] != 0):
        raise ValueError("log_star_unit needs D^(0) = 0")
    T = D.shape[-3] - 1
    out = np.zeros_like(D)
    P = D.copy()
    for n in range(1, T + 1):
        out = out + ((-1) ** (n + 1) / n) * P
        P = pm.star(P, D)
    return out


def scalar_exp(b) -> np.ndarray:
    """Coefficients of exp(b(g)) for a scalar series b with b_0 = 0, shape (..., T+1), by
    k s_k = sum_{j=1}^{k} j b_j s_{k-j}, s_0 = 1 (the derivative of exp(b) is b' exp(b))."""
    b = np.asarray(b, np.complex128)
    T = b.shape[-1] - 1
    s = np.zeros_like(b)
    s[..., 0] = 1.0
    for k in range(1, T + 1):
        acc = np.zeros(b.shape[:-1], np.complex128)
        for j in range(1, k + 1):
            acc = acc + j * b[..., j] * s[..., k - j]
        s[..., k] = acc / k
    return s


def remove_u1_phase(V) -> np.ndarray:
    """For a unitary series V: the phase series a(g) = Im Tr log(V0^+ V(g)) (a_0 = 0) and
    W = V * exp(-i a(g) / N), so that det W = det V^(0) through order T.  The trace part of the
    algebra is the U(1) (zero) mode of the links; an SU(N) evolution keeps it zero, and
    rounding can move it."""
    V = np.asarray(V, np.complex128)
    N = V.shape[-1]
    V0h = np.zeros_like(V)
    V0h[..., 0, :, :] = np.conj(np.swapaxes(V[..., 0, :, :], -1, -2))
    D = pm.star(V0h, V)
    D[..., 0, :, :] = 0.0
    a = np.imag(np.trace(log_star_unit(D), axis1=-2, axis2=-1))     # (..., T+1), a_0 = 0
    s = scalar_exp(-1j * a / N)
    W = np.zeros_like(V)
    T = V.shape[-3] - 1
    for k in range(T + 1):
        for j in range(k + 1):
            W[..., k, :, :] += V[..., j, :, :] * s[..., k - j, None, None]
    W[..., 0, :, :] = V[..., 0, :, :]
    return W


def unitarize(U, special: bool = False) -> np.ndarray:
    """Order-by-order projection of a series onto a unitary series: the polar factor
    V = U * H^(-1/2) with H = U^+ * U (star products), for a series whose order 0 is unitary.

    Then H = 1 + D with D^(0) = U0^+ U0 - 1 = 0, and the inverse square root is the binomial
    series (1 + D)^(-1/2) = sum_{n=0}^{T} c_n D^{star n}, c_n = binom(-1/2, n), exact through
    order T because D^{star n} starts at order n.  D^(0) is set to 0 (order 0 is taken as
    unitary and is left exactly unchanged).  V^+ * V = 1 through order T, and a unitary series
    is its own projection.  With special=True the U(1) phase is removed as well
    (remove_u1_phase): det V = det U^(0) through order T.  Shape (..., T+1, N, N)."""
    U = np.asarray(U, np.complex128)
    N = U.shape[-1]
    T = U.shape[-3] - 1
    lead = U.shape[:-3]
    D = pm.star(pm.dagger(U), U)
    D[..., 0, :, :] = 0.0
    Iser = pm.identity_series(N, T, lead)
    S = np.zeros_like(U)
    P = Iser.copy()
    for n in range(T + 1):
        S = S + binom_minus_half(n) * P
        P = pm.star(P, D)
    V = pm.star(U, S)
    V[..., 0, :, :] = U[..., 0, :, :]
    return remove_u1_phase(V) if special else V
