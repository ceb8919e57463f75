"""Collision kernel, computational domain and precomputed weights (Secs. 3-4).

Every function works in the nondimensional variables of Sec. 3.
"""

import numpy as np
from scipy.special import gamma, j0, roots_jacobi


def b_vss(mi, mj, omega, alpha):
    """Nondimensional VSS prefactor of B_ij (Eq. NVSS):

        alpha / ( sqrt(1 + m_i/m_j) * mu_ij^(omega-0.5) * 2^(1+alpha) * Gamma(2.5-omega) * pi )

    with the reduced mass mu_ij = m_i m_j / (m_i + m_j).  Then
    B_ij = b * |g|^(2(1-omega)) * (1 + cos chi)^(alpha-1).
    """
    mu = mi * mj / (mi + mj)
    return alpha / (np.sqrt(1.0 + mi / mj) * mu ** (omega - 0.5) * 2.0 ** (1.0 + alpha)
                    * gamma(2.5 - omega) * np.pi)


def mass_fractions(mi, mj):
    """(c_i, c_j) = (m_i, m_j) / (m_i + m_j), the factors of g in v' and v_*' (Sec. 4)."""
    return mi / (mi + mj), mj / (mi + mj)


def pair_support_radius(L, mi, mj):
    """Largest support radius S_ij the anti-aliasing condition (Eq. domain) allows for the
    ordered pair (i, j):

        2L >= ( max(4 m_j/(m_i+m_j), 2) + sqrt(1 + m_j/m_i) ) S + S
    """
    _, cj = mass_fractions(mi, mj)
    return 2.0 * L / (max(4.0 * cj, 2.0) + np.sqrt(1.0 + mj / mi) + 1.0)


def support_radius(L, masses):
    """The velocity grid is shared by all species, so S is the minimum of S_ij over all
    ordered pairs (i, j).  The radial truncation is then R = 2S (Sec. 4, item 2)."""
    return min(pair_support_radius(L, mi, mj) for mi in masses for mj in masses)


def sinc(x):
    """sin(x)/x with sinc(0) = 1."""
    return np.sinc(np.asarray(x) / np.pi)


def phi_integral(a, cos_t, alpha, n_t):
    """int_{-1}^{1} (1+t)^(alpha-1) exp(-i a t cos theta) J0(a sqrt(1-t^2) sin theta) dt by the
    n_t-point Gauss-Jacobi rule for the weight (1+t)^(alpha-1)."""
    sin_t = np.sqrt(np.maximum(0.0, 1.0 - cos_t * cos_t))
    t, wt = roots_jacobi(n_t, 0.0, alpha - 1.0)
    acc = np.zeros(np.broadcast(a, cos_t).shape, dtype=np.complex128)
    for tq, wq in zip(t, wt):
        acc += wq * np.exp(-1j * a * tq * cos_t) * j0(a * np.sqrt(1.0 - tq * tq) * sin_t)
    return acc


def jacobi_rule_size(a_max, alpha, tol=1e-13):
    """Size of the t rule that computes F "to high accuracy" (Sec. 4, the precomputation of
    F after Eq. GG), read as a converged integral: starting from 32 points the rule is
    doubled until, at the largest argument a_max (the integrand's highest frequency) and at
    a spread of angles, the change is below tol times the integral's bound
    int (1+t)^(alpha-1) dt = 2^alpha / alpha; the finer rule of the last pair is kept.
    Lower arguments converge sooner, since the integrand's bandwidth grows with a."""
    bound = 2.0 ** alpha / alpha
    cos_t = np.linspace(-1.0, 1.0, 9)
    a = np.array([a_max, 0.5 * a_max])[:, None]
    n = 32
    prev = phi_integral(a, cos_t, alpha, n)
    while True:
        cur = phi_integral(a, cos_t, alpha, 2 * n)
        if np.max(np.abs(cur - prev)) < tol * bound or n >= 4096:
            return 2 * n
        n, prev = 2 * n, cur


def gain_weight(kx, ky, kz, rho, sigma, cj, b, omega, alpha, L, n_t=None):
    """F^{(ij)}(k, rho, sigma) of Eq. GG:

        F = rho^2 * int_{S^2} B_ij(rho, sigma . g_hat) exp(-i pi rho c_j k . g_hat / L) dg_hat

    VHS (alpha = 1): B does not depend on the angle and the sphere integral of the
    plane wave is 4 pi sinc(a), a = pi rho c_j |k| / L, so F = 4 pi b rho^(4-2 omega) sinc(a)
    (real and sigma-independent).

    VSS (alpha > 1): writing g_hat = t sigma + sqrt(1-t^2)(cos phi e1 + sin phi e2), the phi
    integral of the plane wave is 2 pi J0(a sqrt(1-t^2) sin theta) exp(-i a t cos theta),
    cos theta = k_hat . sigma, so

        F = 2 pi b rho^(4-2 omega) int_{-1}^{1} (1+t)^(alpha-1) exp(-i a t cos theta)
                                             J0(a sqrt(1-t^2) sin theta) dt,

    evaluated with a Gauss-Jacobi rule for the weight (1+t)^(alpha-1): n_t points if given,
    else the converged size of jacobi_rule_size at the largest a of the call.
    """
    kn = np.sqrt(kx * kx + ky * ky + kz * kz)
    a = np.pi * rho * cj * kn / L
    pref = b * rho ** (4.0 - 2.0 * omega)
    if alpha == 1.0:
        return (4.0 * np.pi * pref * sinc(a)).astype(np.complex128)
    with np.errstate(invalid="ignore", divide="ignore"):
        cos_t = np.where(kn > 0, (kx * sigma[0] + ky * sigma[1] + kz * sigma[2]) / kn, 1.0)
    if n_t is None:
        n_t = jacobi_rule_size(float(np.max(a)), alpha)
    return 2.0 * np.pi * pref * phi_integral(a, cos_t, alpha, n_t)


def loss_weight(kx, ky, kz, rho_nodes, rho_weights, b, omega, alpha, L):
    """G^{(ij)-}(m) (the loss weight defined after Eq. GG):

        G^- = int_0^R int_{S^2} int_{S^2} rho^2 B_ij e^{-i pi rho m . g_hat / L} dsigma dg_hat drho.

    The sigma integral of (1 + sigma.g_hat)^(alpha-1) is 2 pi 2^alpha / alpha for every g_hat;
    the g_hat integral of the plane wave is 4 pi sinc(pi rho |m| / L).  The remaining radial
    integral is taken with the same Gauss-Legendre rule as the gain term.
    """
    kn = np.sqrt(kx * kx + ky * ky + kz * kz)
    ang = 2.0 * np.pi * 2.0 ** alpha / alpha * 4.0 * np.pi
    G = np.zeros(np.shape(kn))
    for rho, w in zip(rho_nodes, rho_weights):
        G += w * rho ** (4.0 - 2.0 * omega) * sinc(np.pi * rho * kn / L)
    return ang * b * G
