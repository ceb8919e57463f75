"""The O(N^6) direct spectral method (Eq. sum), used only to pin ``fast_spectral``.

    Q_hat_k = sum_{l+m = k} G(l, m) f_hat^(i)_l f_hat^(j)_m,   G = G^+ - G^-,

with the discrete gain weight (the quadrature form of Eq. GG)

    G^+(l, m) = sum_{rho, sigma} w_rho w_sigma F(l+m, rho, sigma)
                    exp(i pi rho (c_j l - c_i m) . sigma / L).

Nothing here is shared with ``fast_spectral``: the grid transforms are written out from
the definition, the sum runs over all (l, m) pairs explicitly, and F and G^- are not taken
from their closed forms but integrated over the sphere by brute force from their
definitions (product rule in (t, phi) around sigma for F, around g_hat for the sigma
integral of G^-).  With enough sphere points the two methods agree to rounding, which pins
the fast method's phases, index conventions, normalisations and both weights.

The sum l + m is periodic (mod N) and F is evaluated at the wrapped mode, the reading the
fast method's FFT convolution implies (the paper writes l + m = k without saying how the
truncated sum treats the modes outside the grid).  A wrapped term l + m = k + pN
carries the grid's aliasing factor N^-1 sum_n exp(i pi p N v_n / L) per axis, which is
what the coefficient of a product of grid values contains.
"""

import numpy as np
from scipy.special import roots_jacobi


def _grid_and_modes(N, L):
    v = -L + (2.0 * L / N) * (np.arange(N) + 0.5)
    k = np.arange(N) - N // 2
    return v, k


def coefficients(f, L):
    """f_hat_k = N^-3 sum_n f(v_n) exp(-i pi k.v_n / L), explicit triple sum per axis."""
    N = f.shape[0]
    v, k = _grid_and_modes(N, L)
    phase = np.exp(-1j * np.pi * k[:, None] * v[None, :] / L) / N
    return np.einsum("ax,by,cz,xyz->abc", phase, phase, phase, f.astype(np.complex128))


def series(fh, L):
    """sum_k f_hat_k exp(i pi k.v_n / L) at the grid."""
    N = fh.shape[0]
    v, k = _grid_and_modes(N, L)
    phase = np.exp(1j * np.pi * v[:, None] * k[None, :] / L)
    return np.einsum("xa,yb,zc,abc->xyz", phase, phase, phase, fh)


def _frame(axis):
    """Two unit vectors completing ``axis`` to an orthonormal frame."""
    axis = axis / np.linalg.norm(axis)
    helper = np.array([1.0, 0.0, 0.0]) if abs(axis[0]) < 0.9 else np.array([0.0, 1.0, 0.0])
    e1 = np.cross(axis, helper)
    e1 /= np.linalg.norm(e1)
    e2 = np.cross(axis, e1)
    return e1, e2


def sphere_rule_around(axis, alpha, n_t, n_phi):
    """Points g_hat and weights for int_{S^2} (1 + axis.g_hat)^(alpha-1) h(g_hat) dg_hat:
    Gauss-Jacobi in t = axis.g_hat (weight (1+t)^(alpha-1)) times the trapezoid rule in phi."""
    t, wt = roots_jacobi(n_t, 0.0, alpha - 1.0)
    phi = 2.0 * np.pi * np.arange(n_phi) / n_phi
    e1, e2 = _frame(np.asarray(axis, dtype=np.float64))
    axis = np.asarray(axis, dtype=np.float64) / np.linalg.norm(axis)
    st = np.sqrt(1.0 - t * t)
    pts = (t[:, None, None] * axis[None, None, :]
           + st[:, None, None] * (np.cos(phi)[None, :, None] * e1[None, None, :]
                                  + np.sin(phi)[None, :, None] * e2[None, None, :]))
    w = (wt[:, None] * np.full(n_phi, 2.0 * np.pi / n_phi)[None, :])
    return pts.reshape(-1, 3), w.reshape(-1)


def gain_weight_by_quadrature(kvec, rho, sigma, cj, b, omega, alpha, L, n_t, n_phi):
    """F(k, rho, sigma) = rho^2 int B(rho, sigma.g_hat) exp(-i pi rho c_j k.g_hat/L) dg_hat,
    integrated point by point over the sphere.  kvec: [K, 3]."""
    pts, w = sphere_rule_around(sigma, alpha, n_t, n_phi)
    phase = np.exp(-1j * np.pi * rho * cj * (kvec @ pts.T) / L)
    return rho ** 2 * b * rho ** (2.0 - 2.0 * omega) * (phase @ w)


def loss_weight_by_quadrature(kvec, rho_nodes, rho_weights, b, omega, alpha, L, n_t, n_phi):
    """G^-(m) = int_0^R rho^2 int int B exp(-i pi rho m.g_hat/L) dsigma dg_hat drho, with both
    sphere integrals by product rules (the sigma rule is taken around each g_hat)."""
    g_pts, g_w = sphere_rule_around(np.array([0.0, 0.0, 1.0]), 1.0, n_t, n_phi)
    _, s_w = sphere_rule_around(np.array([0.0, 0.0, 1.0]), alpha, n_t, n_phi)
    sigma_integral = s_w.sum()
    out = np.zeros(len(kvec), dtype=np.complex128)
    for rho, wr in zip(rho_nodes, rho_weights):
        plane = np.exp(-1j * np.pi * rho * (kvec @ g_pts.T) / L) @ g_w
        out += wr * rho ** 2 * b * rho ** (2.0 - 2.0 * omega) * sigma_integral * plane
    return out


def collision_pair_direct(f_i, f_j, prob, i, j, n_t=40, n_phi=64, truncation="periodic"):
    """Q^(ij) on the grid from the direct sum (Eq. sum); returns complex grid values.

    truncation="periodic": l + m taken modulo N (what the fast method evaluates);
    truncation="literal": only pairs with l + m inside the grid's mode range contribute and
    no term wraps -- the truncated sum read literally.  The difference of the two is the
    aliasing diagnostic of the periodic reading."""
    if truncation not in ("periodic", "literal"):
        raise ValueError(truncation)
    N, L = prob.N, prob.L
    mi, mj = prob.masses[i], prob.masses[j]
    ci, cj = mi / (mi + mj), mj / (mi + mj)
    _, kk = _grid_and_modes(N, L)
    K = np.stack(np.meshgrid(kk, kk, kk, indexing="ij"), axis=-1).reshape(-1, 3).astype(float)
    n_modes = len(K)
    idx = np.stack(np.meshgrid(np.arange(N), np.arange(N), np.arange(N), indexing="ij"),
                   axis=-1).reshape(-1, 3)
    # wrapped index of l + m: (a_l + a_m - N/2) mod N per axis, flattened
    wrap3 = (idx[:, None, :] + idx[None, :, :] - N // 2) % N
    wrap = (wrap3[..., 0] * N + wrap3[..., 1]) * N + wrap3[..., 2]
    # l + m = k + p N with k the wrapped mode; the grid coefficient of exp(i pi (l+m).v/L)
    # at mode k is then N^-1 sum_n exp(i pi p N v_n / L) per axis (+-1 on this grid)
    v, _ = _grid_and_modes(N, L)
    p3 = ((idx[:, None, :] + idx[None, :, :] - N) - (wrap3 - N // 2)) // N
    alias_1d = {p: np.mean(np.exp(1j * np.pi * p * N * v / L)) for p in (-1, 0, 1)}
    alias = np.ones(wrap.shape, dtype=np.complex128)
    for d in range(3):
        for p in (-1, 1):
            alias = np.where(p3[..., d] == p, alias * alias_1d[p], alias)

    fh_i = coefficients(f_i, L).reshape(-1)
    fh_j = coefficients(f_j, L).reshape(-1)

    # the pair's radial rule: the common one, or (per-pair truncation) a Gauss-Legendre rule of
    # the same size on [0, pair_R[i, j]]
    if prob.pair_R is None:
        R_ij, rho_q, w_q = prob.R, prob.rho, prob.w_rho
    else:
        R_ij = float(prob.pair_R[i, j])
        x, w = np.polynomial.legendre.leggauss(len(prob.rho))
        rho_q, w_q = 0.5 * R_ij * (x + 1.0), 0.5 * R_ij * w
    G = np.zeros((n_modes, n_modes), dtype=np.complex128)
    for rho, w_rho in zip(rho_q, w_q):
        for sig, w_sig in zip(prob.sigma, prob.w_sigma):
            F = gain_weight_by_quadrature(K, rho, sig, cj, prob.b[i, j], prob.omega[i, j],
                                          prob.alpha[i, j], L, n_t, n_phi)
            ks = K @ sig
            el = np.exp(1j * np.pi * rho * cj * ks / L)
            em = np.exp(-1j * np.pi * rho * ci * ks / L)
            G += w_rho * w_sig * F[wrap] * el[:, None] * em[None, :]
    if prob.loss_rule == "accurate":
        # 4 N_rho Gauss-Legendre nodes on [0, R] for the loss weight's radial integral
        x, w = np.polynomial.legendre.leggauss(4 * len(prob.rho))
        loss_rho, loss_w = 0.5 * R_ij * (x + 1.0), 0.5 * R_ij * w
    else:
        loss_rho, loss_w = rho_q, w_q
    Gm = loss_weight_by_quadrature(K, loss_rho, loss_w, prob.b[i, j], prob.omega[i, j],
                                   prob.alpha[i, j], L, n_t, n_phi)
    G -= Gm[None, :]
    terms = alias * G * fh_i[:, None] * fh_j[None, :]
    if truncation == "literal":
        terms = np.where(np.all(p3 == 0, axis=-1), G * fh_i[:, None] * fh_j[None, :], 0.0)
    Qh = (np.bincount(wrap.reshape(-1), weights=terms.real.reshape(-1), minlength=n_modes)
          + 1j * np.bincount(wrap.reshape(-1), weights=terms.imag.reshape(-1),
                             minlength=n_modes))
    return series(Qh.reshape(N, N, N), L)


def collision_direct(f, prob, **kw):
    """All s^2 operators by the direct method: f[s, N, N, N] -> Q[s, s, N, N, N] (real part).
    Keyword arguments go to collision_pair_direct (e.g. truncation="literal")."""
    s = f.shape[0]
    N = prob.N
    Q = np.zeros((s, s, N, N, N))
    for i in range(s):
        for j in range(s):
            Q[i, j] = collision_pair_direct(f[i], f[j], prob, i, j, **kw).real
    return Q
