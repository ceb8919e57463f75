"""Macroscopic moments (Sec. 3) and conservation residuals of Eq. consv, on the grid.

Integrals over velocity space are taken with the grid rule sum_n (.) dv^3, dv = 2L/N,
the rule that defines the Fourier coefficients in Sec. 4.
"""

import numpy as np


def grid_vectors(N, L):
    v = -L + (2.0 * L / N) * (np.arange(N) + 0.5)
    vx, vy, vz = np.meshgrid(v, v, v, indexing="ij")
    return vx, vy, vz


def moments(f, m, L):
    """n, u, T of one species (nondimensional definitions of Sec. 3)."""
    N = f.shape[0]
    dv3 = (2.0 * L / N) ** 3
    vx, vy, vz = grid_vectors(N, L)
    n = f.sum() * dv3
    u = np.array([(vx * f).sum(), (vy * f).sum(), (vz * f).sum()]) * dv3 / n
    c2 = (vx - u[0]) ** 2 + (vy - u[1]) ** 2 + (vz - u[2]) ** 2
    T = 2.0 * m / (3.0 * n) * (c2 * f).sum() * dv3
    return n, u, T


def knudsen_weights(masses):
    """kappa_ij = sqrt(1 + m_i/m_j): the pair-dependent part of 1/Kn_ij (Eq. Kn).

    The nondimensional prefactor of Eq. NVSS is not symmetric in (i, j); the dimensional
    kernel is (B_ij = B_ji, Sec. 2), and the right-hand side of Eq. NMBE weights Q_ij by
    1/Kn_ij, whose pair-dependent factor sqrt(1 + m_i/m_j) restores that symmetry.  The
    pairwise momentum and energy laws of Eq. consv hold for kappa_ij Q_ij.
    """
    m = np.asarray(masses, dtype=np.float64)
    return np.sqrt(1.0 + m[:, None] / m[None, :])


def conservation_residuals(Q, masses, L, kappa=None):
    """Residuals of Eq. consv for every pair (i, j), with Q_ij weighted by kappa_ij:

    mass[i, j]      = int Q_ij dv
    momentum[i, j]  = int (m_i v Q_ij + m_j v Q_ji) dv        (3-vector)
    energy[i, j]    = int (m_i |v|^2 Q_ij + m_j |v|^2 Q_ji) dv

    together with the matching scales int |Q_ij|, int m|v||Q|, int m|v|^2|Q| used to
    normalise them.
    """
    if kappa is not None:
        Q = Q * np.asarray(kappa)[:, :, None, None, None]
    s = Q.shape[0]
    N = Q.shape[-1]
    dv3 = (2.0 * L / N) ** 3
    vx, vy, vz = grid_vectors(N, L)
    v2 = vx * vx + vy * vy + vz * vz
    vn = np.sqrt(v2)
    out = {"mass": np.zeros((s, s)), "momentum": np.zeros((s, s, 3)), "energy": np.zeros((s, s)),
           "mass_scale": np.zeros((s, s)), "momentum_scale": np.zeros((s, s)),
           "energy_scale": np.zeros((s, s))}
    for i in range(s):
        for j in range(s):
            mi, mj = masses[i], masses[j]
            a, b = Q[i, j], Q[j, i]
            out["mass"][i, j] = a.sum() * dv3
            out["mass_scale"][i, j] = np.abs(a).sum() * dv3
            out["momentum"][i, j] = [((mi * a + mj * b) * c).sum() * dv3 for c in (vx, vy, vz)]
            out["momentum_scale"][i, j] = ((mi * np.abs(a) + mj * np.abs(b)) * vn).sum() * dv3
            out["energy"][i, j] = ((mi * a + mj * b) * v2).sum() * dv3
            out["energy_scale"][i, j] = ((mi * np.abs(a) + mj * np.abs(b)) * v2).sum() * dv3
    return out


def _constraint_rows(N, L, masses, i, j, w):
    """Constraint vectors of the conservation laws (Eq. consv) on the grid.

    Self pair (i, i): rows 1, v_x, v_y, v_z, |v|^2 acting on Q_ii (5 x N^3).
    Cross pair (i, j): acting on the stacked [Q_ij; Q_ji] (6 x 2N^3): mass of each half,
    m_i w_ij v + m_j w_ji v (3 rows) and m_i w_ij |v|^2 + m_j w_ji |v|^2, where w_ij are the
    pair weights under which the laws hold (w_ij = 1 / b_ij: the weighted operators share one
    symmetric kernel).
    """
    vx, vy, vz = grid_vectors(N, L)
    v2 = vx * vx + vy * vy + vz * vz
    one = np.ones_like(vx)
    if i == j:
        return np.stack([one, vx, vy, vz, v2]).reshape(5, -1)
    zero = np.zeros_like(vx)
    a, b = masses[i] * w[i, j], masses[j] * w[j, i]
    top = [one, zero, a * vx, a * vy, a * vz, a * v2]
    bot = [zero, one, b * vx, b * vy, b * vz, b * v2]
    return np.concatenate([np.stack(top).reshape(6, -1), np.stack(bot).reshape(6, -1)], axis=1)


def conservation_projection(Q, masses, L, b):
    """Minimal-L2 correction of Q that makes the discrete conservation laws exact:
    Q <- Q - C^T (C C^T)^-1 C Q for every self pair and every stacked cross pair
    (a post-processing step of the kind the paper cites for earlier spectral solvers, not
    part of its method; the fast method itself is not exactly conservative).  Q[s, s, N, N, N]; returns a corrected copy."""
    Q = np.array(Q, dtype=np.float64, copy=True)
    s, N = Q.shape[0], Q.shape[-1]
    w = 1.0 / np.asarray(b, dtype=np.float64)
    for i in range(s):
        for j in range(i, s):
            C = _constraint_rows(N, L, masses, i, j, w)
            x = Q[i, i].reshape(-1) if i == j else np.concatenate([Q[i, j].reshape(-1), Q[j, i].reshape(-1)])
            lam = np.linalg.solve(C @ C.T, C @ x)
            x = x - C.T @ lam
            if i == j:
                Q[i, i] = x.reshape(N, N, N)
            else:
                Q[i, j] = x[:N ** 3].reshape(N, N, N)
                Q[j, i] = x[N ** 3:].reshape(N, N, N)
    return Q


def species_sum(Q, kappa=None):
    """sum_j kappa_ij Q_ij for every species i (the right-hand side of Eq. NMBE with
    kappa_ij = 1 / Kn_ij).  Q[s, s, ...] -> [s, ...]."""
    s = Q.shape[0]
    kappa = np.ones((s, s)) if kappa is None else np.asarray(kappa, dtype=np.float64)
    return np.einsum("ij,ij...->i...", kappa, Q)
