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
