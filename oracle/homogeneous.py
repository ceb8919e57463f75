"""Spatially homogeneous time stepping (Secs. 5 and 6.1), test infrastructure.

d_t f_i = sum_j kappa_ij Q_ij(f_i, f_j) advanced by the second-order strong-stability-preserving
Runge-Kutta scheme the paper integrates in time with:
    f1 = f + dt R(f),   f_new = f / 2 + (f1 + dt R(f1)) / 2.
"""

from . import fast_spectral, moments


def ssp_rk2_step(f, dt, rhs):
    """One step for a right-hand side callable rhs(f) -> array like f."""
    f1 = f + dt * rhs(f)
    return 0.5 * f + 0.5 * (f1 + dt * rhs(f1))


def collision_rhs(prob, kappa=None):
    """R(f)_i = sum_j kappa_ij Q_ij(f_i, f_j) with the oracle's fast method."""
    return lambda f: moments.species_sum(fast_spectral.collision(f, prob)[0], kappa)
