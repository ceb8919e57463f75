"""The fast build of the FP32 VSS gain table interpolates Phi_alpha(p, q), the two-argument
function that carries all of F's dependence on (k, rho, sigma) (Sec. 4, F after Eq. GG:
F = pref(rho) Phi(s k.sigma, s |k x sigma|), s = pi rho c_j / L), from a grid of spacing 0.03
with 4 x 4-point Lagrange interpolation.  This pins that choice on the CPU: the same
interpolation of the oracle's converged integral reproduces the oracle's F to 1e-8 of the
integral's bound at arguments up to the N = 48 workload's largest (a ~ 65)."""

import numpy as np
import pytest

from oracle import kernel

H = 0.03  # the plan's grid spacing


def _phi(p, q, alpha, n_t):
    """Phi_alpha(p, q) from the oracle's sphere integral: a = |(p, q)|, cos theta = p / a."""
    a = np.hypot(p, q)
    c = np.where(a > 0, p / np.where(a > 0, a, 1.0), 1.0)
    return kernel.phi_integral(a, c, alpha, n_t)


def _lagrange4(f):
    return np.array([-f * (f - 1) * (f - 2) / 6, (f + 1) * (f - 1) * (f - 2) / 2,
                     -(f + 1) * f * (f - 2) / 2, (f + 1) * f * (f - 1) / 6])


@pytest.mark.parametrize("alpha", [1.4, 2.0])
def test_grid_interpolation_of_phi_matches_the_oracle(alpha):
    A = 65.3
    n_t = kernel.jacobi_rule_size(A, alpha)
    rng = np.random.default_rng(17)
    pts = np.stack([rng.uniform(-A, A, 60), rng.uniform(0.0, A, 60)], axis=1)
    pts[0] = (A, 0.0)      # along sigma at the largest argument
    pts[1] = (0.0, A)      # perpendicular
    p0, q0 = -A - 2 * H, -2 * H
    worst = 0.0
    for p, q in pts:
        u, v = (p - p0) / H, (q - q0) / H
        iu, iv = int(np.floor(u)), int(np.floor(v))
        P = p0 + (iu + np.arange(-1, 3)) * H
        Q = q0 + (iv + np.arange(-1, 3)) * H
        PP, QQ = np.meshgrid(P, Q, indexing="ij")
        grid = _phi(PP.ravel(), QQ.ravel(), alpha, n_t).reshape(4, 4)
        val = _lagrange4(u - iu) @ grid @ _lagrange4(v - iv)
        worst = max(worst, abs(val - _phi(np.array([p]), np.array([q]), alpha, n_t)[0]))
    assert worst < 1e-8 * 2.0 ** alpha / alpha


def test_phi_is_even_in_q_and_conjugate_in_p():
    """The grid's mirrored rows below q = 0 and the antipodal slot sharing rest on
    Phi(p, -q) = Phi(p, q) and Phi(-p, q) = conj Phi(p, q)."""
    p = np.array([3.7, -12.0, 40.0])
    q = np.array([5.1, 0.4, 22.0])
    n_t = kernel.jacobi_rule_size(60.0, 1.4)
    a = np.hypot(p, q)
    assert np.allclose(kernel.phi_integral(a, p / a, 1.4, n_t), np.conj(kernel.phi_integral(a, -p / a, 1.4, n_t)),
                       atol=1e-14)
    # J0 is even: the integrand depends on q only through J0(sqrt(1 - t^2) q)
    t, w = np.polynomial.legendre.leggauss(40)
    from scipy.special import j0
    assert np.allclose(j0(np.sqrt(1 - t * t)[:, None] * q), j0(-np.sqrt(1 - t * t)[:, None] * q))
