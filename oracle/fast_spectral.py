"""The fast Fourier spectral collision operator of Sec. 4, evaluated literally in FP64.

For every ordered species pair (i, j) this module follows the paper's steps in order:

1. truncated Fourier series of f^(i), f^(j) on D_L = [-L, L]^3 with modes
   k in [-N/2, N/2-1]^3 (the coefficient integral taken with the grid rule);
2. for every radial Gauss-Legendre node rho and every design direction sigma, the two
   phase-modulated spectra exp(+i pi rho c_j l.sigma/L) f^(i)_l and
   exp(-i pi rho c_i m.sigma/L) f^(j)_m are taken back to the grid, multiplied
   pointwise, transformed forward (the convolution over l+m=k), weighted by
   w_rho w_sigma F(k, rho, sigma) and summed into the gain spectrum (the fast gain
   formula following Eq. GG);
3. the loss spectrum is the convolution of f^(i)_l with G^-(m) f^(j)_m, done the same way;
4. Q^(ij) on the grid is the real part of the inverse series of (gain - loss).

Transforms are the plain definition: dense DFT matrices applied along each axis
(a matrix product per axis; no FFT).  There is no reuse of (i,j)/(j,i) products, no
antipodal pairing of sigma and no summation over sigma before the forward transform.

Readings of points the paper leaves open:

* grid: cell-centred nodes v_n = -L + (n + 1/2) 2L/N, n = 0..N-1 (with this grid the
  Krook-Wu errors of Table 1 are reproduced; Q at the nodes does not depend on the
  offset once the samples are fixed, only the sample points do);
* convolutions are periodic (mod N): products of grid values, as the FFT evaluates;
  the gain weight F is evaluated at the wrapped mode k;
* the radial truncation R = 2S with S from Eq. domain taken over all ordered pairs
  (optionally per pair: Problem.pair_R);
* G^- uses the same Gauss-Legendre radial rule as the gain term (optionally a 4 N_rho-point
  rule of its own: Problem.loss_rule).
"""

from dataclasses import dataclass, field

import numpy as np

from . import kernel, quadrature


@dataclass
class Problem:
    """Discretisation of the multi-species operator (Sec. 4)."""
    N: int
    L: float
    masses: np.ndarray            # [s] nondimensional masses
    omega: np.ndarray             # [s, s]
    alpha: np.ndarray             # [s, s]
    b: np.ndarray                 # [s, s] kernel prefactors b_ij
    sigma: np.ndarray             # [M, 3] design directions
    w_sigma: np.ndarray           # [M]
    rho: np.ndarray               # [N_rho] radial nodes on [0, R]
    w_rho: np.ndarray             # [N_rho]
    R: float
    extra: dict = field(default_factory=dict)
    # radial rule of the loss weight G^-: "same" (the gain's N_rho nodes) or "accurate"
    # (4 N_rho Gauss-Legendre nodes on [0, R]); the paper asks for G^- "to high accuracy"
    # without naming a rule
    loss_rule: str = "same"
    # optional per-pair truncation: pair_R[i, j] = 2 S_ij (Eq. domain for that pair alone) with
    # its own N_rho-point rule; None = the common R of all pairs (the default reading)
    pair_R: np.ndarray = None

    @property
    def s(self):
        return len(self.masses)


def make_problem(N, L, masses, omega, alpha=1.0, M=6, N_rho=None, R=None,
                 b_override=None, sigma=None, w_sigma=None, loss_rule="same", pair_radius=False):
    """Build the discretisation.  ``omega``/``alpha`` may be scalars or [s, s] arrays."""
    masses = np.asarray(masses, dtype=np.float64)
    s = len(masses)
    omega = np.broadcast_to(np.asarray(omega, dtype=np.float64), (s, s)).copy()
    alpha = np.broadcast_to(np.asarray(alpha, dtype=np.float64), (s, s)).copy()
    if b_override is not None:
        b = np.asarray(b_override, dtype=np.float64).reshape(s, s).copy()
    else:
        b = np.array([[kernel.b_vss(masses[i], masses[j], omega[i, j], alpha[i, j])
                       for j in range(s)] for i in range(s)])
    if sigma is None:
        sigma, w_sigma = quadrature.spherical_design(M)
    sigma = np.asarray(sigma, dtype=np.float64).reshape(-1, 3)
    w_sigma = np.asarray(w_sigma, dtype=np.float64)
    if R is None or R <= 0:
        R = 2.0 * kernel.support_radius(L, masses)
    if N_rho is None:
        N_rho = N
    rho, w_rho = quadrature.gauss_legendre_radial(N_rho, R)
    if loss_rule not in ("same", "accurate"):
        raise ValueError(loss_rule)
    pair_R = None
    if pair_radius:
        pair_R = np.array([[2.0 * kernel.pair_support_radius(L, masses[i], masses[j])
                            for j in range(s)] for i in range(s)])
    return Problem(N=N, L=float(L), masses=masses, omega=omega, alpha=alpha, b=b,
                   sigma=sigma, w_sigma=w_sigma, rho=rho, w_rho=w_rho, R=float(R),
                   loss_rule=loss_rule, pair_R=pair_R)


def radial_rule(prob, i, j):
    """(rho nodes, weights, R) of the pair (i, j): the common rule, or with per-pair
    truncation a Gauss-Legendre rule of the same size on [0, pair_R[i, j]]."""
    if prob.pair_R is None:
        return prob.rho, prob.w_rho, prob.R
    R = float(prob.pair_R[i, j])
    rho, w = quadrature.gauss_legendre_radial(len(prob.rho), R)
    return rho, w, R


def velocity_grid(N, L):
    """Cell-centred nodes v_n = -L + (n + 1/2) 2L/N, n = 0..N-1, along one axis."""
    return -L + (2.0 * L / N) * (np.arange(N) + 0.5)


def modes(N):
    """Fourier modes k = -N/2 .. N/2-1 along one axis (array index a = k + N/2)."""
    return np.arange(N) - N // 2


def mode_grid(N):
    k = modes(N).astype(np.float64)
    return np.meshgrid(k, k, k, indexing="ij")


def _apply_along(mat, x, axis):
    return np.moveaxis(np.tensordot(mat, x, axes=([1], [axis])), 0, axis)


def forward_matrix(N, L):
    """E[a, n] = N^-1 exp(-i pi k_a v_n / L): the coefficient integral with the grid rule."""
    v = velocity_grid(N, L)
    k = modes(N)
    return np.exp(-1j * np.pi * np.outer(k, v) / L) / N


def inverse_matrix(N, L):
    """E[n, a] = exp(+i pi k_a v_n / L): the truncated Fourier series at the grid."""
    v = velocity_grid(N, L)
    k = modes(N)
    return np.exp(1j * np.pi * np.outer(v, k) / L)


def dft3(f, L):
    """Fourier coefficients f_hat_k = (2L)^-3 int f e^{-i pi k.v/L} dv on the grid (Sec. 4)."""
    E = forward_matrix(f.shape[0], L)
    out = f.astype(np.complex128)
    for ax in range(3):
        out = _apply_along(E, out, ax)
    return out


def idft3(fh, L):
    """Truncated Fourier series sum_k f_hat_k e^{i pi k.v/L} at the grid (Sec. 4)."""
    E = inverse_matrix(fh.shape[0], L)
    out = fh.astype(np.complex128)
    for ax in range(3):
        out = _apply_along(E, out, ax)
    return out


def gain_table(prob, i, j, q, m):
    """F^{(ij)}(k, rho_q, sigma_m) on the mode grid (Eq. GG)."""
    kx, ky, kz = mode_grid(prob.N)
    _, cj = kernel.mass_fractions(prob.masses[i], prob.masses[j])
    return kernel.gain_weight(kx, ky, kz, radial_rule(prob, i, j)[0][q], prob.sigma[m], cj, prob.b[i, j],
                              prob.omega[i, j], prob.alpha[i, j], prob.L)


def loss_rule_nodes(prob, i=0, j=0):
    """Radial nodes and weights of the loss weight's rho integral for the pair (i, j) (see
    Problem.loss_rule and Problem.pair_R)."""
    rho, w_rho, R = radial_rule(prob, i, j)
    if prob.loss_rule == "accurate":
        return quadrature.gauss_legendre_radial(4 * len(prob.rho), R)
    return rho, w_rho


def loss_table(prob, i, j):
    """G^{(ij)-}(m) on the mode grid."""
    kx, ky, kz = mode_grid(prob.N)
    rho, w_rho = loss_rule_nodes(prob, i, j)
    return kernel.loss_weight(kx, ky, kz, rho, w_rho, prob.b[i, j],
                              prob.omega[i, j], prob.alpha[i, j], prob.L)


def collision_pair(f_i, f_j, prob, i, j):
    """Q^(ij)(f^(i), f^(j)) on the grid by the fast method of Sec. 4 (literal loop order).

    Returns the complex grid values of (gain - loss); Q^(ij) is their real part.
    """
    L = prob.L
    ci, cj = kernel.mass_fractions(prob.masses[i], prob.masses[j])
    fh_i = dft3(f_i, L)
    fh_j = dft3(f_j, L)
    kx, ky, kz = mode_grid(prob.N)
    gain_hat = np.zeros(fh_i.shape, dtype=np.complex128)
    rho_q, w_q, _ = radial_rule(prob, i, j)
    for q, (rho, w_rho) in enumerate(zip(rho_q, w_q)):
        for m, (sig, w_sig) in enumerate(zip(prob.sigma, prob.w_sigma)):
            k_dot_sigma = kx * sig[0] + ky * sig[1] + kz * sig[2]
            a = idft3(np.exp(1j * np.pi * rho * cj * k_dot_sigma / L) * fh_i, L)
            bb = idft3(np.exp(-1j * np.pi * rho * ci * k_dot_sigma / L) * fh_j, L)
            F = gain_table(prob, i, j, q, m)
            gain_hat += w_rho * w_sig * F * dft3(a * bb, L)
    G_minus = loss_table(prob, i, j)
    loss = idft3(fh_i, L) * idft3(G_minus * fh_j, L)
    return idft3(gain_hat, L) - loss


def collision(f, prob):
    """All s^2 operators: f[s, N, N, N] (real) -> (Q[s, s, N, N, N], max |Im|).

    Q[i, j] = Re Q^(ij)(f^(i), f^(j)).  The second value is the largest imaginary part
    met, a diagnostic of the Nyquist modes (the method's result is the real part).
    """
    f = np.asarray(f, dtype=np.float64)
    s = f.shape[0]
    N = prob.N
    Q = np.zeros((s, s, N, N, N))
    max_imag = 0.0
    for i in range(s):
        for j in range(s):
            qc = collision_pair(f[i], f[j], prob, i, j)
            Q[i, j] = qc.real
            max_imag = max(max_imag, float(np.abs(qc.imag).max()))
    return Q, max_imag


def collision_batch(f_batch, prob):
    """f[B, s, N, N, N] -> Q[B, s, s, N, N, N], one node after the other."""
    return np.stack([collision(f, prob)[0] for f in f_batch])
