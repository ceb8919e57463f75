"""One-dimensional nodal discontinuous Galerkin discretisation of the transport term (Sec. 5),
Maxwell wall boundary condition (Sec. 2) and the RKDG step of the full equation (Eq. NMBE).

Test infrastructure: see the package docstring.  Every matrix below is built from its
integral definition with an explicit quadrature; nothing uses the simplifications the
CUDA path makes (diagonal mass matrix, S = w D), so the two are independent.

Layout of a DG state: F[e, m, i, x, y, z] -- element e (left to right), GLL node m of the
element, species i, then the velocity grid.
"""

import numpy as np

from . import fast_spectral, moments


# ----------------------------------------------------------------------- GLL rule and basis

def gll(K):
    """Gauss-Lobatto-Legendre nodes and weights on [-1, 1] (K >= 2 points): the endpoints and
    the roots of P'_{K-1}; w = 2 / (K (K-1) P_{K-1}(xi)^2)."""
    if K < 2:
        raise ValueError("K >= 2")
    P = np.polynomial.legendre.Legendre.basis(K - 1)
    inner = np.sort(np.real(P.deriv().roots())) if K > 2 else np.zeros(0)
    xi = np.concatenate(([-1.0], inner, [1.0]))
    w = 2.0 / (K * (K - 1) * P(xi) ** 2)
    return xi, w


def lagrange(xi_nodes, m, x):
    """phi_m(x) = prod_{n != m} (x - xi_n) / (xi_m - xi_n)."""
    v = np.ones_like(np.asarray(x, dtype=np.float64))
    for n, xn in enumerate(xi_nodes):
        if n != m:
            v = v * (x - xn) / (xi_nodes[m] - xn)
    return v


def lagrange_deriv(xi_nodes, m, x):
    """phi_m'(x) by the product rule."""
    x = np.asarray(x, dtype=np.float64)
    K = len(xi_nodes)
    out = np.zeros_like(x)
    for k in range(K):
        if k == m:
            continue
        term = np.full_like(x, 1.0 / (xi_nodes[m] - xi_nodes[k]))
        for n in range(K):
            if n != m and n != k:
                term = term * (x - xi_nodes[n]) / (xi_nodes[m] - xi_nodes[n])
        out = out + term
    return out


def element_matrices(K, h):
    """Mass M_ml = int phi_m phi_l dx and stiffness S_ml = int phi_l d/dx phi_m dx on an element
    of width h.  The mass matrix is taken with the K-point GLL rule on the nodes themselves, the
    spectral-element choice of Sec. 5 (it comes out diagonal); the stiffness integrand has degree
    2K-3 and is integrated exactly with a (K+2)-point Gauss-Legendre rule."""
    xi, w = gll(K)
    phi_n = np.array([lagrange(xi, m, xi) for m in range(K)])        # [K, K]
    Mm = (h / 2.0) * np.einsum("mq,lq,q->ml", phi_n, phi_n, w)
    q, wq = np.polynomial.legendre.leggauss(K + 2)
    phi = np.array([lagrange(xi, m, q) for m in range(K)])           # [K, nq]
    dphi = np.array([lagrange_deriv(xi, m, q) for m in range(K)])     # d/dxi
    S = np.einsum("lq,mq,q->ml", phi, dphi, wq)                       # (h/2)(2/h) cancel
    return Mm, S


def collision_tensor(K, h):
    """H_{m l1 l2} = int phi_m phi_l1 phi_l2 dx taken with the K-point GLL rule (the
    spectral-element choice of Sec. 5): diagonal, H_mmm = (h/2) w_m."""
    xi, w = gll(K)
    phi = np.array([lagrange(xi, m, xi) for m in range(K)])          # [K, K] = identity
    return (h / 2.0) * np.einsum("aq,bq,cq,q->abc", phi, phi, phi, w)


# ----------------------------------------------------------------------------- the problem

class DG1D:
    """Ne uniform elements on [x0, x1], K GLL nodes each, velocity grid of ``prob``.

    bc = "periodic", or "walls": boundary sides at x0 (outward normal -x) and x1 (+x).  Side k
    is a Maxwell wall (side_kind[k] = "wall") with temperature Tw[k], velocity uw[k] (3-vector;
    its x component must be 0) and accommodation acc[k] (1 = diffuse, 0 = specular), or an
    in-flow equilibrium boundary (side_kind[k] = "inflow", Sec. 2) whose entering particles
    follow the Maxwellian of densities n_in[k][i], temperature Tw[k] and velocity uw[k]."""

    def __init__(self, prob, Ne, K, x0=0.0, x1=1.0, bc="periodic", Tw=(1.0, 1.0),
                 uw=((0.0, 0.0, 0.0), (0.0, 0.0, 0.0)), acc=(1.0, 1.0),
                 side_kind=("wall", "wall"), n_in=None):
        self.side_kind = tuple(side_kind)
        self.n_in = None if n_in is None else np.asarray(n_in, dtype=np.float64)
        self.prob, self.Ne, self.K = prob, Ne, K
        self.x0, self.x1 = float(x0), float(x1)
        self.h = (self.x1 - self.x0) / Ne
        self.bc = bc
        self.Tw = tuple(float(t) for t in Tw)
        self.uw = tuple(np.asarray(u, dtype=np.float64) for u in uw)
        self.acc = tuple(float(a) for a in acc)
        self.xi, self.w = gll(K)
        self.M, self.S = element_matrices(K, self.h)
        self.Minv = np.linalg.inv(self.M)
        N, L = prob.N, prob.L
        v = fast_spectral.velocity_grid(N, L)
        self.vx = v[:, None, None] * np.ones((N, N, N))
        self.V = np.stack(np.meshgrid(v, v, v, indexing="ij"))      # [3, N, N, N]
        self.dv3 = (2.0 * L / N) ** 3

    def nodes(self):
        """Physical position of every node, [Ne, K]."""
        xl = self.x0 + self.h * np.arange(self.Ne)
        return xl[:, None] + (self.xi[None, :] + 1.0) * self.h / 2.0

    # -- boundary ----------------------------------------------------------------------
    def wall_state(self, side, f_int):
        """Exterior state of the wall face (Sec. 2, Maxwell boundary condition) for interior
        trace f_int[s, N, N, N]: at velocities entering the domain,
        (1 - acc) f_int(reflected v) + acc n_w exp(-m_i |v - u_w|^2 / T_w), with n_w from zero
        net mass flux through the wall (the discrete sums over the velocity grid); elsewhere
        the interior trace (only the upwind side is used)."""
        n_out = -1.0 if side == 0 else 1.0
        out = np.array(f_int, copy=True)
        Tw, uw, a = self.Tw[side], self.uw[side], self.acc[side]
        if self.side_kind[side] == "inflow":
            # in-flow equilibrium (Sec. 2): n_in (m / (pi T))^(3/2) exp(-m |v - u|^2 / T) for
            # entering velocities v . n < 0
            incoming = self.vx * n_out < 0
            for i, m in enumerate(self.prob.masses):
                d2 = sum((self.V[d] - uw[d]) ** 2 for d in range(3))
                inflow = self.n_in[side][i] * (m / (np.pi * Tw)) ** 1.5 * np.exp(-m * d2 / Tw)
                out[i] = np.where(incoming, inflow, f_int[i])
            return out
        cn = self.vx * n_out                                        # (v - u_w) . n, u_w . n = 0
        incoming = cn < 0
        for i, m in enumerate(self.prob.masses):
            d2 = sum((self.V[d] - uw[d]) ** 2 for d in range(3))
            wall = np.exp(-m * d2 / Tw)
            num = np.sum(np.where(~incoming, cn * f_int[i], 0.0))
            den = np.sum(np.where(incoming, cn * wall, 0.0))
            n_w = -num / den
            reflected = f_int[i][::-1, :, :]                        # v_x -> -v_x on the grid
            out[i] = np.where(incoming, (1.0 - a) * reflected + a * n_w * wall, f_int[i])
        return out

    # -- transport ---------------------------------------------------------------------
    def transport_rhs(self, F):
        """d F / dt from the transport term alone (Eq. weakForm without the collision term):
        M dF/dt = v_x S F - [phi_m F_* n] over both faces, upwind flux F_* = v_x f_upwind."""
        Ne, K = self.Ne, self.K
        out = np.zeros_like(F)
        for e in range(Ne):
            # exterior traces at the left and right faces of element e
            if e > 0:
                left_ext = F[e - 1, K - 1]
            elif self.bc == "periodic":
                left_ext = F[Ne - 1, K - 1]
            else:
                left_ext = self.wall_state(0, F[0, 0])
            if e < Ne - 1:
                right_ext = F[e + 1, 0]
            elif self.bc == "periodic":
                right_ext = F[0, 0]
            else:
                right_ext = self.wall_state(1, F[Ne - 1, K - 1])
            vx = self.vx[None]
            # outward normal +1 at the right face, -1 at the left face; upwind: the interior
            # trace when v . n >= 0
            flux_r = vx * np.where(vx >= 0, F[e, K - 1], right_ext)
            flux_l = vx * np.where(-vx >= 0, F[e, 0], left_ext)
            for m in range(K):
                vol = sum(self.S[m, l] * F[e, l] for l in range(K)) * vx
                surf = (1.0 if m == K - 1 else 0.0) * flux_r - (1.0 if m == 0 else 0.0) * flux_l
                out[e, m] = vol - surf
            out[e] = np.einsum("ml,l...->m...", self.Minv, out[e])
        return out

    # -- collision -----------------------------------------------------------------------
    def collision_rhs(self, F, kappa):
        """sum_j kappa_ij Q_ij at every node: the collision term of Eq. weakForm with the
        GLL-quadrature tensor H (diagonal), divided by the diagonal mass matrix.  kappa_ij plays
        1/Kn_ij of Eq. NMBE."""
        Ne, K = self.Ne, self.K
        H = collision_tensor(K, self.h)
        # the GLL rule makes H diagonal: only Q(F_l, F_l) terms remain (Sec. 5)
        off = H.copy()
        for m in range(K):
            off[m, m, m] = 0.0
        assert not np.any(off)
        out = np.zeros_like(F)
        for e in range(Ne):
            Qn = [moments.species_sum(fast_spectral.collision(F[e, l], self.prob)[0], kappa)
                  for l in range(K)]
            for m in range(K):
                out[e, m] = sum(H[m, l, l] * Qn[l] for l in range(K))
            out[e] = np.einsum("ml,l...->m...", self.Minv, out[e])
        return out

    def rhs(self, F, kappa=None, collisions=True):
        r = self.transport_rhs(F)
        if collisions:
            r = r + self.collision_rhs(F, kappa)
        return r

    def ssp_rk2_step(self, F, dt, kappa=None, collisions=True):
        """SSP-RK2 (Sec. 5): F1 = F + dt R(F); F_new = F/2 + (F1 + dt R(F1))/2."""
        F1 = F + dt * self.rhs(F, kappa, collisions)
        return 0.5 * F + 0.5 * (F1 + dt * self.rhs(F1, kappa, collisions))

    def mass(self, F):
        """Total mass per species, sum_e sum_ml M_ml int F_l dv, with the scheme's (GLL) mass
        matrix and the velocity-grid sums."""
        dens = F.sum(axis=(3, 4, 5)) * self.dv3                            # [Ne, K, s]
        return np.einsum("ml,elk->k", self.M, dens)
