"""Pins of the DG oracle (Sec. 5) and of the Maxwell wall condition (Sec. 2).

Each check uses a closed form, a worked value the paper prints, or an identity of the
discretisation, never the oracle against itself."""

import numpy as np
import pytest

from oracle import dg1d, fast_spectral as fs


# ------------------------------------------------------------------------ GLL rule, basis

@pytest.mark.parametrize("K", [2, 3, 4, 5, 6, 8])
def test_gll_rule_integrates_degree_2K_minus_3(K):
    xi, w = dg1d.gll(K)
    for p in range(2 * K - 2):
        exact = 0.0 if p % 2 else 2.0 / (p + 1)
        assert abs(np.sum(w * xi ** p) - exact) < 1e-13
    # and not degree 2K - 2 (the rule is not Gauss-Legendre)
    p = 2 * K - 2
    assert abs(np.sum(w * xi ** p) - 2.0 / (p + 1)) > 1e-6


def test_collision_tensor_matches_the_printed_K3_example():
    """Sec. 5 prints, for K = 3 GLL points, H^(st)_m = diag(1/3, 0, 0), diag(0, 4/3, 0),
    diag(0, 0, 1/3) (H = (h/2) H^(st))."""
    h = 0.7
    H = dg1d.collision_tensor(3, h) / (h / 2.0)
    for m, val in enumerate([1.0 / 3.0, 4.0 / 3.0, 1.0 / 3.0]):
        ref = np.zeros((3, 3))
        ref[m, m] = val
        assert np.max(np.abs(H[m] - ref)) < 1e-14


@pytest.mark.parametrize("K", [2, 3, 5])
def test_lagrange_derivative_differentiates_polynomials_exactly(K):
    xi, _ = dg1d.gll(K)
    x = np.linspace(-1, 1, 7)
    coef = np.random.default_rng(K).normal(size=K)          # degree K - 1
    p = np.polynomial.Polynomial(coef)
    got = sum(p(xi[m]) * dg1d.lagrange_deriv(xi, m, x) for m in range(K))
    assert np.max(np.abs(got - p.deriv()(x))) < 1e-12


@pytest.mark.parametrize("K", [2, 3, 4, 6])
def test_stiffness_summation_by_parts(K):
    """S + S^T = diag(-1, 0, ..., 0, 1): int (phi_l phi_m' + phi_m phi_l') = [phi_l phi_m]."""
    _, S = dg1d.element_matrices(K, 0.3)
    B = np.zeros((K, K))
    B[0, 0], B[-1, -1] = -1.0, 1.0
    assert np.max(np.abs(S + S.T - B)) < 1e-13


# ---------------------------------------------------------------------- transport and walls

def _problem(N=4, s=2):
    return fs.make_problem(N, 4.0, [1.0, 2.0][:s], omega=0.7, M=6, N_rho=2)


def _maxwellian(N, L, m):
    """Resting unit-density Maxwellian of temperature 1 on the grid (Sec. 3 form)."""
    v = fs.velocity_grid(N, L)
    e = np.exp(-m * v ** 2)
    return (m / np.pi) ** 1.5 * e[:, None, None] * e[None, :, None] * e[None, None, :]


def _profile_state(dg, g):
    """F[e, m, i, v] = g(x_em) M_i(v), a spatial profile times a Maxwellian per species."""
    prob = dg.prob
    X = dg.nodes()
    out = np.zeros((dg.Ne, dg.K, prob.s) + (prob.N,) * 3)
    for i, m in enumerate(prob.masses):
        M = _maxwellian(prob.N, prob.L, m)
        out[:, :, i] = g(X)[:, :, None, None, None] * M[None, None]
    return out


@pytest.mark.parametrize("K", [2, 3, 4])
def test_periodic_transport_converges_to_minus_vx_dx(K):
    """With a smooth periodic profile the transport rhs at the nodes approaches
    -v_x g'(x) M(v) at order K - 1 in h (a dropped flux term or a wrong upwind side stalls it)."""
    prob = _problem()
    errs = []
    for Ne in (8, 16, 32):
        dg = dg1d.DG1D(prob, Ne, K, 0.0, 1.0, bc="periodic")
        F = _profile_state(dg, lambda x: 1.0 + 0.3 * np.sin(2 * np.pi * x))
        r = dg.transport_rhs(F)
        dgx = _profile_state(dg, lambda x: 0.3 * 2 * np.pi * np.cos(2 * np.pi * x))
        ref = -dg.vx[None, None, None] * dgx
        errs.append(np.max(np.abs(r - ref)) / np.max(np.abs(ref)))
    rate = errs[1] / errs[2]
    assert 0.9 * 2 ** (K - 1) < rate < 1.1 * 2 ** (K - 1)


@pytest.mark.parametrize("bc,acc", [("periodic", (1.0, 1.0)), ("walls", (1.0, 1.0)),
                                    ("walls", (0.3, 0.8)), ("walls", (0.0, 0.0))])
def test_transport_conserves_mass(bc, acc):
    """sum of M * rhs over elements, nodes and velocities is zero: fluxes telescope, and the
    Maxwell wall returns the outgoing mass flux (n_w's definition; specular part by symmetry)."""
    prob = _problem()
    dg = dg1d.DG1D(prob, 3, 3, 0.0, 1.0, bc=bc, Tw=(0.8, 1.3),
                   uw=((0.0, 0.2, 0.0), (0.0, -0.1, 0.05)), acc=acc)
    rng = np.random.default_rng(7)
    F = rng.random((3, 3, 2) + (prob.N,) * 3)
    r = dg.transport_rhs(F)
    assert np.max(np.abs(dg.mass(r))) < 1e-13 * np.max(np.abs(dg.mass(F)))


def test_wall_at_gas_temperature_keeps_a_resting_maxwellian():
    """A uniform resting Maxwellian between diffuse walls at its own temperature is a steady
    state of the transport term: the wall re-emits exactly the incoming half."""
    prob = _problem()
    dg = dg1d.DG1D(prob, 2, 3, 0.0, 1.0, bc="walls", Tw=(1.0, 1.0))
    F = _profile_state(dg, lambda x: 0.8 + 0.0 * x)
    assert np.max(np.abs(dg.transport_rhs(F))) < 1e-12 * np.max(np.abs(F))


def test_specular_wall_mirrors_the_outgoing_half():
    prob = _problem()
    dg = dg1d.DG1D(prob, 2, 2, 0.0, 1.0, bc="walls", acc=(0.0, 0.0))
    rng = np.random.default_rng(3)
    f = rng.random((2,) + (prob.N,) * 3)
    ext = dg.wall_state(0, f)
    incoming = dg.vx > 0                      # left wall, outward normal -x
    assert np.allclose(ext[:, incoming], f[:, ::-1][:, incoming])


def test_rk_step_without_collisions_conserves_mass_and_is_second_order():
    prob = _problem()
    dg = dg1d.DG1D(prob, 4, 3, 0.0, 1.0, bc="walls", Tw=(0.9, 1.2), acc=(1.0, 0.5))
    rng = np.random.default_rng(11)
    F = 0.5 + rng.random((4, 3, 2) + (prob.N,) * 3)
    m0 = dg.mass(F)
    F1 = dg.ssp_rk2_step(F, 1e-3, collisions=False)
    assert np.max(np.abs(dg.mass(F1) - m0)) < 1e-13 * np.max(m0)
    # halving dt: the local error of a second-order step drops 8x
    fine = dg.ssp_rk2_step(dg.ssp_rk2_step(F, 5e-4, collisions=False), 5e-4, collisions=False)
    ref = F
    for _ in range(16):
        ref = dg.ssp_rk2_step(ref, 1e-3 / 16, collisions=False)
    e1 = np.max(np.abs(F1 - ref))
    e2 = np.max(np.abs(fine - ref))
    assert e2 < e1 / 3.0


def test_upwind_flux_takes_the_upstream_trace():
    """Two periodic elements, F = 1 in the first and 0 in the second (K = 2, w = 1): at the
    second element's left node the transport rhs is (2/h) v_x for v_x > 0 (the upstream
    element's trace enters) and 0 for v_x < 0 (its own zero trace leaves)."""
    prob = _problem()
    dg = dg1d.DG1D(prob, 2, 2, 0.0, 1.0, bc="periodic")
    F = np.zeros((2, 2, 2) + (prob.N,) * 3)
    F[0] = 1.0
    r = dg.transport_rhs(F)
    ref = np.where(dg.vx > 0, (2.0 / dg.h) * dg.vx, 0.0)
    for i in range(2):
        assert np.max(np.abs(r[1, 0, i] - ref)) < 1e-13


def test_inflow_boundary_keeps_its_own_maxwellian():
    """In-flow equilibrium sides (Sec. 2): a uniform state equal to the in-flow Maxwellian
    (drifting along x, so particles enter through both sides) is steady under transport; a
    different interior state is not."""
    prob = _problem()
    u, T, n = (0.3, 0.1, 0.0), 1.2, (0.8, 0.5)
    dg = dg1d.DG1D(prob, 3, 3, 0.0, 1.0, bc="walls", Tw=(T, T), uw=(u, u),
                   side_kind=("inflow", "inflow"), n_in=(n, n))
    v = fs.velocity_grid(prob.N, prob.L)
    F = np.zeros((3, 3, 2) + (prob.N,) * 3)
    for i, m in enumerate(prob.masses):
        e = [np.exp(-m * (v - u[d]) ** 2 / T) for d in range(3)]
        M = n[i] * (m / (np.pi * T)) ** 1.5 * e[0][:, None, None] * e[1][None, :, None] * e[2][None, None, :]
        F[:, :, i] = M
    assert np.max(np.abs(dg.transport_rhs(F))) < 1e-12 * np.max(F)
    assert np.max(np.abs(dg.transport_rhs(0.5 * F))) > 1e-3 * np.max(F)
