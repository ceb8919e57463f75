"""The 1D DG path (dgfs_dg_*) against the DG oracle: transport right-hand side, the full
SSP-RK2 step with collisions, node positions, mass conservation over many steps, and argument
checks."""

import numpy as np
import pytest

from gpu_helpers import TOL_FP32
from oracle import dg1d, fast_spectral as fs
from paper_1903_03056_gb300 import build, dgfs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    build.build()
    dgfs.load()


def _state(Ne, K, s, N, seed):
    rng = np.random.default_rng(seed)
    return 0.2 + rng.random((Ne, K, s, N, N, N))


def _setup(precision, N, L, masses, Ne, K, bc, Tw, uw, acc, kappa=None, flags=0, M=6, N_rho=4,
           side_kind=("wall", "wall"), n_in=None):
    coll = dgfs.Plan(N, L, list(masses), 0.7, M=M, N_rho=N_rho, precision=precision, flags=flags,
                     max_batch=Ne * K, kappa=kappa)
    dg = dgfs.DGPlan(coll, Ne, K, 0.0, 1.3, bc=bc, Tw=Tw, uw=uw, acc=acc, side_kind=side_kind,
                     n_in=n_in)
    prob = fs.make_problem(N, L, list(masses), omega=0.7, M=M, N_rho=N_rho)
    ora = dg1d.DG1D(prob, Ne, K, 0.0, 1.3, bc=bc, Tw=Tw, uw=uw, acc=acc, side_kind=side_kind,
                    n_in=n_in)
    return coll, dg, ora


WALLS = dict(Tw=(0.8, 1.3), uw=((0.0, 0.3, 0.0), (0.0, -0.2, 0.1)))


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("bc,acc,K", [("periodic", (1.0, 1.0), 3), ("walls", (1.0, 1.0), 3),
                                      ("walls", (0.4, 0.9), 2), ("walls", (0.0, 1.0), 4)])
def test_transport_matches_oracle(precision, bc, acc, K):
    import torch
    N, L, masses, Ne = 8, 4.0, (1.0, 2.0), 3
    coll, dg, ora = _setup(precision, N, L, masses, Ne, K, bc, acc=acc, **WALLS)
    F = _state(Ne, K, 2, N, seed=K * 10 + int(acc[0] * 10))
    dt = torch.float64 if precision == "fp64" else torch.float32
    fd = torch.from_numpy(F.reshape(Ne * K, 2, N, N, N)).to("cuda", dt)
    r = dg.transport(fd)
    torch.cuda.synchronize()
    got = r.double().cpu().numpy().reshape(F.shape)
    ref = ora.transport_rhs(F)
    err = np.max(np.abs(got - ref)) / np.max(np.abs(ref))
    assert err < (1e-12 if precision == "fp64" else TOL_FP32), err
    dg.close()
    coll.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("sides", [("inflow", "wall"), ("inflow", "inflow")])
def test_transport_with_inflow_sides_matches_oracle(precision, sides):
    """In-flow equilibrium sides (Sec. 2): drifting in-flow Maxwellians with their own
    densities, temperature and velocity (x components allowed there)."""
    import torch
    N, L, masses, Ne, K = 8, 4.0, (1.0, 2.0), 3, 3
    uw = ((0.4, 0.1, 0.0), (0.0 if sides[1] == "wall" else -0.3, -0.2, 0.1))
    coll, dg, ora = _setup(precision, N, L, masses, Ne, K, "walls", Tw=(1.1, 0.9), uw=uw,
                           acc=(1.0, 0.7), side_kind=sides, n_in=((0.9, 0.4), (0.6, 0.7)))
    F = _state(Ne, K, 2, N, seed=31)
    dt = torch.float64 if precision == "fp64" else torch.float32
    fd = torch.from_numpy(F.reshape(Ne * K, 2, N, N, N)).to("cuda", dt)
    got = dg.transport(fd).double().cpu().numpy().reshape(F.shape)
    ref = ora.transport_rhs(F)
    err = np.max(np.abs(got - ref)) / np.max(np.abs(ref))
    assert err < (1e-12 if precision == "fp64" else TOL_FP32), err
    dg.close()
    coll.close()


def test_nodes_match_oracle():
    coll, dg, ora = _setup("fp64", 4, 3.0, (1.0, 2.0), 5, 4, "periodic", acc=(1.0, 1.0), **WALLS)
    assert np.max(np.abs(dg.nodes() - ora.nodes())) < 1e-14
    dg.close()
    coll.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_full_step_matches_oracle(precision):
    """One SSP-RK2 step of transport + sum_j kappa_ij Q_ij against the oracle's step."""
    import torch
    N, L, masses, Ne, K = 8, 4.0, (1.0, 2.0), 2, 3
    kappa = [1.3, 0.7, 0.9, 1.1]
    coll, dg, ora = _setup(precision, N, L, masses, Ne, K, "walls", acc=(1.0, 0.6),
                           kappa=kappa, flags=dgfs.DGFS_SUM_SPECIES, **WALLS)
    F = _state(Ne, K, 2, N, seed=5)
    dtt = torch.float64 if precision == "fp64" else torch.float32
    fd = torch.from_numpy(F.reshape(Ne * K, 2, N, N, N)).to("cuda", dtt)
    dt = 2e-3
    dg.step(fd, dt)
    torch.cuda.synchronize()
    got = fd.double().cpu().numpy().reshape(F.shape)
    ref = ora.ssp_rk2_step(F, dt, kappa=np.asarray(kappa).reshape(2, 2))
    # compare the change of the step (the state itself is O(1))
    err = np.max(np.abs((got - F) - (ref - F))) / np.max(np.abs(ref - F))
    assert err < (1e-10 if precision == "fp64" else 1e-4), err
    dg.close()
    coll.close()


def test_mass_is_conserved_over_many_steps_with_walls():
    """Each species' mass is conserved: the fluxes telescope, the Maxwell walls return the
    outgoing flux, and the projected collision term has no mass.  FP64, N = 16, 8 elements of
    K = 3, 20 steps."""
    import torch
    N, L, masses, Ne, K = 16, 5.0, (1.0, 2.0), 8, 3
    coll, dg, ora = _setup("fp64", N, L, masses, Ne, K, "walls", acc=(1.0, 0.5),
                           kappa=[1.0, 1.0, 1.0, 1.0],
                           flags=dgfs.DGFS_SUM_SPECIES | dgfs.DGFS_CONSERVE, **WALLS)
    # the collision plan projects onto the conservation laws (the fast method alone conserves
    # mass only to its spectral accuracy), so what remains is the transport's and the walls'
    # conservation
    X = ora.nodes()
    v = fs.velocity_grid(N, L)
    F = np.zeros((Ne, K, 2, N, N, N))
    for i, m in enumerate(masses):
        e = np.exp(-m * v ** 2)
        Mx = (m / np.pi) ** 1.5 * e[:, None, None] * e[None, :, None] * e[None, None, :]
        F[:, :, i] = (1.0 + 0.4 * np.sin(2 * np.pi * X / 1.3))[:, :, None, None, None] * Mx
    m0 = ora.mass(F)
    fd = torch.from_numpy(F.reshape(Ne * K, 2, N, N, N)).cuda()
    for _ in range(20):
        dg.step(fd, 2e-3)
    torch.cuda.synchronize()
    m1 = ora.mass(fd.cpu().numpy().reshape(F.shape))
    assert np.max(np.abs(m1 - m0) / m0) < 1e-10
    dg.close()
    coll.close()


def test_argument_checks():
    import torch
    coll = dgfs.Plan(8, 4.0, [1.0, 2.0], 0.7, M=6, N_rho=2, precision="fp64")
    bad = [dict(Ne=0, K=3), dict(Ne=2, K=9), dict(Ne=2, K=1),
           dict(Ne=2, K=3, bc="walls", uw=((0.1, 0.0, 0.0), (0.0, 0.0, 0.0))),
           dict(Ne=2, K=3, bc="walls", acc=(1.2, 1.0)), dict(Ne=2, K=3, bc="walls", Tw=(0.0, 1.0)),
           dict(Ne=2, K=3, bc="walls", side_kind=("inflow", "wall")),               # no n_in
           dict(Ne=2, K=3, bc="walls", side_kind=("inflow", "wall"), n_in=((-1.0, 1.0), (1.0, 1.0)))]
    for kw in bad:
        Ne, K = kw.pop("Ne"), kw.pop("K")
        with pytest.raises(dgfs.DgfsError) as ei:
            dgfs.DGPlan(coll, Ne, K, **kw)
        assert ei.value.code == dgfs.DGFS_ERR_INVALID_ARG
    # a step needs a species-summing collision plan with room for Ne * K nodes
    dg = dgfs.DGPlan(coll, 2, 3)
    f = torch.zeros((6, 2, 8, 8, 8), dtype=torch.float64, device="cuda")
    with pytest.raises(dgfs.DgfsError) as ei:
        dg.step(f, 1e-3)
    assert ei.value.code == dgfs.DGFS_ERR_INVALID_ARG
    dg.close()
    coll2 = dgfs.Plan(8, 4.0, [1.0, 2.0], 0.7, M=6, N_rho=2, precision="fp64",
                      flags=dgfs.DGFS_SUM_SPECIES, max_batch=4)
    dg2 = dgfs.DGPlan(coll2, 2, 3)
    with pytest.raises(dgfs.DgfsError) as ei:
        dg2.step(f, 1e-3)
    assert ei.value.code == dgfs.DGFS_ERR_BUDGET
    dg2.close()
    coll2.close()
    coll.close()
