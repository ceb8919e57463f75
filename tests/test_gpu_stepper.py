"""SSP-RK2 homogeneous stepping on the device (dgfs_ssp_rk2_step): one step against the
oracle's step, and the Krook-Wu evolution against the exact solution (Sec. 6.1)."""

import numpy as np
import pytest

from oracle import fast_spectral as fs, homogeneous, krook_wu
from paper_1903_03056_gb300 import build, dgfs, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    build.build()
    dgfs.load()


def test_one_step_matches_oracle():
    import torch
    N, L, masses = 12, 5.0, [1.0, 2.0]
    kappa = np.array([[1.0, 0.8], [1.3, 1.0]])
    w = synth.Workload("rk", 2, N, L, tuple(masses), 0.6, 1.0, 6, 3, "bimaxwellian", 0.0, 17)
    f = synth.batch_distribution(w)
    plan = dgfs.Plan(N, L, masses, 0.6, M=6, N_rho=3, precision="fp64", kappa=kappa,
                     flags=dgfs.DGFS_SUM_SPECIES, max_batch=2)
    fd = torch.from_numpy(f).cuda()
    plan.ssp_rk2_step(fd, 0.05)
    torch.cuda.synchronize()
    assert plan.launches() == 6
    prob = fs.make_problem(N, L, masses, omega=0.6, M=6, N_rho=3)
    ref = np.stack([homogeneous.ssp_rk2_step(fb, 0.05, homogeneous.collision_rhs(prob, kappa)) for fb in f])
    got = fd.cpu().numpy()
    assert np.max(np.abs(got - ref)) < 1e-11 * np.max(np.abs(ref))
    plan.close()


def test_krook_wu_evolution_follows_the_exact_solution():
    """From t = 4 to t = 5 with dt = 0.01 (N = 32, M = 6, N_rho = 16, m1/m2 = 2): the numerical
    f stays within twice the Table 1 error of d_t f (1.729e-3) integrated over the unit time."""
    import torch
    N, L, ratio = 32, 12.0, 2.0
    kw = krook_wu.KrookWu(ratio, 1.0)
    v = fs.velocity_grid(N, L)
    vx, vy, vz = np.meshgrid(v, v, v, indexing="ij")
    v2 = vx * vx + vy * vy + vz * vz
    f0 = np.stack([kw.f(0, 4.0, v2), kw.f(1, 4.0, v2)])[None]
    plan = dgfs.Plan(N, L, [ratio, 1.0], 1.0, M=6, N_rho=16, precision="fp64",
                     b_override=kw.kernel_prefactors(), flags=dgfs.DGFS_SUM_SPECIES, max_batch=1)
    fd = torch.from_numpy(np.ascontiguousarray(f0)).cuda()
    for _ in range(100):
        plan.ssp_rk2_step(fd, 0.01)
    torch.cuda.synchronize()
    got = fd.cpu().numpy()[0]
    exact = np.stack([kw.f(0, 5.0, v2), kw.f(1, 5.0, v2)])
    err = np.max(np.abs(got - exact), axis=(1, 2, 3))
    change = np.max(np.abs(exact - f0[0]), axis=(1, 2, 3))
    print("Krook-Wu t=4->5: max error per species", err, "exact change", change)
    assert np.all(err < 2 * 1.729e-3 * 1.0)
    assert np.all(err < 0.2 * change)
    plan.close()
