"""DGFS_CONSERVE (FP64 moment sums, projection onto the discrete laws of Eq. consv) and
DGFS_SUM_SPECIES (sum_j kappa_ij Q_ij) against the oracle's projection and sum."""

import numpy as np
import pytest

from gpu_helpers import check, oracle_collision, TOL_FP32, TOL_FP64
from oracle import fast_spectral as fs, moments
from paper_1903_03056_gb300 import build, dgfs, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    build.build()
    dgfs.load()


def _inputs(N, L, masses, B, seed):
    w = synth.Workload("cons", B, N, L, tuple(masses), 0.5, 1.0, 6, 4, "bimaxwellian", 0.05, seed)
    return synth.batch_distribution(w)


def _gpu(f, precision, flags, kappa=None, **kw):
    import torch
    dt = torch.float32 if precision == "fp32" else torch.float64
    plan = dgfs.Plan(kw["N"], kw["L"], list(kw["masses"]), kw["omega"], M=kw["M"], N_rho=kw["N_rho"],
                     precision=precision, flags=flags, kappa=kappa, max_batch=f.shape[0])
    Q = plan.eval(torch.from_numpy(f).to(device="cuda", dtype=dt))
    torch.cuda.synchronize()
    n = plan.launches()
    out = Q.double().cpu().numpy()
    plan.close()
    return out, n


def _residual(Q, masses, L, b):
    r = moments.conservation_residuals(Q, masses, L, kappa=1.0 / b)
    return max(np.max(np.abs(r["mass"]) / r["mass_scale"]),
               np.max(np.linalg.norm(r["momentum"], axis=-1) / r["momentum_scale"]),
               np.max(np.abs(r["energy"]) / r["energy_scale"]))


CASES = [dict(N=16, L=6.0, masses=(1.0, 2.0), omega=0.5, M=12, N_rho=8, B=3),
         dict(N=12, L=5.0, masses=(1.0, 1.5, 2.6), omega=0.74, M=6, N_rho=4, B=2)]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("case", range(len(CASES)))
def test_conserve_matches_oracle_projection(case, precision):
    kw = dict(CASES[case])
    B = kw.pop("B")
    f = _inputs(kw["N"], kw["L"], kw["masses"], B, seed=50 + case)
    Q, n = _gpu(f, precision, dgfs.DGFS_CONSERVE, **kw)
    assert n == 2
    prob = fs.make_problem(kw["N"], kw["L"], list(kw["masses"]), omega=kw["omega"], M=kw["M"],
                           N_rho=kw["N_rho"])
    raw = oracle_collision(f, **kw)
    ref = np.stack([moments.conservation_projection(q, kw["masses"], kw["L"], prob.b) for q in raw])
    assert check(Q, ref, precision)
    before = max(_residual(q, kw["masses"], kw["L"], prob.b) for q in raw)
    after = max(_residual(q, kw["masses"], kw["L"], prob.b) for q in Q)
    print("%s conservation residual: method %.2e, projected %.2e" % (precision, before, after))
    assert after < (1e-12 if precision == "fp64" else 1e-6)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_species_sum_with_kappa_and_projection(precision):
    kw = dict(CASES[1])
    B = kw.pop("B")
    f = _inputs(kw["N"], kw["L"], kw["masses"], B, seed=61)
    kappa = np.array([[1.0, 0.5, 2.0], [0.7, 1.3, 0.2], [1.1, 0.9, 0.4]])
    flags = dgfs.DGFS_CONSERVE | dgfs.DGFS_SUM_SPECIES
    S, n = _gpu(f, precision, flags, kappa=kappa, **kw)
    assert n == 3 and S.shape == (B, 3) + (kw["N"],) * 3
    prob = fs.make_problem(kw["N"], kw["L"], list(kw["masses"]), omega=kw["omega"], M=kw["M"],
                           N_rho=kw["N_rho"])
    raw = oracle_collision(f, **kw)
    ref = np.stack([moments.species_sum(moments.conservation_projection(q, kw["masses"], kw["L"], prob.b), kappa)
                    for q in raw])
    err = max(np.max(np.abs(S[b] - ref[b])) / np.max(np.abs(ref[b])) for b in range(B))
    assert err < (TOL_FP64 if precision == "fp64" else TOL_FP32)


def test_species_sum_needs_max_batch():
    import torch
    plan = dgfs.Plan(8, 4.0, [1.0, 2.0], 0.5, M=6, N_rho=2, precision="fp32",
                     flags=dgfs.DGFS_SUM_SPECIES, max_batch=2)
    f = torch.zeros((3, 2, 8, 8, 8), dtype=torch.float32, device="cuda")
    Q = torch.zeros((3, 2, 8, 8, 8), dtype=torch.float32, device="cuda")
    assert dgfs.dgfs_eval_collision(plan.handle, f.data_ptr(), Q.data_ptr(), 3, None) == dgfs.DGFS_ERR_BUDGET
    plan.close()
