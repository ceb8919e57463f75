"""dgfs_eval_collision_noalloc: the plan-free entry point for callers that cannot allocate
device memory (a host application that owns every device allocation, code that may not call
cudaMalloc after start-up).  It must give the same Q as dgfs_eval_collision, call after call,
while allocating nothing, and agree with the oracle.  This file is collected last."""

import numpy as np
import pytest

from gpu_helpers import max_rel_error, oracle_collision, TOL_FP32
from paper_1903_03056_gb300 import build, dgfs, synth

pytestmark = pytest.mark.gpu

# set once the first call of this process has returned: that call performs the one-time
# set-up in the CUDA context (symbol lookup, shared-memory limits); every later call must
# leave the device's free memory unchanged
_SETUP = {"done": False}


@pytest.fixture(scope="module", autouse=True)
def built():
    build.build()
    dgfs.load()


def _inputs(N, L, masses, B, seed):
    w = synth.Workload("noalloc", B, N, L, tuple(masses), 0.5, 1.0, 6, 4, "bimaxwellian", 0.05, seed)
    return synth.batch_distribution(w, dtype=np.float32)


def _noalloc(desc, f, B, s, N):
    """One call through the C ABI; checks that it allocated nothing once set up."""
    import torch
    Q = torch.full((B, s, s, N, N, N), float("nan"), dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    was_set_up = _SETUP["done"]
    free_before = torch.cuda.mem_get_info()[0]
    code = dgfs.dgfs_eval_collision_noalloc(desc, f.data_ptr(), Q.data_ptr(), B, None)
    torch.cuda.synchronize()
    assert code == dgfs.DGFS_OK, dgfs.dgfs_strerror(code)
    _SETUP["done"] = True
    if was_set_up:
        assert torch.cuda.mem_get_info()[0] == free_before
    assert not bool(torch.isnan(Q).any()), "an element of Q was not written"
    return Q


CASES = {
    # built-in antipodal designs: unordered tasks, halved self pairs
    "n16_icosahedron": dict(N=16, L=6.0, masses=(1.0, 2.0), omega=0.5, M=12, N_rho=8, B=70),
    "n12_three_species": dict(N=12, L=5.0, masses=(1.0, 1.5, 2.6), omega=0.74, M=6, N_rho=4, B=5),
    # user radius and kernel prefactors
    "n8_user_R_and_b": dict(N=8, L=4.0, masses=(1.0, 3.0), omega=0.8, M=6, N_rho=3, B=3, R=2.5,
                            b_override=np.array([[0.11, 0.07], [0.05, 0.13]])),
}


def _user_sigma():
    """Five directions without antipodes and unequal weights: every ordered pair is its own
    task with the full rule (no halving, no (i,j)/(j,i) reuse)."""
    rng = np.random.default_rng(21)
    sigma = rng.normal(size=(5, 3))
    sigma /= np.linalg.norm(sigma, axis=1, keepdims=True)
    return sigma, np.array([2.1, 2.9, 2.4, 2.6, 2.566370614359172])


@pytest.mark.parametrize("name", sorted(CASES) + ["n8_non_antipodal"])
def test_noalloc_matches_plan_path_and_oracle_on_two_calls(name):
    import torch
    if name == "n8_non_antipodal":
        sigma, w = _user_sigma()
        kw = dict(N=8, L=4.0, masses=(1.0, 2.0), omega=0.7, M=5, N_rho=3, sigma=sigma, w_sigma=w)
        B = 4
    else:
        kw = dict(CASES[name])
        B = kw.pop("B")
    N, L, masses, omega = kw["N"], kw["L"], list(kw["masses"]), kw["omega"]
    extra = {k: v for k, v in kw.items() if k in ("M", "N_rho", "sigma", "w_sigma", "R", "b_override")}
    plan = dgfs.Plan(N, L, masses, omega, precision="fp32", **extra)
    desc, keep = dgfs.make_desc(N, L, masses, omega, precision="fp32", **extra)
    s = len(masses)
    for call, seed in enumerate((11, 12)):
        f_np = _inputs(N, L, masses, B, seed)
        f = torch.from_numpy(f_np).cuda()
        ref = plan.eval(f)
        Q = _noalloc(desc, f, B, s, N)
        err = max_rel_error(Q.double().cpu().numpy(), ref.double().cpu().numpy(), "node")
        assert err < TOL_FP32, (call, err)
        if call == 0:
            # the first two nodes against the FP64 oracle
            okw = dict(M=kw["M"], N_rho=kw["N_rho"], sigma=kw.get("sigma"), w_sigma=kw.get("w_sigma"),
                       b_override=kw.get("b_override"), R=kw.get("R"))
            oref = oracle_collision(f_np[:2].astype(np.float64), N=N, L=L, masses=masses, omega=omega, **okw)
            err_o = max_rel_error(Q[:2].double().cpu().numpy(), oref, "node")
            assert err_o < TOL_FP32, err_o
    plan.close()
    del keep


@pytest.mark.parametrize("kw,code", [
    (dict(N=32), dgfs.DGFS_ERR_UNSUPPORTED_N),
    (dict(N=24), dgfs.DGFS_ERR_UNSUPPORTED_N),
    (dict(masses=[1.0, 2.0, 3.0, 4.0]), dgfs.DGFS_ERR_UNSUPPORTED),
    (dict(M=32), dgfs.DGFS_ERR_UNSUPPORTED),
    (dict(N_rho=17), dgfs.DGFS_ERR_UNSUPPORTED),
    (dict(precision="fp64"), dgfs.DGFS_ERR_UNSUPPORTED),
    (dict(L=float("inf")), dgfs.DGFS_ERR_INVALID_ARG),
    (dict(R=float("inf")), dgfs.DGFS_ERR_INVALID_ARG),
    (dict(R=float("nan")), dgfs.DGFS_ERR_INVALID_ARG),
    (dict(b_override=np.array([[0.1, float("inf")], [0.1, 0.1]])), dgfs.DGFS_ERR_INVALID_ARG),
    (dict(b_override=np.array([[0.1, 0.1], [float("nan"), 0.1]])), dgfs.DGFS_ERR_INVALID_ARG),
    (dict(w_sigma=np.array([1.0] * 11 + [float("nan")])), dgfs.DGFS_ERR_INVALID_ARG),
])
def test_noalloc_rejects_sizes_beyond_its_limits(kw, code):
    import torch
    base = dict(N=16, L=6.0, masses=[1.0, 2.0], omega=0.5, M=12, N_rho=8, precision="fp32")
    base.update(kw)
    if "w_sigma" in kw:
        from oracle import quadrature
        base["sigma"] = quadrature.spherical_design(12)[0]
    N, L, masses, omega = base.pop("N"), base.pop("L"), base.pop("masses"), base.pop("omega")
    desc, keep = dgfs.make_desc(N, L, masses, omega, **base)
    buf = torch.zeros(16, dtype=torch.float32, device="cuda")
    assert dgfs.dgfs_eval_collision_noalloc(desc, buf.data_ptr(), buf.data_ptr(), 1, None) == code
