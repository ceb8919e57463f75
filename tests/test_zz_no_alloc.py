"""dgfs_eval_collision_noalloc: the plan-free entry point for callers that cannot allocate
device memory (a host application that owns every device allocation, code that may not call
cudaMalloc after start-up).  It must give the same Q as dgfs_eval_collision, call after call,
while allocating nothing.  This file is collected last."""

import numpy as np
import pytest

from gpu_helpers import max_rel_error, TOL_FP32
from paper_1903_03056_gb300 import build, dgfs, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    build.build()
    dgfs.load()


def _inputs(N, L, masses, B, seed):
    w = synth.Workload("noalloc", B, N, L, tuple(masses), 0.5, 1.0, 6, 4, "bimaxwellian", 0.05, seed)
    return synth.batch_distribution(w, dtype=np.float32)


@pytest.mark.parametrize("N,L,masses,omega,M,N_rho,B", [
    (16, 6.0, (1.0, 2.0), 0.5, 12, 8, 70),
    (12, 5.0, (1.0, 1.5, 2.6), 0.74, 6, 4, 5),
])
def test_noalloc_matches_plan_path_on_two_calls(N, L, masses, omega, M, N_rho, B):
    import torch
    plan = dgfs.Plan(N, L, list(masses), omega, M=M, N_rho=N_rho, precision="fp32")
    desc, keep = dgfs.make_desc(N, L, list(masses), omega, M=M, N_rho=N_rho, precision="fp32")
    s = len(masses)
    for call, seed in enumerate((11, 12)):
        f = torch.from_numpy(_inputs(N, L, masses, B, seed)).cuda()
        ref = plan.eval(f)
        Q = torch.full((B, s, s, N, N, N), float("nan"), dtype=torch.float32, device="cuda")
        free_before = torch.cuda.mem_get_info()[0]
        code = dgfs.dgfs_eval_collision_noalloc(desc, f.data_ptr(), Q.data_ptr(), B, None)
        torch.cuda.synchronize()
        assert code == dgfs.DGFS_OK, dgfs.dgfs_strerror(code)
        if call > 0:  # the first call on the device performs the one-time set-up
            assert torch.cuda.mem_get_info()[0] == free_before
        err = max_rel_error(Q.double().cpu().numpy(), ref.double().cpu().numpy(), "node")
        assert err < TOL_FP32, (call, err)
    plan.close()
    del keep


@pytest.mark.parametrize("kw,code", [
    (dict(N=32), dgfs.DGFS_ERR_UNSUPPORTED_N),
    (dict(N=24), dgfs.DGFS_ERR_UNSUPPORTED_N),
    (dict(masses=[1.0, 2.0, 3.0, 4.0]), dgfs.DGFS_ERR_UNSUPPORTED),
    (dict(M=32), dgfs.DGFS_ERR_UNSUPPORTED),
    (dict(N_rho=17), dgfs.DGFS_ERR_UNSUPPORTED),
    (dict(precision="fp64"), dgfs.DGFS_ERR_UNSUPPORTED),
])
def test_noalloc_rejects_sizes_beyond_its_limits(kw, code):
    import torch
    base = dict(N=16, L=6.0, masses=[1.0, 2.0], omega=0.5, M=12, N_rho=8, precision="fp32")
    base.update(kw)
    N, L, masses, omega = base.pop("N"), base.pop("L"), base.pop("masses"), base.pop("omega")
    desc, keep = dgfs.make_desc(N, L, masses, omega, **base)
    buf = torch.zeros(16, dtype=torch.float32, device="cuda")
    assert dgfs.dgfs_eval_collision_noalloc(desc, buf.data_ptr(), buf.data_ptr(), 1, None) == code
