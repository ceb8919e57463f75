"""DGFS_BF16X3: the transforms of Sec. 4 as tensor-core matrix products with every FP32 operand
split into three BF16 terms.

* The batched 3D DFT building block against numpy's FFT (N = 8, 16, 24; both directions;
  ragged batch counts).
* The collision operator against the FP64 oracle at the FP32 bar (1e-5 of the node's max |Q|):
  N = 8, 16 and 24, two and three species, a user rule without antipodes, and the N = 24
  hard-sphere workload's parameters on a few nodes.
* The 16384-node N = 24 hard-sphere batch at full size in the launch configuration that
  run_case times: sampled nodes against the oracle.
"""

import numpy as np
import pytest

from gpu_helpers import TOL_FP32, gpu_collision, max_rel_error, oracle_collision
from paper_1903_03056_gb300 import build, dgfs, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    build.build()
    dgfs.load()


@pytest.mark.parametrize("N", [8, 16, 24])
@pytest.mark.parametrize("direction", [-1, 1])
def test_dft3_matches_numpy_fft(N, direction):
    import torch
    rng = np.random.default_rng(N + 7 * direction)
    count = 5
    x = (rng.normal(size=(count, N, N, N)) + 1j * rng.normal(size=(count, N, N, N))).astype(np.complex64)
    xd = torch.from_numpy(x).cuda()
    yd = torch.full_like(xd, complex(float("nan"), float("nan")))
    code = dgfs.dgfs_dft3_bf16x3(N, direction, xd.data_ptr(), yd.data_ptr(), count, None)
    assert code == dgfs.DGFS_OK, dgfs.dgfs_strerror(code)
    y = yd.cpu().numpy().astype(np.complex128)
    xx = x.astype(np.complex128)
    ref = np.fft.fftn(xx, axes=(1, 2, 3)) if direction < 0 else np.fft.ifftn(xx, axes=(1, 2, 3)) * N ** 3
    err = np.max(np.abs(y - ref)) / np.max(np.abs(ref))
    print("N=%d dir=%+d: max error / max |y| = %.3e" % (N, direction, err))
    assert err < 2e-6


def test_dft3_rejects_unsupported_sizes():
    import torch
    buf = torch.zeros(64, dtype=torch.complex64, device="cuda")
    assert dgfs.dgfs_dft3_bf16x3(32, 1, buf.data_ptr(), buf.data_ptr(), 1, None) == dgfs.DGFS_ERR_UNSUPPORTED_N
    assert dgfs.dgfs_dft3_bf16x3(8, 2, buf.data_ptr(), buf.data_ptr(), 1, None) == dgfs.DGFS_ERR_INVALID_ARG
    assert dgfs.dgfs_dft3_bf16x3(8, 1, buf.data_ptr(), buf.data_ptr(), 0, None) == dgfs.DGFS_OK


def _inputs(N, L, masses, B, seed, recipe="bimaxwellian"):
    w = synth.Workload("bf16x3", B, N, L, tuple(masses), 0.5, 1.0, 12, 4, recipe, 0.05, seed)
    return synth.batch_distribution(w)


CASES = {
    "n8_two_species": dict(N=8, L=4.0, masses=(1.0, 2.0), omega=0.7, M=6, N_rho=3, B=3),
    "n16_three_species": dict(N=16, L=6.0, masses=(1.0, 1.5, 2.6), omega=0.74, M=12, N_rho=4, B=2),
    "n24_hard_sphere_mass_ratio_4": dict(N=24, L=6.0, masses=(1.0, 4.0), omega=0.5, M=12, N_rho=12, B=2),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_bf16x3_collision_parity_with_oracle(name):
    kw = dict(CASES[name])
    B = kw.pop("B")
    f = _inputs(kw["N"], kw["L"], kw["masses"], B, seed=300 + kw["N"])
    Q = gpu_collision(f, precision="bf16x3", **kw)
    ref = oracle_collision(f, **kw)
    err = max_rel_error(Q, ref, "node")
    print("%s: bf16x3 error vs oracle per node %.3e" % (name, err))
    assert err < TOL_FP32


def test_bf16x3_non_antipodal_rule():
    """Ordered-pair tasks with the full rule (no reuse), a user radius."""
    rng = np.random.default_rng(31)
    sigma = rng.normal(size=(5, 3))
    sigma /= np.linalg.norm(sigma, axis=1, keepdims=True)
    kw = dict(N=8, L=4.0, masses=(1.0, 2.0), omega=0.8, N_rho=2, sigma=sigma,
              w_sigma=np.full(5, 4 * np.pi / 5), R=2.6)
    f = _inputs(8, 4.0, (1.0, 2.0), 2, seed=333)
    Q = gpu_collision(f, precision="bf16x3", **kw)
    ref = oracle_collision(f, **kw)
    assert max_rel_error(Q, ref, "node") < TOL_FP32


def test_bf16x3_rejects_vss_and_large_n():
    with pytest.raises(dgfs.DgfsError) as e:
        dgfs.Plan(32, 7.0, [1.0, 2.0], 0.7, M=6, N_rho=2, precision="bf16x3")
    assert e.value.code == dgfs.DGFS_ERR_UNSUPPORTED_N
    with pytest.raises(dgfs.DgfsError) as e:
        dgfs.Plan(16, 6.0, [1.0, 2.0], 0.7, alpha=1.4, M=6, N_rho=2, precision="bf16x3")
    assert e.value.code == dgfs.DGFS_ERR_UNSUPPORTED


def test_bf16x3_full_hs_batch_sampled_nodes():
    """The 16384-node N = 24 hard-sphere batch in one launch; the first, a middle and the last
    node against the oracle, and the batch against the FP32 FFT path."""
    import torch
    w = synth.WORKLOADS["hs_n24"]
    f = synth.batch_distribution(w)
    fd = torch.from_numpy(f.astype(np.float32)).cuda()
    plan = dgfs.Plan(w.N, w.L, list(w.masses), w.omega, alpha=w.alpha, M=w.M, N_rho=w.N_rho,
                     precision="bf16x3")
    Q = plan.eval(fd)
    torch.cuda.synchronize()
    assert plan.check()
    plan.close()
    assert bool(torch.isfinite(Q).all())
    nodes = [0, 8191, w.batch - 1]
    sample = Q[nodes].double().cpu().numpy()
    p32 = dgfs.Plan(w.N, w.L, list(w.masses), w.omega, alpha=w.alpha, M=w.M, N_rho=w.N_rho, precision="fp32")
    Q32 = p32.eval(fd)
    torch.cuda.synchronize()
    p32.close()
    err32 = float(((Q - Q32).abs().amax(dim=(1, 2, 3, 4, 5)) / Q32.abs().amax(dim=(1, 2, 3, 4, 5))).max())
    del Q, Q32, fd
    from oracle import fast_spectral as fs
    prob = fs.make_problem(w.N, w.L, list(w.masses), omega=w.omega, alpha=w.alpha, M=w.M, N_rho=w.N_rho)
    ref = np.stack([fs.collision(f[b], prob)[0] for b in nodes])
    err = max_rel_error(sample, ref, "node")
    print("hs_n24 bf16x3: error vs oracle per node %.3e, vs the FP32 path over the batch %.3e" % (err, err32))
    assert err < TOL_FP32
    assert err32 < 2 * TOL_FP32


def test_bounded_wait_gives_up_and_reports():
    """The tensor-core kernels' wait on an mbarrier gives up after its limit and reports the
    timeout instead of hanging; the context stays usable afterwards."""
    import time
    import torch
    t0 = time.perf_counter()
    assert dgfs.dgfs_check_bounded_wait(0.05) == dgfs.DGFS_ERR_DEVICE_TIMEOUT
    assert time.perf_counter() - t0 < 5.0
    x = torch.ones(8, device="cuda")
    assert float((x * 2).sum()) == 16.0
    assert dgfs.dgfs_check_bounded_wait(0.0) == dgfs.DGFS_ERR_INVALID_ARG


def test_bf16x3_graph_replay_matches_direct_launch():
    """The tensor-core evaluation (counter reset, kernel) is stream-ordered and capturable: a
    replayed CUDA graph computes the same bits as the direct launch, also after the input
    changes in place."""
    import torch
    f = torch.from_numpy(_inputs(16, 6.0, (1.0, 2.0), 3, seed=351)).float().cuda()
    plan = dgfs.Plan(16, 6.0, [1.0, 2.0], 0.5, M=12, N_rho=4, precision="bf16x3")
    Q = torch.empty((3, 2, 2, 16, 16, 16), dtype=torch.float32, device="cuda")
    g = plan.capture(f, Q)
    for k in range(2):
        f.mul_(1.0 + 0.5 * k)
        ref = plan.eval(f).clone()
        Q.zero_()
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(Q, ref)
    assert plan.check()
    plan.close()


def test_bf16x3_per_pair_truncation_and_loss_rule_against_oracle():
    """Ordered-pair tasks with their own radial rules (DGFS_PER_PAIR_R) and the loss weight's
    own radial rule (DGFS_LOSS_ACCURATE) through the tensor-core precision."""
    kw = dict(N=8, L=4.0, masses=(1.0, 3.0), omega=0.7, M=6, N_rho=3)
    f = _inputs(8, 4.0, (1.0, 3.0), 2, seed=355)
    Q = gpu_collision(f, precision="bf16x3", flags=dgfs.DGFS_PER_PAIR_R | dgfs.DGFS_LOSS_ACCURATE, **kw)
    ref = oracle_collision(f, pair_radius=True, loss_rule="accurate", **kw)
    assert max_rel_error(Q, ref, "node") < TOL_FP32


def test_bf16x3_ssp_rk2_step_against_oracle():
    """One homogeneous SSP-RK2 step (two species-summed evaluations and the stage kernels) with a
    tensor-core plan, against the oracle's step, at the FP32 bar of the step's change."""
    import torch
    from oracle import fast_spectral as fs, homogeneous
    N, L, masses = 8, 4.0, [1.0, 2.0]
    kappa = np.array([[1.0, 0.8], [1.3, 1.0]])
    f = _inputs(N, L, masses, 2, seed=357)
    plan = dgfs.Plan(N, L, masses, 0.6, M=6, N_rho=3, precision="bf16x3", kappa=kappa,
                     flags=dgfs.DGFS_SUM_SPECIES, max_batch=2)
    fd = torch.from_numpy(f.astype(np.float32)).cuda()
    plan.ssp_rk2_step(fd, 0.05)
    torch.cuda.synchronize()
    plan.close()
    prob = fs.make_problem(N, L, masses, omega=0.6, M=6, N_rho=3)
    ref = np.stack([homogeneous.ssp_rk2_step(fb, 0.05, homogeneous.collision_rhs(prob, kappa)) for fb in f])
    change = np.max(np.abs(ref - f))
    assert np.max(np.abs(fd.cpu().numpy() - ref)) < 1e-4 * change + 1e-6 * np.max(np.abs(ref))
