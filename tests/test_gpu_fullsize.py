"""The 4096-node N=32^3 batch in the launch configuration bench.py times: sampled nodes
(first, second, middle, last) against the oracle one by one, and properties that hold at any
size (finite output, identical repeat)."""

import numpy as np
import pytest

from gpu_helpers import TOL_FP32, TOL_FP64, max_rel_error
from oracle import fast_spectral as fs
from paper_1903_03056_gb300 import build, dgfs, synth

pytestmark = pytest.mark.gpu

W = synth.WORKLOADS["dg_batch_n32"]


@pytest.fixture(scope="module")
def batch_inputs():
    build.build()
    dgfs.load()
    return synth.batch_distribution(W)


def _oracle_nodes(f, nodes):
    prob = fs.make_problem(W.N, W.L, list(W.masses), omega=W.omega, alpha=W.alpha, M=W.M,
                           N_rho=W.N_rho)
    return np.stack([fs.collision(f[b], prob)[0] for b in nodes])


@pytest.mark.parametrize("precision,nodes", [("fp32", [0, 1, 2047, 4095]), ("fp64", [0, 4095])])
def test_full_batch_sampled_nodes(batch_inputs, precision, nodes):
    import torch
    dt = torch.float32 if precision == "fp32" else torch.float64
    plan = dgfs.Plan(W.N, W.L, list(W.masses), W.omega, alpha=W.alpha, M=W.M, N_rho=W.N_rho,
                     precision=precision)
    fd = torch.from_numpy(batch_inputs).to(device="cuda", dtype=dt)
    Q = plan.eval(fd)
    torch.cuda.synchronize()
    assert bool(torch.isfinite(Q).all())
    sample = Q[nodes].double().cpu().numpy()
    del Q
    ref = _oracle_nodes(batch_inputs, nodes)
    if precision == "fp32":
        err_node = max_rel_error(sample, ref, "node")
        err_pair = max_rel_error(sample, ref, "pair")
        print("fp32 error vs oracle: per node %.3e, per pair %.3e" % (err_node, err_pair))
        assert err_node < TOL_FP32
    else:
        err = max_rel_error(sample, ref, "pair")
        print("fp64 error vs oracle: per pair %.3e" % err)
        assert err < TOL_FP64
    plan.close()
