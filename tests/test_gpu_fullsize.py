"""Full-size batches in the launch configuration that bench.py and run_case time.

* 4096-node N=32^3 batch (the bench workload) and 16384-node N=24^3 hard-sphere batch:
  sampled nodes (first, second, middle, last) against the oracle one by one, plus finite
  output; FP32 and FP64 paths, each on the whole batch.
* 1024-node N=48^3 three-species VSS batch: the oracle's VSS gain table alone would take
  tens of minutes per node at this size, so it is checked through properties that hold at
  any size.  The FP32 batch agrees with the FP64 path on sampled nodes (the FP64 VSS path is
  pinned to the oracle at small N), and a node evaluated inside the batch is bitwise equal to
  the same node evaluated alone.
"""

import numpy as np
import pytest

from gpu_helpers import TOL_FP32, TOL_FP64, max_rel_error, oracle_node_of_workload
from oracle import fast_spectral as fs
from paper_1903_03056_gb300 import build, dgfs, synth

pytestmark = pytest.mark.gpu

_INPUTS = {}


def _inputs(key):
    if key not in _INPUTS:
        build.build()
        dgfs.load()
        _INPUTS.clear()  # keep one batch in host memory at a time
        _INPUTS[key] = synth.batch_distribution(synth.WORKLOADS[key])
    return _INPUTS[key]


def _plan(w, precision):
    return dgfs.Plan(w.N, w.L, list(w.masses), w.omega, alpha=w.alpha, M=w.M, N_rho=w.N_rho,
                     precision=precision)


def _oracle_nodes(w, f, nodes):
    prob = fs.make_problem(w.N, w.L, list(w.masses), omega=w.omega, alpha=w.alpha, M=w.M,
                           N_rho=w.N_rho)
    return np.stack([fs.collision(f[b], prob)[0] for b in nodes])


def _eval(w, f, precision, nodes=None):
    """Evaluate the whole batch (nodes=None) or only the listed nodes; returns a torch tensor."""
    import torch
    dt = torch.float64 if precision == "fp64" else torch.float32
    plan = _plan(w, precision)
    src = f if nodes is None else f[nodes]
    fd = torch.from_numpy(np.ascontiguousarray(src)).to(device="cuda", dtype=dt)
    Q = plan.eval(fd)
    torch.cuda.synchronize()
    assert plan.check(), "a kernel wrote outside the plan's workspace"
    plan.close()
    return Q


@pytest.mark.parametrize("key,precision,nodes", [
    ("dg_batch_n32", "fp32", [0, 1, 2047, 4095]),
    ("dg_batch_n32", "fp64", [0, 4095]),
    ("hs_n24", "fp32", [0, 1, 8191, 16383]),
    ("hs_n24", "fp64", [0, 16383]),
])
def test_full_batch_sampled_nodes(key, precision, nodes):
    import torch
    w = synth.WORKLOADS[key]
    f = _inputs(key)
    Q = _eval(w, f, precision)
    assert bool(torch.isfinite(Q).all())
    sample = Q[nodes].double().cpu().numpy()
    del Q
    ref = _oracle_nodes(w, f, nodes)
    if precision == "fp32":
        err_node = max_rel_error(sample, ref, "node")
        err_pair = max_rel_error(sample, ref, "pair")
        print("%s fp32 error vs oracle: per node %.3e, per pair %.3e" % (key, err_node, err_pair))
        assert err_node < TOL_FP32
    else:
        err = max_rel_error(sample, ref, "pair")
        print("%s fp64 error vs oracle: per pair %.3e" % (key, err))
        assert err < TOL_FP64


def test_vss_n48_full_batch_properties():
    import torch
    w = synth.WORKLOADS["vss_n48"]
    f = _inputs("vss_n48")
    nodes = [0, w.batch - 1]
    Q = _eval(w, f, "fp32")
    assert bool(torch.isfinite(Q).all())
    sample = Q[nodes].cpu()
    del Q
    # the same nodes alone: bitwise equal (work items do not interact)
    alone = _eval(w, f, "fp32", nodes).cpu()
    assert torch.equal(sample, alone)
    # against the FP64 path on the same nodes
    ref = _eval(w, f, "fp64", nodes).cpu().numpy()
    err = max_rel_error(sample.double().numpy(), ref, "node")
    print("vss_n48 fp32 vs fp64 path: per node %.3e" % err)
    assert err < TOL_FP32


@pytest.mark.parametrize("precision", ["fp32", "bf16x3"])
def test_hs_n24_64_node_subsample_against_the_oracle(precision):
    """The error of the 16384-node N = 24 batch, evaluated whole in one launch, on its first 64
    nodes against the oracle (the subsample the workload's error is stated on); the oracle runs
    in a spawn pool of worker processes."""
    import multiprocessing as mp
    import os
    w = synth.WORKLOADS["hs_n24"]
    f = _inputs("hs_n24")
    Q = _eval(w, f, precision)
    sample = Q[:64].double().cpu().numpy()
    del Q
    key = "hs_n24_oracle_64"
    if key not in _ORACLE_CACHE:
        # one BLAS thread per worker: the limits are set before the workers start (they import
        # numpy on start-up), else every worker's BLAS spawns a thread per core
        saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
        for k in saved:
            os.environ[k] = "1"
        try:
            with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
                _ORACLE_CACHE[key] = np.stack(pool.map(oracle_node_of_workload, [("hs_n24", b) for b in range(64)]))
        finally:
            for k, v in saved.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v
    err = max_rel_error(sample, _ORACLE_CACHE[key], "node")
    print("hs_n24 %s: 64-node subsample, error vs oracle per node %.3e" % (precision, err))
    assert err < TOL_FP32


_ORACLE_CACHE = {}
