"""Shared helpers of the GPU parity tests: run the CUDA path through the C ABI and the
oracle on the same seeded inputs."""

import numpy as np

from oracle import fast_spectral as fs
from paper_1903_03056_gb300 import dgfs

# mixed-precision bound of the FP32 path relative to max |Q| (the stated target) and the
# FP64 path's bound against the FP64 oracle
TOL_FP32 = 1e-5
TOL_FP64 = 1e-11


def gpu_collision(f, *, N, L, masses, omega, M=12, N_rho=8, precision="fp64", sigma=None,
                  w_sigma=None, b_override=None, R=0.0, alpha=1.0, flags=0):
    """f: numpy [B, s, N, N, N] float64 -> Q numpy [B, s, s, N, N, N] from libdgfs."""
    import torch
    dt = torch.float64 if precision == "fp64" else torch.float32
    plan = dgfs.Plan(N, L, masses, omega, alpha=alpha, M=M, N_rho=N_rho, precision=precision,
                     sigma=sigma, w_sigma=w_sigma, b_override=b_override, R=R, flags=flags)
    fd = torch.from_numpy(np.ascontiguousarray(f)).to(device="cuda", dtype=dt)
    f_before = fd.clone()
    # Q between two margins of a sentinel value: nothing outside Q may be written, every
    # element of Q must be
    B, s = f.shape[0], len(masses)
    n_out = B * s * s * N ** 3
    pad = 4096
    buf = torch.full((n_out + 2 * pad,), 1.25e30, dtype=dt, device="cuda")
    Q = buf[pad:pad + n_out].view(B, s, s, N, N, N)
    plan.eval(fd, Q)
    torch.cuda.synchronize()
    assert plan.launches() == 1
    assert plan.check(), "a kernel wrote outside the plan's workspace"
    assert bool((buf[:pad] == 1.25e30).all()) and bool((buf[pad + n_out:] == 1.25e30).all()), \
        "a kernel wrote outside Q"
    assert not bool((Q == 1.25e30).any()), "an element of Q was not written"
    assert torch.equal(fd, f_before), "the input was modified"
    out = Q.double().cpu().numpy()
    plan.close()
    return out


def oracle_collision(f, *, N, L, masses, omega, M=12, N_rho=8, sigma=None, w_sigma=None,
                     b_override=None, R=None, alpha=1.0, loss_rule="same", pair_radius=False):
    prob = fs.make_problem(N, L, masses, omega=omega, alpha=alpha, M=M, N_rho=N_rho, sigma=sigma,
                           w_sigma=w_sigma, b_override=b_override, R=R, loss_rule=loss_rule,
                           pair_radius=pair_radius)
    return np.stack([fs.collision(fb, prob)[0] for fb in f])


def max_rel_error(Q_gpu, Q_ref, per="pair"):
    """Largest max|Q_gpu - Q_ref| / scale over nodes and pairs.

    per="pair": scale = max|Q_ref| of the same node and pair (the FP64 bar);
    per="node": scale = max|Q_ref| over all s^2 operators of the node (the FP32 bar: a pair
    whose gain and loss nearly cancel keeps the absolute FP32 error of the larger terms).
    """
    err = 0.0
    for b in range(Q_ref.shape[0]):
        node_scale = np.max(np.abs(Q_ref[b]))
        for i in range(Q_ref.shape[1]):
            for j in range(Q_ref.shape[2]):
                scale = np.max(np.abs(Q_ref[b, i, j])) if per == "pair" else node_scale
                err = max(err, np.max(np.abs(Q_gpu[b, i, j] - Q_ref[b, i, j])) / scale)
    return err


def check(Q_gpu, Q_ref, precision):
    if precision == "fp64":
        return max_rel_error(Q_gpu, Q_ref, "pair") < TOL_FP64
    return max_rel_error(Q_gpu, Q_ref, "node") < TOL_FP32


def oracle_node_of_workload(args):
    """(workload key, node) -> the oracle's Q of that node of the seeded workload (for spawned
    worker processes: single-threaded BLAS, imports inside)."""
    import os
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
    from paper_1903_03056_gb300 import synth
    key, node = args
    w = synth.WORKLOADS[key]
    prob = fs.make_problem(w.N, w.L, list(w.masses), omega=w.omega, alpha=w.alpha, M=w.M, N_rho=w.N_rho)
    return fs.collision(synth.node_distribution(w, node), prob)[0]
