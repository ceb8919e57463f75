"""Time the 1D DG transport kernel and the full RKDG step (dgfs_dg_transport, dgfs_dg_step).

    python -m paper_1903_03056_gb300.run_dg --Ne 1024 --K 4 --N 32 --precision fp32

Inputs: a seeded two-species state of bi-Maxwellians (synth) at every node, between Maxwell
walls.  Prints one JSON line: transport time and achieved bandwidth (algorithmic bytes: the
state read once and the right-hand side written once), and the time of one full step
(two transport passes and two collision evaluations of Ne*K nodes).
"""

import argparse
import json


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--Ne", type=int, default=1024)
    ap.add_argument("--K", type=int, default=4)
    ap.add_argument("--N", type=int, default=32)
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--repeat", type=int, default=5)
    ap.add_argument("--steps", type=int, default=1, help="full RKDG steps to time (0: none)")
    a = ap.parse_args()

    import numpy as np
    import torch

    from paper_1903_03056_gb300 import build, dgfs, synth

    build.build()
    B = a.Ne * a.K
    L = {16: 6.0, 24: 6.0, 32: 7.0, 48: 8.0}.get(a.N, 6.0)
    w = synth.Workload("dg state", min(B, 64), a.N, L, (1.0, 2.1), 0.81, 1.0, 12, a.N // 2,
                       "bimaxwellian", 0.05, 7000)
    pool = synth.batch_distribution(w)
    f = np.concatenate([pool] * (B // len(pool) + 1))[:B]
    dt = torch.float32 if a.precision == "fp32" else torch.float64
    fd = torch.from_numpy(f).to("cuda", dt).contiguous()
    coll = dgfs.Plan(a.N, L, list(w.masses), w.omega, M=w.M, N_rho=w.N_rho, precision=a.precision,
                     flags=dgfs.DGFS_SUM_SPECIES, max_batch=B)
    dg = dgfs.DGPlan(coll, a.Ne, a.K, 0.0, 1.0, bc="walls", Tw=(0.9, 1.2),
                     uw=((0.0, 0.2, 0.0), (0.0, -0.2, 0.0)), acc=(1.0, 1.0))
    rhs = torch.empty_like(fd)
    st = torch.cuda.current_stream()
    for _ in range(2):
        dg.transport(fd, rhs, st)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(st)
    for _ in range(a.repeat):
        dg.transport(fd, rhs, st)
    ev1.record(st)
    torch.cuda.synchronize()
    t_ms = ev0.elapsed_time(ev1) / a.repeat
    nbytes = 2 * fd.numel() * fd.element_size()
    out = {"Ne": a.Ne, "K": a.K, "N": a.N, "species": 2, "nodes": B, "precision": a.precision,
           "transport_ms": t_ms, "transport_bytes": nbytes, "transport_GBps": nbytes / (t_ms * 1e-3) / 1e9,
           "finite": bool(torch.isfinite(rhs).all())}
    if a.steps > 0:
        ev0.record(st)
        for _ in range(a.steps):
            dg.step(fd, 1e-3, st)
        ev1.record(st)
        torch.cuda.synchronize()
        out["step_ms"] = ev0.elapsed_time(ev1) / a.steps
        out["step_finite"] = bool(torch.isfinite(fd).all())
    print(json.dumps(out))
    dg.close()
    coll.close()


if __name__ == "__main__":
    main()
