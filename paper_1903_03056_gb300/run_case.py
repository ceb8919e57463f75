"""Evaluate one synthetic workload a few times (for profiling a single kernel launch).

    python -m paper_1903_03056_gb300.run_case --workload dg_batch_n32 --batch 288 \
        --precision fp32 --repeat 3

Prints one JSON line with the mean time per evaluation measured with CUDA events.
"""

import argparse
import json


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="dg_batch_n32")
    ap.add_argument("--batch", type=int, default=None)
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64", "bf16x3"])
    ap.add_argument("--repeat", type=int, default=3)
    ap.add_argument("--checksum", action="store_true", help="add the SHA-1 of the output bytes")
    ap.add_argument("--compare-fp64", type=int, default=0, metavar="K",
                    help="also evaluate the first K nodes with an FP64 plan and report the largest "
                         "per-node max |Q - Q_fp64| / max |Q_fp64|")
    ap.add_argument("--n-rho", type=int, default=None,
                    help="override the workload's radial nodes (smaller tables for profiling)")
    a = ap.parse_args()

    import torch

    from paper_1903_03056_gb300 import build, dgfs, synth

    build.build()
    w = synth.WORKLOADS[a.workload]
    if a.n_rho is not None:
        import dataclasses
        w = dataclasses.replace(w, N_rho=a.n_rho)
    B = a.batch or w.batch
    f = synth.batch_distribution(w, nodes=range(B))
    dt = torch.float64 if a.precision == "fp64" else torch.float32
    fd = torch.from_numpy(f).to(device="cuda", dtype=dt)
    Q = torch.empty((B, w.s, w.s, w.N, w.N, w.N), dtype=dt, device="cuda")
    import time
    t0 = time.perf_counter()
    plan = dgfs.Plan(w.N, w.L, list(w.masses), w.omega, alpha=w.alpha, M=w.M, N_rho=w.N_rho,
                     precision=a.precision)
    plan_s = time.perf_counter() - t0
    tables, workspace = plan.bytes(0)
    st = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(st)
    for _ in range(a.repeat):
        plan.eval_ptr(fd.data_ptr(), Q.data_ptr(), B, st)
    ev1.record(st)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / a.repeat
    out = {"workload": w.name, "batch": B, "precision": a.precision, "ms": ms,
           "evals_per_s": B / (ms * 1e-3), "finite": bool(torch.isfinite(Q).all()),
           "plan_s": plan_s, "table_bytes": tables, "workspace_bytes": workspace}
    if a.checksum:
        import hashlib
        out["sha1"] = hashlib.sha1(Q.cpu().numpy().tobytes()).hexdigest()
    if a.compare_fp64 > 0:
        K = min(a.compare_fp64, B)
        p64 = dgfs.Plan(w.N, w.L, list(w.masses), w.omega, alpha=w.alpha, M=w.M, N_rho=w.N_rho, precision="fp64")
        Q64 = p64.eval(fd[:K].double().contiguous())
        torch.cuda.synchronize()
        p64.close()
        dims = tuple(range(1, Q64.dim()))
        err = ((Q[:K].double() - Q64).abs().amax(dim=dims) / Q64.abs().amax(dim=dims)).max()
        out["err_vs_fp64"] = float(err)
    print(json.dumps(out))
    plan.close()


if __name__ == "__main__":
    main()
